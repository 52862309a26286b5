"""Replicas-only multi-process path of bench.py, on CPU with the gloo backend
(world size 2): the whole-job rate is all ranks' cell-updates over the slowest
rank's time, and only a barrier / max / sum cross the ranks."""
import os
import socket
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    ms_local = [100.0, 250.0][rank]
    cells = [2_000_000, 2_000_000][rank]
    ms, value = bench.replica_aggregate(dist, cells, 10, ms_local, device="cpu")
    dist.barrier()
    out[rank] = (ms, value)
    dist.destroy_process_group()


def test_replica_aggregate_two_ranks():
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    for r in range(2):
        ms, value = out[r]
        assert ms == 250.0
        assert abs(value - 4_000_000 * 10 / 0.25) < 1e-6


def test_replica_aggregate_single_process():
    sys.path.insert(0, ROOT)
    import bench
    ms, value = bench.replica_aggregate(None, 1000, 5, 2.0)
    assert ms == 2.0 and value == 1000 * 5 / 0.002
