"""Request server: runs of different mesh sizes submitted while others are on the
GPU are admitted as memory and slots free up, stepped together (continuous
batching), and each result equals the same run alone, bitwise."""
import time

import numpy as np
import pytest

import oracle
from paper_2102_12862_b300 import bm
from paper_2102_12862_b300 import workloads as W

pytestmark = pytest.mark.gpu


def scenarios():
    out = []
    for k in range(6):
        out.append(W.ensemble_instance(k, size_override=[3000, 9000, 1500, 12000, 5000, 800][k]))
    return out


def solo(mesh, s, t_end, precision):
    st = bm.State.from_scenario(s, mesh=mesh, precision=precision)
    st.run_until(t_end)
    H, qx, qy, t = st.download()
    return H, qx, qy


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_results_same_alone_and_in_the_mix(precision):
    scs = scenarios()
    meshes = [bm.Mesh.from_scenario(s) for s in scs]
    t_ends = [30.0, 12.0, 45.0, 8.0, 20.0, 60.0]
    sv = bm.Server(precision=precision, steps_per_round=16)
    tickets = []
    for k, s in enumerate(scs):
        prm = {key: val for key, val in s.params.items()}
        tickets.append(sv.submit(meshes[k], s.H, s.qx, s.qy, t_end=t_ends[k], **prm))
        time.sleep(0.01 * k)  # arrivals while earlier runs are on the GPU
    results = [sv.wait(tk, 300.0) for tk in tickets]
    for k, (s, r) in enumerate(zip(scs, results)):
        H, qx, qy, lat = r
        assert lat > 0
        Hs, qxs, qys = solo(meshes[k], s, t_ends[k], precision)
        assert np.array_equal(H, Hs), f"run {k}: H differs from the solo run"
        assert np.array_equal(qx, qxs) and np.array_equal(qy, qys), f"run {k}: q differs"
        # and the served result against the FP64 oracle run to the same end time:
        # FP64 element by element (relative L-inf of h, hu, hv), FP32-bulk at its
        # L1 depth bar
        o = oracle.Oracle(s)
        o.run_until(t_ends[k])
        if precision == "fp64":
            tol = 1e-11 if o.steps <= 400 else 1e-10
            for a, b in ((H - s.z, o.depth()), (qx, o.qx), (qy, o.qy)):
                assert np.max(np.abs(a - b)) <= tol * max(np.max(np.abs(b)), 1e-300), f"run {k} vs oracle"
        else:
            area = o.area()
            assert np.sum(area * np.abs((H - s.z) - o.depth())) / area.sum() <= 1e-4, f"run {k} vs oracle"
    st = sv.stats()
    assert st["completed"] == len(scs) and st["running"] == 0 and st["queued"] == 0
    assert st["cell_updates"] > 0
    sv.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_tracked_runs_in_the_mix(precision):
    """Flood tracking as a serving output: tracked and untracked runs share the batches;
    each tracked run's record equals the same run alone, bitwise."""
    scs = scenarios()[:4]
    meshes = [bm.Mesh.from_scenario(s) for s in scs]
    t_ends = [25.0, 10.0, 40.0, 15.0]
    track = [0.05, None, 0.02, 0.1]
    sv = bm.Server(precision=precision, steps_per_round=16)
    tickets = [sv.submit(meshes[k], s.H, s.qx, s.qy, t_end=t_ends[k], track=track[k], **dict(s.params))
               for k, s in enumerate(scs)]
    for k, (s, tk) in enumerate(zip(scs, tickets)):
        bm.bm_server_wait(sv.handle, tk, 300.0)
        if track[k] is None:
            with pytest.raises(bm.BMError, match="without tracking"):
                sv.poll_track(tk)
        else:
            rec = sv.poll_track(tk)
            st = bm.State.from_scenario(s, mesh=meshes[k], precision=precision)
            st.track(track[k])
            st.run_until(t_ends[k])
            ref = st.download_track()
            for f in ref:
                assert np.array_equal(rec[f], ref[f], equal_nan=True), f"run {k}: {f}"
            assert np.nanmax(rec["t_arrival"]) > 0  # the flood front moved
        assert sv.poll(tk) is not None
    sv.close()


def test_admission_by_budget_and_slots():
    scs = scenarios()
    meshes = [bm.Mesh.from_scenario(s) for s in scs]
    # a budget for about two of these runs at a time, and at most two slots
    sv = bm.Server(precision="fp32", hbm_budget_bytes=3_000_000, max_slots=2, steps_per_round=8)
    tks = [sv.submit(m, s.H, s.qx, s.qy, t_end=15.0, **s.params) for m, s in zip(meshes, scs)]
    seen_queue = False
    for _ in range(200):
        stt = sv.stats()
        assert stt["running"] <= 2
        assert stt["resident_bytes"] <= 3_000_000
        seen_queue |= stt["queued"] > 0
        if stt["completed"] == len(scs):
            break
        time.sleep(0.01)
    for tk in tks:
        assert sv.wait(tk, 300.0) is not None
    assert seen_queue
    sv.close()


def test_server_errors():
    s = W.dam_break(nx=20, ny=4)
    mesh = bm.Mesh.from_scenario(s)
    sv = bm.Server(precision="fp32", hbm_budget_bytes=10_000)
    with pytest.raises(bm.BMError) as ei:
        sv.submit(mesh, s.H, s.qx, s.qy, t_end=1.0, precision="fp64")
    assert ei.value.status == bm.BM_EINVAL
    with pytest.raises(bm.BMError) as ei:
        sv.submit(mesh, s.H, s.qx, s.qy, t_end=1.0)
    assert ei.value.status == bm.BM_ENOMEM  # alone larger than the budget
    with pytest.raises(bm.BMError) as ei:
        bm.bm_poll(sv.handle, 12345, mesh.n_cells)
    assert ei.value.status == bm.BM_EINVAL
    sv.close()
    # a run still in flight when the server goes away does not hang or crash
    big = W.floodplain(nx=200, ny=80, Lx=2000.0, Ly=800.0, seed=61)
    bmesh = bm.Mesh.from_scenario(big)
    sv = bm.Server(precision="fp32")
    tk = sv.submit(bmesh, big.H, big.qx, big.qy, t_end=1e6, **big.params)
    assert sv.poll(tk) is None  # BM_EAGAIN right after submission
    sv.close()
