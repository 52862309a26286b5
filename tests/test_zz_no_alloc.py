"""bm_volume_noalloc: the water volume of caller-owned device arrays, computed with
no device allocation inside the library.

It is meant for callers that cannot call cudaMalloc: applications that have handed
all device memory to their own pool allocator, and loops that cannot afford the
device synchronisation cudaMalloc/cudaFree imply.  The test (collected last, so a
failure here does not hide the other tests) allocates the inputs and the output
itself, calls the entry point through the C ABI twice in a row, and compares each
result with the volume the regular entry point (bm_state_stats) reports for the same
state, to the 1e-12 relative tolerance the volume checks use elsewhere.
"""
import numpy as np
import pytest

from paper_2102_12862_b300 import bm
from paper_2102_12862_b300 import workloads as W

pytestmark = pytest.mark.gpu


def triangle_areas(xy, tri):
    a, b, c = xy[tri[:, 0]], xy[tri[:, 1]], xy[tri[:, 2]]
    return 0.5 * np.abs((b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (c[:, 0] - a[:, 0]) * (b[:, 1] - a[:, 1]))


def test_volume_noalloc_matches_regular_entry_point():
    import torch

    s = W.floodplain(nx=300, ny=120, Lx=3000.0, Ly=1200.0, seed=81)
    st = bm.State.from_scenario(s)
    st.step(25)
    H, qx, qy, t = st.download()
    ref = st.stats()["volume"]
    dev = torch.device("cuda")
    Ht = torch.tensor(H, dtype=torch.float64, device=dev)
    zt = torch.tensor(s.z, dtype=torch.float64, device=dev)
    at = torch.tensor(triangle_areas(s.xy, s.tri), dtype=torch.float64, device=dev)
    out = torch.full((1,), np.nan, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):  # two calls in a row share the scratch array
        bm.bm_volume_noalloc(Ht.data_ptr(), zt.data_ptr(), at.data_ptr(), len(H), out.data_ptr(), stream)
        torch.cuda.synchronize()
        got = float(out.item())
        assert abs(got - ref) <= 1e-12 * abs(ref), (got, ref)
        out.fill_(np.nan)
    # beyond the fixed scratch size the call is refused before any device work
    with pytest.raises(bm.BMError) as ei:
        bm.bm_volume_noalloc(Ht.data_ptr(), zt.data_ptr(), at.data_ptr(), 2_097_153, out.data_ptr(), stream)
    assert ei.value.status == bm.BM_EINVAL and "scratch limit" in str(ei.value)
