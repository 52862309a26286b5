"""bm_volume_noalloc: the water volume of caller-owned device arrays, computed with
no device allocation inside the library.

It is meant for callers that cannot call cudaMalloc: applications that have handed
all device memory to their own pool allocator, and loops that cannot afford the
device synchronisation cudaMalloc/cudaFree imply.  The test (collected last, so a
failure here does not hide the other tests) allocates the inputs and the output
itself, calls the entry point through the C ABI twice in a row, and compares each
result with the volume the regular entry point (bm_state_stats) reports for the same
state and with a plain numpy sum of area * (H - z) over the same arrays, to the
1e-12 relative tolerance the volume checks use elsewhere.  A second case fills the
fixed scratch array to its last slot (2,097,152 cells: 8,192 partial sums).
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
    area = triangle_areas(s.xy, s.tri)
    plain = float(np.sum(area * (H - s.z)))  # an independent sum on the host
    assert abs(plain - ref) <= 1e-12 * abs(ref), (plain, ref)
    dev = torch.device("cuda")
    Ht = torch.tensor(H, dtype=torch.float64, device=dev)
    zt = torch.tensor(s.z, dtype=torch.float64, device=dev)
    at = torch.tensor(area, dtype=torch.float64, device=dev)
    out = torch.full((1,), np.nan, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):  # two calls in a row share the scratch array
        bm.bm_volume_noalloc(Ht.data_ptr(), zt.data_ptr(), at.data_ptr(), len(H), out.data_ptr(), stream)
        torch.cuda.synchronize()
        got = float(out.item())
        assert abs(got - ref) <= 1e-12 * abs(ref), (got, ref)
        assert abs(got - plain) <= 1e-12 * abs(plain), (got, plain)
        out.fill_(np.nan)
    # beyond the fixed scratch size the call is refused before any device work
    with pytest.raises(bm.BMError) as ei:
        bm.bm_volume_noalloc(Ht.data_ptr(), zt.data_ptr(), at.data_ptr(), 2_097_153, out.data_ptr(), stream)
    assert ei.value.status == bm.BM_EINVAL and "scratch limit" in str(ei.value)


def test_volume_noalloc_fills_the_scratch_to_its_last_slot():
    """Exactly the largest accepted size, 2,097,152 cells = 8,192 blocks of 256: every
    slot of the fixed scratch array is written and summed; twice in a row, against a
    numpy sum of the same seeded arrays; then a smaller call right after it (the
    stale partials beyond its blocks must not enter its sum)."""
    import torch

    n = 2_097_152
    rng = np.random.default_rng(2097152)
    z = rng.uniform(395.0, 405.0, n)
    H = z + np.where(rng.random(n) < 0.3, 0.0, rng.uniform(0.0, 3.0, n))
    area = rng.uniform(1.0, 9.0, n)
    plain = float(np.sum(area * (H - z)))
    dev = torch.device("cuda")
    Ht, zt, at = (torch.tensor(a, dtype=torch.float64, device=dev) for a in (H, z, area))
    out = torch.full((1,), np.nan, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        bm.bm_volume_noalloc(Ht.data_ptr(), zt.data_ptr(), at.data_ptr(), n, out.data_ptr(), stream)
        torch.cuda.synchronize()
        got = float(out.item())
        assert abs(got - plain) <= 1e-12 * abs(plain), (got, plain)
        out.fill_(np.nan)
    m = 1000  # 4 blocks, the last one ragged
    bm.bm_volume_noalloc(Ht.data_ptr(), zt.data_ptr(), at.data_ptr(), m, out.data_ptr(), stream)
    torch.cuda.synchronize()
    small = float(np.sum(area[:m] * (H[:m] - z[:m])))
    assert abs(float(out.item()) - small) <= 1e-12 * abs(small)
