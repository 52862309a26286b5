"""Tile skipping: a step launch takes the fixed tiles (boundary edges that carry mass,
inflow, outflow or source cells, item 0) and the tiles the previous launch listed (those
that were not quiet and the tiles next to them); every other tile is dry, at rest and
has no changed neighbour, so its step would copy it through and the launch skips it.

Each case must end bitwise equal to the same run with skipping off (every tile stepped
by every launch): the skipped tiles' values are those the step would have written.
The cases cover moving wet/dry fronts in both precisions, flood tracking, a log-law
friction closure, sources, run_until (launches past an instance's end time), a state
that moves between its own list and a batch's, an upload in mid-run, and a dry closed
basin whose only work is item 0.
"""
import numpy as np
import pytest

from paper_2102_12862_b300 import bm
from paper_2102_12862_b300 import workloads as W

pytestmark = pytest.mark.gpu


def same(a, b):
    A, B = a.download(), b.download()
    for x, y in zip(A[:3], B[:3]):
        assert np.array_equal(x, y)
    assert A[3] == B[3]


def pair(s, **ov):
    a = bm.State.from_scenario(s, **ov)
    b = bm.State.from_scenario(s, **ov)
    b.set_tile_skipping(False)
    return a, b


def plain(seed=23, nx=160, ny=64):
    return W.floodplain(nx=nx, ny=ny, Lx=1600.0, Ly=640.0, seed=seed, q_peak=150.0, ramp=120.0,
                        outlet=W.TRANSMISSIVE)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_floodplain_fronts_bitwise(precision):
    """81,920 cells (320 tiles), inflow, a transmissive outlet, a front moving over dry
    land for 400 steps; the launches take a part of the tiles only."""
    a, b = pair(plain(nx=320, ny=128), precision=precision)
    seen = []
    for _ in range(8):
        a.step(50)
        b.step(50)
        same(a, b)
        seen.append(a.work())
        assert b.work()[0] == b.work()[1]  # skipping off: every tile
    # launches take a part of the tiles at first; as the flood spreads the lists hold
    # most tiles and the launches take them all again, in work-list order
    assert seen[0][0] < seen[0][1] and all(n > 0 for n, _ in seen), seen


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_tracking_and_chezy_bitwise(precision):
    """The optional-feature instantiations (tracking: level 1; Chezy: level 2) skip too;
    the tracking records match as well."""
    s = plain(seed=31)
    a, b = pair(s, precision=precision)
    for x in (a, b):
        x.set_friction(bm.FRICTION_CHEZY, 30.0)
        x.track(0.05)
    a.step(300)
    b.step(300)
    same(a, b)
    ta, tb = a.download_track(), b.download_track()
    for k in ta:
        assert np.array_equal(np.asarray(ta[k]), np.asarray(tb[k]), equal_nan=True), k


def test_rain_disk_bitwise():
    """Rain on a disk of dry cells (source tiles are fixed; the disk's neighbours get
    wet and are listed as the water spreads)."""
    s = plain(seed=37)
    reg = W.disk_region(s, 1100.0, 150.0, 60.0)
    a, b = pair(s)
    for x in (a, b):
        x.set_sources(reg, [bm.SOURCE_INTENSITY], [bm.SINK_EXACT], [(np.array([0.0, 1e6]), np.array([200.0, 200.0]))])
    a.step(300)
    b.step(300)
    same(a, b)


def test_run_until_and_resume_bitwise():
    """run_until stops on the end time; launches past it take the listed tiles without
    stepping them, and the next run continues with the same lists."""
    a, b = pair(plain(seed=41), precision="fp32")
    for t in (7.5, 20.0, 31.25):
        a.run_until(t)
        b.run_until(t)
        same(a, b)
    a.step(40)
    b.step(40)
    same(a, b)


def test_between_solo_and_batch_bitwise():
    """A state stepped alone, then in a batch (another work list), then alone again:
    each change of list starts with a launch of every tile."""
    scs = [plain(seed=43), W.floodplain(nx=90, ny=33, Lx=900.0, Ly=330.0, seed=51, q_peak=120.0, ramp=60.0)]
    on = [bm.State.from_scenario(s) for s in scs]
    off = [bm.State.from_scenario(s) for s in scs]
    for x in off:
        x.set_tile_skipping(False)
    for x, y in zip(on, off):
        x.step(30)
        y.step(30)
    bm.Batch(on).step(60)
    for y in off:
        y.step(60)
    for x, y in zip(on, off):
        x.step(30)
        y.step(30)
        same(x, y)


def test_upload_mid_run_bitwise():
    """An upload replaces the state: the next launch takes every tile."""
    s = plain(seed=47)
    a, b = pair(s)
    a.step(100)
    b.step(100)
    c = bm.State.from_scenario(s)  # another state of the same mesh, further on
    c.step(170)
    H, qx, qy, t = c.download()
    a.upload(H, qx, qy, t)
    b.upload(H, qx, qy, t)
    a.step(100)
    b.step(100)
    same(a, b)


def test_dry_closed_basin_takes_one_tile():
    """A dry closed basin (walls only, no water): only item 0 is taken, the time still
    advances by dt_max per step."""
    s = W.fractal_lake(nx=60, ny=30, Lx=600.0, Ly=300.0, seed=5, level=390.0)
    st = bm.State.from_scenario(s, dt_max=0.5)
    st.step(3)
    assert st.work()[0] == 1
    st.step(10)
    assert st.stats()["t"] == pytest.approx(6.5, abs=1e-12)
    H, qx, qy, _ = st.download()
    assert np.array_equal(H, np.maximum(s.H, s.z)) and not qx.any() and not qy.any()
