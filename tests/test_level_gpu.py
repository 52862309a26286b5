"""The water-level boundary on the GPU (the zhydrograph of Section "Boundary conditions",
standard inflows and outflows) against the FP64 oracle, through the C ABI.

Bars: FP64 relative L-inf 1e-11 on h, hu, hv (normwise), time 1e-12, boundary volume
1e-9 relative; FP32-bulk L1 of h <= 1e-4 m (that mode's bar); still water at the
imposed level bitwise at rest in both precisions.  Meshes span several 256-cell tiles
with a ragged last tile; the level rises and falls over a rolling bed with dry high
ground, floods dry cells as a dam break, rises past a dry boundary cell's bed between
two steps, and carries passive species out (none in).
"""
import numpy as np
import pytest

import oracle
from paper_2102_12862_b300 import bm
from paper_2102_12862_b300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-11
LEVEL_T = np.array([0.0, 40.0, 90.0, 150.0])
LEVEL_Z = np.array([1.3, 1.6, 1.6, 0.9])


def rel_linf(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def compare(s, st, o, tol=TOL):
    H, qx, qy, t = st.download()
    assert abs(t - o.time) <= 1e-12 * max(1.0, abs(o.time)), (t, o.time)
    errs = {"h": rel_linf(H - s.z, o.H - s.z), "hu": rel_linf(qx, o.qx), "hv": rel_linf(qy, o.qy)}
    for k, e in errs.items():
        assert e <= tol, f"{k}: rel Linf {e:.3e} > {tol:.0e} ({errs})"
    return errs


def basin(nx=60, ny=20, L=300.0, Wd=100.0, Q=15.0, seed=9, jitter=0.1, cfl_mode=1, H0=1.3):
    """A jittered basin (2 nx ny cells): inflow Q at x = 0, a water level at x = L, walls
    along y = 0 and y = Wd; a rolling bed 0.2-1.6 m, water at H0 (the high ground dry),
    Manning n = 0.03."""
    xy, tri, tag = W.rect_mesh(nx, ny, L, Wd, jitter=jitter, seed=seed,
                               side_tags=(W.INFLOW, W.WATER_LEVEL, W.WALL, W.WALL))
    c = xy[tri].mean(axis=1)
    N = len(tri)
    z = 0.9 + 0.7 * np.sin(2 * np.pi * c[:, 0] / 170.0) * np.cos(2 * np.pi * c[:, 1] / 90.0)
    H = np.maximum(z, H0)
    return W.Scenario("level_basin", xy, tri, z, np.full(N, 0.03), tag, H, np.zeros(N), np.zeros(N),
                      W.default_params(cfl_mode=cfl_mode, hydro_t=np.array([0.0, 60.0, 1e9]),
                                       hydro_q=np.array([0.0, Q, Q])))


def both(s, t=LEVEL_T, z=LEVEL_Z, precision="fp64", **kw):
    st = bm.State.from_scenario(s, precision=precision, **kw)
    o = oracle.Oracle(s, **kw)
    st.set_level(t, z)
    o.set_level(t, z)
    return st, o


@pytest.mark.parametrize("cfl_mode", [0, 1])
def test_level_rises_and_falls_fp64(cfl_mode):
    """Fed at x = 0, the level at x = L rising 1.3 -> 1.6 m (water enters over the
    rolling bed), holding, then falling to 0.9 m (the basin drains through it): 400
    steps, then to t = 200 s, against the oracle.  With Eq. 21's per-edge time step
    (cfl_mode 0) the basin's inflow corner runs through negative depths after about
    390 steps (the oracle's too, and the same basin with walls sooner): that mode
    takes 300 steps."""
    s = basin(cfl_mode=cfl_mode)
    assert s.n_cells % 256 != 0 and s.n_cells > 4 * 256
    st, o = both(s)
    assert abs(st.stats()["dt_next"] - o.next_dt()) <= 1e-12 * o.next_dt()
    n = 400 if cfl_mode == 1 else 300
    st.step(n)
    o.step(n)
    compare(s, st, o)
    assert o.boundary_volume != 0.0
    assert abs(st.stats()["boundary_volume"] - o.boundary_volume) <= 1e-9 * abs(o.boundary_volume)
    if cfl_mode == 0:
        return
    bv = []
    for T in (120.0, 200.0):
        st.run_until(T)
        o.run_until(T)
        compare(s, st, o)
        assert abs(st.stats()["boundary_volume"] - o.boundary_volume) <= 1e-9 * abs(o.boundary_volume)
        bv.append(o.boundary_volume)
    # the falling level drains more than the inflow brings
    assert bv[1] < bv[0]


def test_level_rises_and_falls_fp32():
    s = basin()
    st, o = both(s, precision="fp32")
    st.run_until(200.0)
    o.run_until(200.0)
    H, qx, qy, t = st.download()
    area = o.area()
    l1 = float(np.sum(area * np.abs((H - s.z) - (o.H - s.z))) / area.sum())
    assert t == 200.0
    assert l1 <= 1e-4, l1
    assert abs(st.stats()["boundary_volume"] - o.boundary_volume) <= 1e-4 * max(abs(o.boundary_volume), 1.0)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("cfl_mode", [0, 1])
def test_rest_at_the_imposed_level_is_bitwise(precision, cfl_mode):
    """The fractal lake (rough bed, dry islands above the level) with one side at the
    lake's own level: 500 steps leave every value unchanged, nothing crosses."""
    s = W.fractal_lake(nx=48, ny=24, Lx=480.0, Ly=240.0, seed=11)
    xy, tri, tag = W.rect_mesh(48, 24, 480.0, 240.0, jitter=0.1, seed=11,
                               side_tags=(W.WALL, W.WATER_LEVEL, W.WALL, W.WALL))
    s.edge_tag = tag
    st = bm.State.from_scenario(s, precision=precision, cfl_mode=cfl_mode)
    st.set_level([0.0], [403.0])
    H0, _, _, _ = st.download()
    st.step(500)
    H, qx, qy, _ = st.download()
    assert np.array_equal(H, H0)
    assert not np.any(qx) and not np.any(qy)
    assert st.stats()["boundary_volume"] == 0.0


@pytest.mark.parametrize("cfl_mode", [0, 1])
def test_dry_channel_flooded_from_a_level(cfl_mode):
    """A dry flat channel with a 0.5 m level at x = 0: the level floods the dry cell as a
    dam break and the front runs in; the first dt comes from the boundary state over
    the dry cells alone. 300 steps against the oracle."""
    xy, tri, tag = W.rect_mesh(200, 3, 400.0, 6.0, jitter=0.05, seed=3,
                               side_tags=(W.WATER_LEVEL, W.WALL, W.WALL, W.WALL))
    N = len(tri)
    s = W.Scenario("dry_channel", xy, tri, np.zeros(N), np.full(N, 0.02), tag, np.zeros(N), np.zeros(N),
                   np.zeros(N), W.default_params(cfl_mode=cfl_mode))
    st, o = both(s, t=[0.0], z=[0.5])
    assert abs(st.stats()["dt_next"] - o.next_dt()) <= 1e-12 * o.next_dt()
    st.step(300)
    o.step(300)
    compare(s, st, o)
    assert abs(st.stats()["boundary_volume"] - o.boundary_volume) <= 1e-9 * abs(o.boundary_volume)


def test_level_rising_past_a_dry_bed():
    """The level starts below the bed of every boundary cell (a wall in effect: nothing
    moves, the cells are dry and at rest) and rises above it at t = 3 s: the step whose
    new time first puts the level over the bed takes its rate into Eq. 21 while the
    cells are still copied through. Against the oracle, 200 steps."""
    xy, tri, tag = W.rect_mesh(120, 4, 240.0, 8.0, jitter=0.05, seed=5,
                               side_tags=(W.WATER_LEVEL, W.WALL, W.WALL, W.WALL))
    N = len(tri)
    x = xy[tri].mean(axis=1)[:, 0]
    z = 0.2 + 0.001 * x
    s = W.Scenario("dry_ramp", xy, tri, z, np.full(N, 0.02), tag, z.copy(), np.zeros(N), np.zeros(N),
                   W.default_params(cfl_mode=1, dt_max=0.5))
    st, o = both(s, t=[0.0, 2.0, 3.0, 30.0], z=[0.0, 0.1, 0.2, 1.0])
    for n in (4, 3, 200):
        st.step(n)
        o.step(n)
        compare(s, st, o)
        assert abs(st.stats()["dt_next"] - o.next_dt()) <= 1e-12 * o.next_dt()
    assert o.boundary_volume > 0.0


def test_species_leave_and_none_enter():
    """One passive species in the basin: it leaves through the falling level with the
    inside concentration, and the water the rising level brings in carries none;
    against the oracle's species run, 300 steps, then to t = 160 s."""
    s = basin()
    x = s.centroids()[:, 0]
    hc = np.where(x > 150.0, 1.0, 0.25) * np.maximum(s.H - s.z, 0.0)
    st, o = both(s)
    st.set_scalars(hc[None, :], [0.0])
    o.set_scalars(hc[None, :], [0.0])
    st.step(300)
    o.step(300)
    compare(s, st, o)
    assert rel_linf(st.download_scalars()[0], o.hc[0]) <= 1e-11
    st.run_until(160.0)
    o.run_until(160.0)
    compare(s, st, o)
    assert rel_linf(st.download_scalars()[0], o.hc[0]) <= 1e-11


def test_batch_member_with_a_level_equals_solo():
    """A batch of the level basin and a plain floodplain member: the level member is
    bitwise the solo run."""
    s = basin()
    f = W.floodplain(nx=120, ny=48, Lx=1200.0, Ly=480.0, seed=5, q_peak=80.0, ramp=60.0)
    solo = bm.State.from_scenario(s)
    solo.set_level(LEVEL_T, LEVEL_Z)
    a = bm.State.from_scenario(s)
    a.set_level(LEVEL_T, LEVEL_Z)
    b = bm.Batch([a, bm.State.from_scenario(f)])
    solo.step(200)
    b.step(200)
    A = a.download()
    B = solo.download()
    for x, y in zip(A[:3], B[:3]):
        assert np.array_equal(x, y)
    assert A[3] == B[3]


def test_tile_skipping_with_a_level_bitwise():
    """A dry floodplain flooded from a rising level: the launches take the level tiles
    every time (fixed) and the flood's tiles as it spreads, bitwise the run that steps
    every tile."""
    s = basin(nx=160, ny=40, L=800.0, Wd=200.0, Q=0.0, H0=0.0)
    s.params["hydro_q"] = np.zeros(3)
    a = bm.State.from_scenario(s)
    b = bm.State.from_scenario(s)
    b.set_tile_skipping(False)
    for x in (a, b):
        x.set_level([0.0, 60.0], [0.5, 1.4])
    seen = []
    for _ in range(6):
        a.step(60)
        b.step(60)
        A, B = a.download(), b.download()
        for x, y in zip(A[:3], B[:3]):
            assert np.array_equal(x, y)
        seen.append(a.work())
    assert seen[0][0] < seen[0][1], seen


def test_set_level_validates_reprimes_and_unsets():
    s = basin()
    st = bm.State.from_scenario(s)
    with pytest.raises(bm.BMError):
        st.set_level([1.0, 1.0], [0.0, 1.0])
    with pytest.raises(bm.BMError):
        st.set_level([0.0, float("nan")], [0.0, 1.0])
    with pytest.raises(bm.BMError):
        st.set_level([0.0], [float("inf")])
    with pytest.raises(ValueError):
        st.set_level([0.0, 1.0], [0.0])
    # a level far above the basin changes the first dt at once (re-primed, as the oracle)
    o = oracle.Oracle(s)
    dt_walls = st.stats()["dt_next"]
    assert abs(dt_walls - o.next_dt()) <= 1e-12 * dt_walls
    for x in (st, o):
        x.set_level([0.0], [6.0])
    assert abs(st.stats()["dt_next"] - o.next_dt()) <= 1e-12 * o.next_dt()
    assert st.stats()["dt_next"] < dt_walls
    assert st.stats()["t"] == 0.0 and st.stats()["steps"] == 0
    # unset: walls again; the still basin (no inflow yet) stays at rest
    s2 = basin(Q=0.0)
    s2.params["hydro_q"] = np.zeros(3)
    st2 = bm.State.from_scenario(s2)
    st2.set_level([0.0], [6.0])
    st2.set_level([], [])
    H0, _, _, _ = st2.download()
    st2.step(100)
    H, qx, qy, _ = st2.download()
    assert np.array_equal(H, H0) and not np.any(qx) and not np.any(qy)
