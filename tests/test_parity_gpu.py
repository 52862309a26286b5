"""Parity of the CUDA FP64 step (through the C ABI) with the FP64 CPU oracle.

Bar: relative L-infinity <= 1e-11 on h = H - z, hu = q_x and hv = q_y (normwise:
||a - b||_inf / max(||b||_inf, 1e-300)), time and dt equal to 1e-12 relative.
Inputs are seeded synthetic meshes; sizes span many 256-cell tiles with a ragged
last tile, plus the degenerate cases (one and two triangles, all dry).
"""
import numpy as np
import pytest

import oracle
from paper_2102_12862_b300 import bm
from paper_2102_12862_b300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-11


def rel_linf(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def compare(s, st, o, tol=TOL):
    H, qx, qy, t = st.download()
    assert abs(t - o.time) <= 1e-12 * max(1.0, abs(o.time)), (t, o.time)
    errs = {"h": rel_linf(H - s.z, o.H - s.z), "hu": rel_linf(qx, o.qx), "hv": rel_linf(qy, o.qy)}
    for k, e in errs.items():
        assert e <= tol, f"{k}: rel Linf {e:.3e} > {tol:.0e} ({errs})"
    return errs


def both(s, **ov):
    st = bm.State.from_scenario(s, **ov)
    o = oracle.Oracle(s, **ov)
    return st, o


def test_dam_break_500_steps():
    """Dam break on the 200 x 10 jittered channel (4,000 cells): 500 steps."""
    s = W.dam_break()
    st, o = both(s)
    st.step(500)
    o.step(500)
    compare(s, st, o)
    stt = st.stats()
    assert stt["steps"] == 500
    assert abs(stt["volume"] - o.volume()) <= 1e-12 * o.volume()
    assert abs(stt["boundary_volume"] - o.boundary_volume) <= 1e-9 * abs(o.boundary_volume)


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("nx,ny", [(40, 13), (101, 7)])
def test_random_states_wet_dry_friction(seed, nx, ny):
    """Random beds, depths (20 % dry, some below h_min), velocities and Manning n on
    jittered meshes with walls and transmissive ends: 1 step, then 30 more.  These
    rough states need the positivity time step (cfl_mode 1): Eq. 21 as printed lets
    the depth go negative on them (see test_negative_depth_flagged)."""
    s = W.random_state(W.dam_break(nx=nx, ny=ny, seed=seed), seed=seed)
    st, o = both(s, cfl_mode=1)
    st.step(1)
    o.step(1)
    compare(s, st, o)
    st.step(30)
    o.step(30)
    compare(s, st, o)


def test_floodplain_inflow_transmissive_small():
    """Small floodplain: inflow hydrograph, transmissive outlet, walls, wet/dry fronts."""
    s = W.floodplain(nx=120, ny=50, Lx=1200.0, Ly=500.0, seed=22, q_peak=200.0, ramp=100.0,
                     outlet=W.TRANSMISSIVE)
    st, o = both(s)
    st.run_until(150.0)
    o.run_until(150.0)
    compare(s, st, o, tol=1e-10 if o.steps > 400 else TOL)
    stt = st.stats()
    assert stt["steps"] == o.steps
    assert abs(stt["boundary_volume"] - o.boundary_volume) <= 1e-10 * abs(o.boundary_volume)


def test_negative_depth_flagged():
    """Eq. 21 as printed (cfl_mode 0) on a rough random state drives some depths below
    -h_min in the first step; the kernel flags it (BM_ENEGDEPTH, no fault) and the state
    still matches the oracle, which computes the same negative depths."""
    s = W.random_state(W.dam_break(nx=40, ny=13, seed=0), seed=0)
    st, o = both(s)
    with pytest.raises(bm.BMError) as ei:
        st.step(1)
    assert ei.value.status == bm.BM_ENEGDEPTH
    o.step(1)
    assert o.depth().min() < -s.params["h_min"]
    compare(s, st, o)


def test_cfl_mode_positivity():
    s = W.random_state(W.dam_break(nx=30, ny=9, seed=4), seed=4)
    st, o = both(s, cfl_mode=1)
    st.step(40)
    o.step(40)
    compare(s, st, o)


def test_lake_at_rest_bitwise():
    """C-property on the GPU: still water over rough terrain with dry islands stays
    bitwise still over 2,000 steps."""
    s = W.fractal_lake(nx=80, ny=40, Lx=800.0, Ly=400.0, seed=31)
    st = bm.State.from_scenario(s)
    st.step(2000)
    H, qx, qy, t = st.download()
    assert np.array_equal(H, s.H)
    assert not qx.any() and not qy.any()


def test_mass_closed_domain():
    s = W.dam_break(nx=100, ny=10, closed=True, h_right=0.0, manning=0.02)
    st = bm.State.from_scenario(s)
    v0 = st.stats()["volume"]
    st.step(1000)
    assert abs(st.stats()["volume"] - v0) / v0 < 1e-13


def test_run_until_exact_time_and_resume():
    s = W.dam_break()
    st, o = both(s)
    st.run_until(10.0)
    o.run_until(10.0)
    compare(s, st, o)
    assert st.stats()["t"] == 10.0
    # checkpoint: download, continue; a second state resumed from the checkpoint agrees bitwise
    H, qx, qy, t = st.download()
    st.step(37)
    r = bm.State(st.mesh, H, qx, qy, **s.params)
    r.upload(H, qx, qy, t)
    r.step(37)
    a, b = st.download(), r.download()
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_tiny_meshes_and_all_dry():
    # one triangle with a wall on every edge
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    tri = np.array([[0, 1, 2]], np.int32)
    s = W.Scenario("one", xy, tri, np.zeros(1), np.zeros(1), np.zeros((1, 3), np.uint8), np.ones(1),
                   np.array([0.3]), np.array([-0.2]), W.default_params())
    st, o = both(s)
    st.step(5)
    o.step(5)
    compare(s, st, o)
    # two triangles, one dry, transmissive boundary
    s = W.dam_break(nx=1, ny=1, jitter=0.0, h_right=0.0, x_dam=50.0, Lx=100.0, Ly=10.0)
    s.H = np.array([1.0, 0.0])
    st, o = both(s)
    st.step(7)
    o.step(7)
    compare(s, st, o)
    # all dry without inflow: dt = dt_max, nothing moves
    s = W.dam_break(nx=20, ny=3)
    s.H = s.z.copy()
    st = bm.State.from_scenario(s)
    st.step(3)
    stt = st.stats()
    assert stt["t"] == 3.0 and stt["volume"] == 0.0


def test_ragged_tail_sizes():
    for nx in (1, 64, 129):  # 2*nx*ny cells around multiples of the 256-cell tile
        s = W.random_state(W.dam_break(nx=nx, ny=2, seed=nx), seed=nx)
        st, o = both(s, cfl_mode=1)
        st.step(3)
        o.step(3)
        compare(s, st, o)


def test_invalid_state_rejected():
    s = W.dam_break(nx=10, ny=2)
    mesh = bm.Mesh.from_scenario(s)
    H = s.H.copy()
    H[3] = s.z[3] - 0.1
    with pytest.raises(bm.BMError, match="H < z_bed"):
        bm.State(mesh, H, s.qx, s.qy)
    H = s.H.copy()
    H[0] = np.nan
    with pytest.raises(bm.BMError, match="non-finite"):
        bm.State(mesh, H, s.qx, s.qy)


def test_floodplain_full_size():
    """The 2,000,000-cell floodplain (the benchmark workload, same kernels and launch
    configuration): 5 steps from its initial state, then 3 steps from a seeded random
    wet/dry state on the same mesh; every cell compared with the oracle."""
    s = W.floodplain()
    st, o = both(s)
    st.step(5)
    o.step(5)
    compare(s, st, o)
    r = W.random_state(s, seed=77, depth=(0.01, 3.0), keep_bed=True)
    st2, o2 = both(r, cfl_mode=1)
    st2.step(3)
    o2.step(3)
    compare(r, st2, o2)


def test_floodplain_full_size_mid_run_window():
    """The 2,000,000-cell floodplain mid-run (moving wet/dry fronts, the inflow at its
    500 m^3/s plateau): the FP64 GPU run to t = 1,800 s is downloaded, the oracle
    starts from that snapshot (same time, so the same Q(t)), and both take 20 steps;
    every cell compared (h, hu, hv) at the 1e-11 bar."""
    s = W.floodplain()
    st = bm.State.from_scenario(s)
    st.run_until(1800.0)
    H, qx, qy, t = st.download()
    assert t == 1800.0
    wet = float(np.mean(H - s.z > 1e-6))
    assert wet > 0.08, wet  # well past the initial 4 % wet channel
    snap = s.copy()
    snap.H, snap.qx, snap.qy = H, qx, qy
    o = oracle.Oracle(snap)
    o.t.value = t
    st.step(20)
    o.step(20)
    compare(s, st, o)


def test_non_finite_state_is_flagged_and_the_mesh_stays_usable():
    """A total-discharge source of 1e308 m^3/s on one cell of 0.25 m^2 makes S_h overflow
    to infinity: the step returns BM_ENONFINITE (the device's status word, no fault),
    the state still downloads, and a fresh state on the same mesh steps and matches the
    oracle."""
    s = W.dam_break(manning=0.02)
    mesh = bm.Mesh.from_scenario(s)
    for prec in ("fp64", "fp32"):
        st = bm.State.from_scenario(s, mesh=mesh, precision=prec)
        region = np.full(s.n_cells, -1, np.int32)
        region[1234] = 0
        st.set_sources(region, [bm.SOURCE_TOTAL], [bm.SINK_EXACT], [(np.array([0.0]), np.array([1e308]))])
        with pytest.raises(bm.BMError) as ei:
            st.step(3)
        assert ei.value.status == bm.BM_ENONFINITE, ei.value
        H, qx, qy, t = st.download()
        assert not np.isfinite(H[1234])
        st.close()
    st, o = bm.State.from_scenario(s, mesh=mesh), oracle.Oracle(s)
    st.step(20)
    o.step(20)
    compare(s, st, o)
