"""The outflow boundaries on the GPU (h-Q relation and weir; Section "Boundary
conditions", standard outflows) against the FP64 oracle, through the C ABI.

Bars: FP64 relative L-inf 1e-11 on h, hu, hv (normwise), time 1e-12, boundary volume
1e-9 relative; FP32-bulk L1 of h <= 1e-4 m (that mode's bar).  Meshes span several
256-cell tiles with a ragged last tile; the outlets are fed, drained, capped at the
critical discharge (Ritter) and below the crest (a wall, bitwise at rest).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2102_12862_b300 import bm
from paper_2102_12862_b300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-11
RATING_S = np.array([0.8, 1.2, 1.6, 2.2])
RATING_Q = np.array([0.0, 5.0, 15.0, 40.0])


def rel_linf(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def compare(s, st, o, tol=TOL):
    H, qx, qy, t = st.download()
    assert abs(t - o.time) <= 1e-12 * max(1.0, abs(o.time)), (t, o.time)
    errs = {"h": rel_linf(H - s.z, o.H - s.z), "hu": rel_linf(qx, o.qx), "hv": rel_linf(qy, o.qy)}
    for k, e in errs.items():
        assert e <= tol, f"{k}: rel Linf {e:.3e} > {tol:.0e} ({errs})"
    return errs


def outlets(nx=60, ny=20, L=300.0, Wd=100.0, Q=20.0, seed=7, jitter=0.1):
    """A jittered basin (2 nx ny cells): inflow Q at x = 0, a weir at x = L, an h-Q
    outlet along y = 0, a wall along y = Wd; a rolling bed 0.2-1.6 m, water at 1.3 m
    (the high ground dry), Manning n = 0.03."""
    xy, tri, tag = W.rect_mesh(nx, ny, L, Wd, jitter=jitter, seed=seed,
                               side_tags=(W.INFLOW, W.WEIR, W.HQ_OUTFLOW, W.WALL))
    c = xy[tri].mean(axis=1)
    N = len(tri)
    z = 0.9 + 0.7 * np.sin(2 * np.pi * c[:, 0] / 170.0) * np.cos(2 * np.pi * c[:, 1] / 90.0)
    H = np.maximum(z, 1.3)
    return W.Scenario("outlets", xy, tri, z, np.full(N, 0.03), tag, H, np.zeros(N), np.zeros(N),
                      W.default_params(cfl_mode=1, hydro_t=np.array([0.0, 60.0, 1e9]),
                                       hydro_q=np.array([0.0, Q, Q])))


def laws(x):
    x.set_outflow(hq_stage=RATING_S, hq_discharge=RATING_Q, weir_crest=1.1, weir_poleni=0.6)


def both(s, precision="fp64", **kw):
    st = bm.State.from_scenario(s, precision=precision, **kw)
    o = oracle.Oracle(s, **kw)
    laws(st)
    laws(o)
    return st, o


def test_weir_and_hq_outlets_fp64():
    """Fed, filling over the rolling bed and draining over the weir and through the h-Q
    outlet: 400 steps, then to t = 120 s, against the oracle."""
    s = outlets()
    assert s.n_cells % 256 != 0 and s.n_cells > 4 * 256
    st, o = both(s)
    assert abs(st.stats()["dt_next"] - o.next_dt()) <= 1e-12 * o.next_dt()
    st.step(400)
    o.step(400)
    compare(s, st, o)
    stt = st.stats()
    assert stt["boundary_volume"] != 0.0
    assert abs(stt["boundary_volume"] - o.boundary_volume) <= 1e-9 * abs(o.boundary_volume)
    st.run_until(120.0)
    o.run_until(120.0)
    compare(s, st, o)
    # both outlets let water out by then
    _, qo = o.boundary_discharge()
    L, R, nx, ny, ln = o.edges()
    assert np.sum((qo * ln)[R == -4]) > 0 and np.sum((qo * ln)[R == -5]) > 0


def test_weir_and_hq_outlets_fp32():
    s = outlets()
    st, o = both(s, precision="fp32")
    st.run_until(120.0)
    o.run_until(120.0)
    H, qx, qy, t = st.download()
    area = o.area()
    l1 = float(np.sum(area * np.abs((H - s.z) - (o.H - s.z))) / area.sum())
    assert t == 120.0
    assert l1 <= 1e-4, l1
    assert abs(st.stats()["boundary_volume"] - o.boundary_volume) <= 1e-4 * abs(o.boundary_volume)


@pytest.mark.parametrize("cfl_mode", [0, 1])
def test_outlet_capped_at_ritter_discharge(cfl_mode):
    """Poleni with mu = 50 on a crest far below the bed: the outlet passes the critical
    discharge of the characteristic (Ritter's dam-site flow) and its wave speed decides
    Eq. 21; 60 steps of the draining strip against the oracle."""
    xy, tri, tag = W.rect_mesh(30, 3, 60.0, 30.0, jitter=0.1, seed=4,
                               side_tags=(W.WALL, W.WEIR, W.WALL, W.WALL))
    N = len(tri)
    s = W.Scenario("strip", xy, tri, np.zeros(N), np.zeros(N), tag, np.full(N, 2.0), np.zeros(N), np.zeros(N),
                   W.default_params(cfl_mode=cfl_mode))
    st = bm.State.from_scenario(s)
    o = oracle.Oracle(s)
    for x in (st, o):
        x.set_outflow(weir_crest=-10.0, weir_poleni=50.0)
    assert abs(st.stats()["dt_next"] - o.next_dt()) <= 1e-12 * o.next_dt()
    st.step(60)
    o.step(60)
    compare(s, st, o)
    assert abs(st.stats()["boundary_volume"] - o.boundary_volume) <= 1e-9 * abs(o.boundary_volume)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_water_below_the_crest_stays_at_rest_bitwise(precision):
    """Still water below the weir crest and an h-Q outlet whose rating gives 0 at that
    stage: both are walls, and the lake stays bitwise at rest for 500 steps."""
    s = outlets(Q=0.0)
    s.params["hydro_q"] = np.zeros(3)
    s.H = np.maximum(s.z, 1.0)
    st = bm.State.from_scenario(s, precision=precision, cfl_mode=0)
    st.set_outflow(hq_stage=[1.0, 2.0], hq_discharge=[0.0, 10.0], weir_crest=1.1, weir_poleni=0.6)
    H0, _, _, _ = st.download()
    st.step(500)
    H, qx, qy, _ = st.download()
    assert np.array_equal(H, H0)
    assert not np.any(qx) and not np.any(qy)
    assert st.stats()["boundary_volume"] == 0.0


def test_species_leave_with_the_inside_concentration():
    """One passive species in the filling basin: it leaves through the weir and the h-Q
    outlet with the inside cell's concentration (the inflow brings c = 0), against the
    oracle's species run, 300 steps."""
    s = outlets()
    x = s.centroids()[:, 0]
    hc = np.where(x > 150.0, 1.0, 0.25) * np.maximum(s.H - s.z, 0.0)
    st, o = both(s)
    st.set_scalars(hc[None, :], [0.0])
    o.set_scalars(hc[None, :], [0.0])
    st.step(300)
    o.step(300)
    compare(s, st, o)
    g, r = st.download_scalars(), o.hc
    assert rel_linf(g[0], r[0]) <= 1e-11
    # species mass left through the outlets
    assert np.sum(o.area() * r[0]) < np.sum(o.area() * hc)


def test_batch_member_with_outflow_laws_equals_solo():
    """A batch of the outlet basin (with its laws) and a plain floodplain member: the
    outlet member is bitwise the solo run."""
    s = outlets()
    f = W.floodplain(nx=120, ny=48, Lx=1200.0, Ly=480.0, seed=5, q_peak=80.0, ramp=60.0)
    solo = bm.State.from_scenario(s)
    laws(solo)
    a = bm.State.from_scenario(s)
    laws(a)
    b = bm.Batch([a, bm.State.from_scenario(f)])
    solo.step(200)
    b.step(200)
    A = a.download()
    B = solo.download()
    for x, y in zip(A[:3], B[:3]):
        assert np.array_equal(x, y)
    assert A[3] == B[3]


def test_set_outflow_validates_and_reprimes():
    s = outlets()
    st = bm.State.from_scenario(s)
    with pytest.raises(bm.BMError):
        st.set_outflow(hq_stage=[1.0, 1.0], hq_discharge=[0.0, 1.0])
    with pytest.raises(bm.BMError):
        st.set_outflow(hq_stage=[1.0, 2.0], hq_discharge=[0.0, -1.0])
    with pytest.raises(bm.BMError):
        st.set_outflow(hq_stage=[1.0], hq_discharge=[1.0])
    with pytest.raises(bm.BMError):
        st.set_outflow(weir_crest=float("nan"))
    with pytest.raises(bm.BMError):
        st.set_outflow(weir_poleni=-1.0)
    # laws that let water out at t = 0 change the first dt: re-primed, as the oracle.
    # The strip of long legs (dy >> dx) whose weir edge decides Eq. 21 once water leaves
    xy, tri, tag = W.rect_mesh(6, 1, 12.0, 10.0, jitter=0.0, side_tags=(W.WALL, W.WEIR, W.WALL, W.WALL))
    N = len(tri)
    s2 = W.Scenario("strip", xy, tri, np.zeros(N), np.zeros(N), tag, np.full(N, 2.0), np.zeros(N), np.zeros(N),
                    W.default_params(cfl_mode=0))
    st2 = bm.State.from_scenario(s2)
    o2 = oracle.Oracle(s2)
    dt_walls = st2.stats()["dt_next"]
    assert abs(dt_walls - o2.next_dt()) <= 1e-12 * dt_walls
    for x in (st2, o2):
        x.set_outflow(weir_crest=-10.0, weir_poleni=50.0)
    assert abs(st2.stats()["dt_next"] - o2.next_dt()) <= 1e-12 * o2.next_dt()
    assert st2.stats()["dt_next"] < dt_walls
    assert st2.stats()["t"] == 0.0 and st2.stats()["steps"] == 0
