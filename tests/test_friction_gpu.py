"""Table 1's logarithmic friction closures (Chezy, Bezzola) in the step kernel against
the oracle: one step of uniform flow in a box in every branch of each law, and uniform
flow on a slope run to its normal depth.  FP64: relative L-inf 1e-11 (1e-10 past 400
steps) on h, q_x, q_y; FP32-bulk: 1e-5 on the one-step discharge (single-precision
closure), the normal depth within 1e-4 m.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2102_12862_b300 import bm
from paper_2102_12862_b300 import workloads as W

pytestmark = pytest.mark.gpu


def rel_linf(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def box(h):
    Lx, Ly, nx, ny = 20.0, 10.0, 20, 10
    xy, tri, tag = W.rect_mesh(nx, ny, Lx, Ly, jitter=0.0, side_tags=(W.WALL, W.WALL, W.WALL, W.WALL))
    N = len(tri)
    return W.Scenario("box", xy, tri, np.zeros(N), np.full(N, 0.03), tag, np.full(N, h), np.full(N, 0.6 * h),
                      np.full(N, 0.2 * h), W.default_params())


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("law,h,r", [(1, 0.8, 0.05), (1, 0.04, 0.05), (2, 0.9, 0.1), (2, 0.15, 0.1),
                                     (2, 0.04, 0.1)])
def test_one_step_box(precision, law, h, r):
    s = box(h)
    st = bm.State.from_scenario(s, precision=precision)
    o = oracle.Oracle(s)
    st.set_friction(law, r)
    o.set_friction(law, r)
    st.step(1)
    o.step(1)
    H, qx, qy, _ = st.download()
    tol = 1e-11 if precision == "fp64" else 1e-5
    assert rel_linf(qx, o.qx) <= tol and rel_linf(qy, o.qy) <= tol
    assert np.median(qx) < 0.6 * h  # friction acted (wall cells also see fluxes)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("law,r", [(1, 0.02), (2, 0.05)])
def test_uniform_flow_channel(precision, law, r):
    L, Wd, S, q = 1000.0, 20.0, 0.002, 2.0
    xy, tri, tag = W.rect_mesh(100, 4, L, Wd, jitter=0.1, seed=3,
                               side_tags=(W.INFLOW, W.TRANSMISSIVE, W.WALL, W.WALL))
    c = xy[tri].mean(axis=1)
    N = len(tri)
    z = S * (L - c[:, 0])
    s = W.Scenario("uniform_flow", xy, tri, z, np.full(N, 0.03), tag, z + 0.5, np.full(N, q), np.zeros(N),
                   W.default_params(hydro_t=np.array([0.0, 1e9]), hydro_q=np.array([q * Wd, q * Wd])))
    st = bm.State.from_scenario(s, precision=precision)
    o = oracle.Oracle(s)
    st.set_friction(law, r)
    o.set_friction(law, r)
    st.run_until(600.0)
    o.run_until(600.0)
    H, qx, qy, _ = st.download()
    if precision == "fp64":
        tol = 1e-10 if o.steps > 400 else 1e-11
        for a, b in ((H - s.z, o.H - s.z), (qx, o.qx), (qy, o.qy)):
            assert rel_linf(a, b) <= tol
    else:
        assert np.max(np.abs((H - s.z) - (o.H - s.z))) <= 1e-4


def test_friction_api_rules():
    s = W.dam_break(nx=40, ny=4, manning=0.02)
    st = bm.State.from_scenario(s)
    with pytest.raises(bm.BMError, match="law"):
        st.set_friction(3, 0.05)
    with pytest.raises(bm.BMError, match=">= 0"):
        st.set_friction(1, -1.0)
    st.set_friction(bm.FRICTION_CHEZY, 0.05)
    with pytest.raises(bm.BMError, match="Manning"):
        st.set_morpho()
    st.step(5)
    st.set_friction(bm.FRICTION_MANNING, 0.02)  # back to the default law
    st.track(0.1)
    st.step(5)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_with_a_log_law_member_equals_solo(precision):
    """A batch of a Chezy member, a Bezzola member and a Manning member steps each
    bitwise as it steps alone (the descriptor carries the law)."""
    scs = [W.dam_break(manning=0.02, seed=s) for s in (1, 2, 3)]
    laws = [(bm.FRICTION_CHEZY, 0.05), (bm.FRICTION_BEZZOLA, 0.1), (bm.FRICTION_MANNING, 0.03)]
    solo = [bm.State.from_scenario(s, precision=precision) for s in scs]
    members = [bm.State.from_scenario(s, precision=precision) for s in scs]
    for st_list in (solo, members):
        for st, (law, r) in zip(st_list, laws):
            st.set_friction(law, r)
    # flood tracking on every member: a mixed-law batch runs the optional-feature
    # instantiation for all, so the Manning member's record comes from the law-0 branch
    # of the shared code; each record must equal the member's solo record bit for bit
    for st in solo + members:
        st.track(0.05)
    for st in solo:
        st.step(60)
    bm.Batch(members).step(60)
    for a, b in zip(solo, members):
        for x, y in zip(a.download(), b.download()):
            assert np.array_equal(np.asarray(x), np.asarray(y))
        ra, rb = a.download_track(), b.download_track()
        for f in ra:
            assert np.array_equal(ra[f], rb[f], equal_nan=True), f


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("law,r", [(bm.FRICTION_CHEZY, 0.01), (bm.FRICTION_BEZZOLA, 0.25)])
def test_tracking_under_a_log_law(precision, law, r):
    """Flood tracking on a wet dam break (h 1.0 | 0.1 m) under Chezy's and Bezzola's laws:
    the record (shear stress rho u^2 / c_f^2 of the law in force) matches the oracle's.
    With y_R = 0.25 m, h / y_R runs from 0.4 (the right state) past 2 (the middle
    state is 0.4 m) to 4 (the left state), so all three Bezzola branches are visited.
    FP64: 200 steps, relative L-inf 1e-11 on the maxima of h and |q|, 1e-9 on |u| and
    the stress (they divide by the depth); FP32-bulk (its closure in single precision):
    20 steps, 1e-4 on every maximum."""
    s = W.dam_break(manning=0.02, seed=4)
    st = bm.State.from_scenario(s, precision=precision)
    o = oracle.Oracle(s)
    for x in (st, o):
        x.set_friction(law, r)
        x.track(0.2)
    n = 200 if precision == "fp64" else 20
    st.step(n)
    o.step(n)
    g, ref = st.download_track(), o.tracking
    tight, loose = (1e-11, 1e-9) if precision == "fp64" else (1e-4, 1e-4)
    for k in ("h_max", "q_max"):
        assert rel_linf(g[k], ref[k]) <= tight, k
    for k in ("u_max", "tau_max"):
        assert rel_linf(g[k], ref[k]) <= loose, k
    assert g["tau_max"].max() > 0
    if law == bm.FRICTION_BEZZOLA:
        ratio = o.depth() / r  # the branches the run visited
        assert ratio.min() < 0.5 and ratio.max() > 2.0
