"""Bed evolution on the GPU (the bed-flux kernel and the update after each step)
against the oracle (Section "Morphodynamics": Eq. 13 with the HLL sediment flux of
Eq. 14-16 and Table 2's MPM-like closure).

FP64: the bed change z - z0 within relative L-inf 1e-11 of the oracle's (normwise, as
the state parity; 1e-10 past 400 steps), the water state within the state parity bar,
sediment and water volumes conserved in a closed basin to 1e-12.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2102_12862_b300 import bm
from paper_2102_12862_b300 import workloads as W

pytestmark = pytest.mark.gpu
SAND = dict(porosity=0.4, s=2.65, d=0.001, alpha=8.0, m=1.5, theta_cr=0.047)


def rel_linf(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def both(s, **kw):
    st = bm.State.from_scenario(s, **kw)
    o = oracle.Oracle(s, **kw)
    st.set_morpho(**SAND)
    o.set_morpho(**SAND)
    return st, o


def compare(s, st, o):
    tol = 1e-10 if o.steps > 400 else 1e-11
    z = st.download_bed()
    H, qx, qy, t = st.download()
    assert abs(t - o.time) <= 1e-12 * max(1.0, o.time)
    e = rel_linf(z - s.z, o.z - s.z)
    assert e <= tol, f"bed change: rel Linf {e:.3e} ({o.steps} steps)"
    for name, a, b in (("h", H - z, o.H - o.z), ("hu", qx, o.qx), ("hv", qy, o.qy)):
        e = rel_linf(a, b)
        assert e <= tol, f"{name}: rel Linf {e:.3e} ({o.steps} steps)"
    return z, H


def test_closed_basin_fp64():
    """Random wet/dry state with friction in a closed basin (several tiles, a ragged
    last tile): parity after 300 steps; sediment and water volumes conserved."""
    s = W.random_state(W.dam_break(nx=150, ny=20, seed=4, closed=True, manning=0.03), seed=4, dry_frac=0.1)
    st, o = both(s, cfl_mode=1)
    area = o.area()
    v0 = o.volume()
    st.step(300)
    o.step(300)
    z, H = compare(s, st, o)
    dz = z - s.z
    assert np.max(np.abs(dz)) > 1e-4
    assert abs(area @ dz) <= 1e-12 * (area @ np.abs(dz))
    assert abs(area @ (H - z) - v0) <= 1e-12 * v0


@pytest.mark.parametrize("angle", [0.0, 30.0])
def test_uniform_flow_box_one_step(angle):
    Lx, Ly, nx, ny = 40.0, 20.0, 40, 20
    xy, tri, tag = W.rect_mesh(nx, ny, Lx, Ly, jitter=0.0, side_tags=(W.WALL, W.WALL, W.WALL, W.WALL))
    N = len(tri)
    ux, uy = 1.2 * math.cos(math.radians(angle)), 1.2 * math.sin(math.radians(angle))
    s = W.Scenario("box", xy, tri, np.zeros(N), np.full(N, 0.03), tag, np.full(N, 0.5), np.full(N, 0.5 * ux),
                   np.full(N, 0.5 * uy), W.default_params())
    st, o = both(s)
    st.step(1)
    o.step(1)
    z = st.download_bed()
    assert np.max(np.abs(z - o.z)) <= 1e-12 * np.max(np.abs(o.z))
    assert np.max(np.abs(o.z)) > 0


def test_channel_inflow_outlet_fp64():
    """Sloping sand channel fed at capacity at the inflow, transmissive outlet, a bump:
    parity after 1,000 steps."""
    L, Wd, S, n, q = 200.0, 4.0, 0.001, 0.02, 1.0
    xy, tri, tag = W.rect_mesh(100, 4, L, Wd, jitter=0.15, seed=2,
                               side_tags=(W.INFLOW, W.TRANSMISSIVE, W.WALL, W.WALL))
    c = xy[tri].mean(axis=1)
    N = len(tri)
    z = S * (L - c[:, 0]) + 0.05 * np.exp(-((c[:, 0] - 80.0) / 6.0) ** 2)
    hn = (n * q / math.sqrt(S)) ** 0.6
    H = np.maximum(S * (L - c[:, 0]) + hn, z)
    s = W.Scenario("channel", xy, tri, z, np.full(N, n), tag, H, np.full(N, q), np.zeros(N),
                   W.default_params(hydro_t=np.array([0.0, 1e9]), hydro_q=np.array([q * Wd, q * Wd])))
    st, o = both(s)
    st.step(1000)
    o.step(1000)
    compare(s, st, o)


def test_morpho_api_rules():
    s = W.dam_break(nx=40, ny=4, manning=0.03)
    st32 = bm.State.from_scenario(s, precision="fp32")
    with pytest.raises(bm.BMError, match="FP64"):
        st32.set_morpho(**SAND)
    st = bm.State.from_scenario(s)
    with pytest.raises(bm.BMError, match="porosity"):
        st.set_morpho(**dict(SAND, porosity=1.0))
    st.set_morpho(**SAND)
    st.step(20)
    z1 = st.download_bed()
    assert np.max(np.abs(z1 - s.z)) > 0
    st.set_morpho(on=False)
    st.step(20)
    assert np.array_equal(st.download_bed(), z1)
