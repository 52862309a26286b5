"""Passive species on the GPU (the step kernel's exported edge mass fluxes and upwind
sides, then the species kernel) against the oracle (Section "Scalar
advection-diffusion", Eq. 8 with the diffusion and source terms off).

FP64: q_c = h phi_c within relative L-inf 1e-11 of the oracle's (normwise per species,
as the state parity: 1e-10 after more than 400 steps), the steady contact of Section
T5 kept to 1e-12, a uniform concentration kept uniform to 1e-12, species mass
conserved in a closed domain to 1e-12 relative.  FP32-bulk: phi within that mode's
accuracy (its depth bar is 1e-4 m L1 on metre depths, so 1e-3 in the area-weighted
mean of |phi - phi_oracle| over wet cells, and species mass within 1e-4 relative).
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


def both(s, hc, c_in=None, precision="fp64", **kw):
    st = bm.State.from_scenario(s, precision=precision, **kw)
    o = oracle.Oracle(s, **kw)
    st.set_scalars(hc, c_in)
    o.set_scalars(hc, c_in)
    return st, o


def compare_fp64(st, o):
    tol = 1e-10 if o.steps > 400 else 1e-11
    g, r = st.download_scalars(), o.hc
    for c in range(r.shape[0]):
        e = rel_linf(g[c], r[c])
        assert e <= tol, f"species {c}: rel Linf {e:.3e} ({o.steps} steps)"
    return g


def test_t5_steady_contact_fp64():
    """Section T5: phi = 1 left of x = 50 m, 0 right, under two diverging rarefactions;
    the contact stays in place exactly, and the GPU equals the oracle."""
    s = W.two_rarefaction()
    x = s.centroids()[:, 0]
    phi0 = np.where(x < 50.0, 1.0, 0.0)
    h0 = np.maximum(s.H - s.z, 0.0)
    st, o = both(s, phi0 * h0)
    st.run_until(2.5)
    o.run_until(2.5)
    compare_fp64(st, o)
    H, _, _, _ = st.download()
    wet = H - s.z > 1e-3
    assert wet.mean() > 0.9
    assert np.max(np.abs(st.concentration()[0][wet] - phi0[wet])) <= 1e-12


def test_uniform_concentration_fp64():
    s = W.dam_break(manning=0.03)
    h0 = np.maximum(s.H - s.z, 0.0)
    st, o = both(s, np.stack([0.7 * h0, 0.2 * h0]))
    st.step(300)
    o.step(300)
    compare_fp64(st, o)
    H, _, _, _ = st.download()
    wet = H - s.z > 1e-3
    phi = st.concentration()
    assert np.max(np.abs(phi[0][wet] - 0.7)) <= 1e-12
    assert np.max(np.abs(phi[1][wet] - 0.2)) <= 1e-12


@pytest.mark.parametrize("seed", [31, 32])
def test_random_wet_dry_closed_fp64(seed):
    """Random wet/dry state with friction in a closed domain (several tiles and a ragged
    last tile): element-wise parity and species mass to 1e-12 relative."""
    s = W.random_state(W.dam_break(nx=150, ny=20, seed=seed, closed=True, manning=0.02), seed=seed)
    rng = np.random.default_rng(seed)
    h0 = np.maximum(s.H - s.z, 0.0)
    hc = rng.uniform(0, 1, (3, len(h0))) * h0
    st, o = both(s, hc, cfl_mode=1)
    area = o.area()
    m0 = hc @ area
    st.step(250)
    o.step(250)
    g = compare_fp64(st, o)
    assert np.all(np.abs(g @ area - m0) <= 1e-12 * np.abs(m0))


def test_inflow_front_fp64():
    """Uniform channel flow with c_in = 1 at the inflow and a transmissive outlet: the
    front the oracle advects, element for element."""
    L, Wd, S, n, Q = 1000.0, 20.0, 1e-3, 0.03, 20.0
    xy, tri, tag = W.rect_mesh(200, 6, L, Wd, jitter=0.2, side_tags=(W.INFLOW, W.TRANSMISSIVE, W.WALL, W.WALL),
                               seed=4)
    c = xy[tri].mean(axis=1)
    N = len(tri)
    z = S * (L - c[:, 0])
    hn = (Q / Wd * n / math.sqrt(S)) ** 0.6
    s = W.Scenario("uniform_flow", xy, tri, z, np.full(N, n), tag, z + hn, np.full(N, Q / Wd), np.zeros(N),
                   W.default_params(hydro_t=np.array([0.0, 1e9]), hydro_q=np.array([Q, Q])))
    st, o = both(s, np.zeros((2, N)), c_in=[1.0, 0.25])
    st.run_until(200.0)
    o.run_until(200.0)
    g = compare_fp64(st, o)
    assert g[0].max() > 0.5  # the front entered
    phi = st.concentration()
    assert phi[1].max() <= 0.25 + 1e-12


def test_floodplain_fp32_within_its_accuracy():
    """Inflow hydrograph over a dry floodplain with a species entering at c_in = 1 and a
    second one initially in the river: FP32-bulk against the FP64 oracle."""
    s = W.floodplain(nx=160, ny=64, Lx=1600.0, Ly=640.0, seed=23, q_peak=150.0, ramp=120.0)
    h0 = np.maximum(s.H - s.z, 0.0)
    st, o = both(s, np.stack([np.zeros_like(h0), 0.5 * h0]), c_in=[1.0, 0.0], precision="fp32")
    st.run_until(200.0)
    o.run_until(200.0)
    area = o.area()
    g, r = st.download_scalars(), o.hc
    for c in range(2):
        assert abs(g[c] @ area - r[c] @ area) <= 1e-4 * abs(r[c] @ area)
    wet = o.depth() > 1e-3
    dphi = np.abs(st.concentration() - o.concentration())[:, wet]
    assert np.all(dphi @ area[wet] / area[wet].sum() <= 1e-3)


def test_species_follow_upload_and_removal():
    """Uploading a state keeps the species; zero species removes them; a batch refuses a
    state with species."""
    s = W.dam_break(nx=40, ny=4, manning=0.02)
    h0 = np.maximum(s.H - s.z, 0.0)
    st = bm.State.from_scenario(s)
    st.set_scalars(0.3 * h0[None, :])
    st.step(3)  # odd: the state sits in buffer 1
    before = st.download_scalars()
    H, qx, qy, t = st.download()
    st.upload(H, qx, qy, t)
    assert np.array_equal(st.download_scalars(), before)
    b = bm.Batch([st])  # a batch made before the species change below
    st.set_scalars(np.zeros((0, st.n_cells)))
    with pytest.raises(bm.BMError, match="changed after bm_batch_create"):
        b.step(1)
    with pytest.raises(bm.BMError, match="carries no species"):
        st.download_scalars()
    with pytest.raises(bm.BMError, match="n_species"):
        st.set_scalars(np.zeros((6, st.n_cells)))
    st.step(2)  # the state steps on without species


def test_t6_three_humps_fp64():
    """Section T6's two species (Eq. 24) in the dam break over three humps: wet/dry
    fronts over the humps, friction, walls; element-wise parity after 30 s and the
    paper's mixed values (species mass over water volume) kept."""
    s = W.three_humps(nx=75, ny=30)
    x = s.centroids()[:, 0]
    h0 = np.maximum(s.H - s.z, 0.0)
    hc = np.stack([np.where(x < 16.0, 0.5, 0.0) * h0, np.where(x < 16.0, 0.0, 0.1) * h0])
    st, o = both(s, hc)
    st.run_until(30.0)
    o.run_until(30.0)
    g = compare_fp64(st, o)
    area = o.area()
    H, _, _, _ = st.download()
    mean = (g @ area) / np.sum(area * (H - s.z))
    assert abs(mean[0] - 0.386) <= 5e-4 and abs(mean[1] - 0.023) <= 5e-4


@pytest.mark.parametrize("seed", [41, 42])
def test_species_with_rain_and_a_sink_fp64(seed):
    """Species together with external sources (Eq. 8 with its source term off: the
    sources' water carries no species): a dam break with friction under rain on one
    region and an Available sink on another, 300 steps; q_c and the state element-wise
    against the oracle."""
    s = W.dam_break(nx=150, ny=20, seed=seed, manning=0.02)
    h0 = np.maximum(s.H - s.z, 0.0)
    x = s.centroids()[:, 0]
    st, o = both(s, np.stack([np.where(x < 30.0, 1.0, 0.3) * h0, 0.5 * h0]), c_in=None)
    region = np.where(x < 20.0, 0, np.where(x > 70.0, 1, -1)).astype(np.int32)
    series = [(np.array([0.0, 2.0]), np.array([3600.0, 720.0])), (np.array([0.0]), np.array([-1800.0]))]
    args = (region, [bm.SOURCE_INTENSITY, bm.SOURCE_INTENSITY], [bm.SINK_EXACT, bm.SINK_AVAILABLE], series)
    st.set_sources(*args)
    o.set_sources(*args)
    st.step(300)
    o.step(300)
    compare_fp64(st, o)
    H, qx, qy, _ = st.download()
    assert rel_linf(H - s.z, o.H - s.z) <= 1e-11
    assert rel_linf(qx, o.qx) <= 1e-11 and rel_linf(qy, o.qy) <= 1e-11


def test_rain_dilutes_species_fp32():
    """FP32-bulk: rain on a lake at rest dilutes each cell's concentration to
    phi0 h0 / (h0 + i t) (closed form) within that mode's accuracy."""
    s = W.fractal_lake(nx=40, ny=20, Lx=400.0, Ly=200.0, seed=11, relief=5.0, level=406.0)
    h0 = s.H - s.z
    phi0 = np.random.default_rng(5).uniform(0.2, 1.0, len(h0))
    st = bm.State.from_scenario(s, precision="fp32")
    st.set_scalars(np.stack([phi0 * h0]))
    st.set_sources(np.zeros(len(h0), dtype=np.int32), [bm.SOURCE_INTENSITY], [bm.SINK_EXACT],
                   [(np.array([0.0]), np.array([36.0]))])
    st.run_until(200.0)
    phi = st.concentration()[0]
    assert np.max(np.abs(phi - phi0 * h0 / (h0 + 1e-5 * 200.0))) <= 1e-5
