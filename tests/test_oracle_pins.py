"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test would fail on a plausible mistake in the oracle: a dropped or
wrong-signed pressure correction (lake at rest), a wrong wave speed or flux
(Stoker, Ritter, T5 closed forms), a leaking boundary (mass), a transposed
normal or index (mirror / rotation symmetry, free-stream preservation), a
wrong rho_ij or lambda_ij (hand-computed CFL step), a wrong friction stage
(closed form and the exact ODE), or a wrong rest level (paper value of T6).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2102_12862_b300 import workloads as W
from tests import riemann_exact as RX

G = 9.81
GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _cells_x(s):
    return s.centroids()[:, 0]


# ------------------------------------------------------------------ point pieces

def test_hllc_consistency_equal_states():
    """F(U, U) is the physical flux (h u, h u^2 + g h^2/2, h u v), exactly."""
    rng = np.random.default_rng(0)
    for _ in range(200):
        h = rng.uniform(1e-4, 5.0)
        u, v = rng.uniform(-8, 8, 2)
        F = oracle.hllc(h, u, v, h, u, v, G)
        assert F[0] == h * u
        assert F[1] == h * u * u + 0.5 * G * h * h
        assert F[2] == h * u * v


def test_hllc_antisymmetry():
    """Swapping sides and reversing the normal reverses the mass flux and keeps the
    momentum-flux vector: F(L, R; n) = -F(R, L; -n) to round-off (the HLL form is
    written from the left state, so it is not bitwise symmetric; edges are therefore
    always evaluated in one canonical orientation)."""
    rng = np.random.default_rng(1)
    for _ in range(500):
        hL, hR = rng.uniform(0, 3, 2) * (rng.random(2) > 0.15)
        uL, vL, uR, vR = rng.uniform(-6, 6, 4)
        F = oracle.hllc(hL, uL, vL, hR, uR, vR, G)
        Fr = oracle.hllc(hR, -uR, -vR, hL, -uL, -vL, G)
        tol = 1e-14 * (1 + np.abs(F).max())
        assert abs(F[0] + Fr[0]) <= tol
        assert abs(F[1] - Fr[1]) <= tol
        assert abs(F[2] - Fr[2]) <= tol


def test_wave_speeds_bracket_exact_riemann_waves():
    """The HLL speeds must bound the exact waves (Einfeldt's condition for a positive,
    entropy-satisfying HLL flux): S_L <= slowest exact signal, S_R >= fastest.  The
    exact speeds come from the exact Riemann solution (shock speeds from
    Rankine-Hugoniot, rarefaction heads u -+ c, dry fronts u +- 2c).  The
    two-rarefaction star estimate can miss a strong shock by a fraction of a
    percent, hence the 1 % allowance."""
    rng = np.random.default_rng(4)
    n_checked = 0
    for _ in range(3000):
        hL, hR = rng.uniform(0.01, 5.0, 2)
        uL, uR = rng.uniform(-5, 5, 2)
        try:
            hs, us = RX.star_state(hL, uL, hR, uR)
        except ValueError:
            continue
        cL, cR = math.sqrt(G * hL), math.sqrt(G * hR)
        exL = uL - cL * math.sqrt(0.5 * (hs + hL) * hs / hL ** 2) if hs > hL else uL - cL
        exR = uR + cR * math.sqrt(0.5 * (hs + hR) * hs / hR ** 2) if hs > hR else uR + cR
        SL, SR = oracle.wave_speeds(hL, uL, hR, uR)
        assert SL <= exL + 0.01 * abs(exL) + 1e-12 and SR >= exR - 0.01 * abs(exR) - 1e-12
        n_checked += 1
    assert n_checked > 2000
    # dry right side: the exact waves are the left rarefaction head and the dry front
    SL, SR = oracle.wave_speeds(1.0, 0.5, 0.0, 0.0)
    assert SL == 0.5 - math.sqrt(G) and SR == 0.5 + 2 * math.sqrt(G)
    SL, SR = oracle.wave_speeds(0.0, 0.0, 2.0, -1.0)
    assert SL == -1.0 - 2 * math.sqrt(2 * G) and SR == -1.0 + math.sqrt(2 * G)


def test_hllc_supersonic_upwind():
    """All waves to the right: the flux is the left physical flux (and vice versa)."""
    h, u = 1.0, 10.0  # Froude > 1
    F = oracle.hllc(h, u, 0.3, 0.5, u, -0.2, G)
    assert F[0] == h * u and F[1] == h * u * u + 0.5 * G * h * h and F[2] == h * u * 0.3
    F = oracle.hllc(0.5, -u, 0.1, h, -u, 0.7, G)
    assert F[0] == -h * u and F[2] == -h * u * 0.7


def test_hllc_symmetric_rarefactions_and_contact():
    """Symmetric two-rarefaction problem: the exact Godunov mass flux h* u* is 0 and so
    is the HLLC one; the tangential velocity is carried by the contact: upwind of the
    sign of the mass flux."""
    hL, uL, hR, uR = 1.0, -1.0, 1.0, 1.0
    hs, us = RX.star_state(hL, uL, hR, uR)
    F = oracle.hllc(hL, uL, 0.7, hR, uR, -0.4, G)
    assert abs(F[0] - hs * us) < 1e-12
    F = oracle.hllc(1.0, 0.5, 0.7, 1.0, 0.5, -0.4, G)
    assert F[0] > 0 and F[2] == F[0] * 0.7
    F = oracle.hllc(1.0, -0.5, 0.7, 1.0, -0.5, -0.4, G)
    assert F[0] < 0 and F[2] == F[0] * -0.4


def test_friction_closed_form_and_exact_ode():
    """Two semi-implicit stages combined as Heun: q = q0 (1 + a) / (1 + 2a) with
    a = dt g n^2 |q0| / h^(7/3) (hand algebra of the stages); as dt -> 0 the step
    approaches the exact solution q0 / (1 + a) of dq/dt = -g n^2 |q| q / h^(7/3)
    with an error O(a^2); direction is kept and the flow never reverses."""
    rng = np.random.default_rng(2)
    for _ in range(200):
        h = rng.uniform(0.01, 3.0)
        n = rng.uniform(0.01, 0.1)
        dt = rng.uniform(1e-3, 5.0)
        qx, qy = rng.uniform(-5, 5, 2)
        q0 = math.hypot(qx, qy)
        a = dt * G * n * n * q0 / h ** (7.0 / 3.0)
        fx, fy = oracle.friction(h, n, dt, qx, qy)
        ratio = (1 + a) / (1 + 2 * a)
        assert abs(fx - qx * ratio) <= 1e-13 * abs(qx) + 1e-300
        assert abs(fy - qy * ratio) <= 1e-13 * abs(qy) + 1e-300
        assert abs(fx) <= abs(qx) and abs(fy) <= abs(qy)
        assert fx * qx >= 0 and fy * qy >= 0
    # convergence to the exact ODE solution
    h, n, q0 = 0.5, 0.05, 2.0
    T = 10.0
    errs = []
    for steps in (10, 20, 40, 80):
        dt = T / steps
        qx = q0
        for _ in range(steps):
            qx, _ = oracle.friction(h, n, dt, qx, 0.0)
        exact = q0 / (1 + T * G * n * n * q0 / h ** (7.0 / 3.0))
        errs.append(abs(qx - exact))
    for a, b in zip(errs, errs[1:]):
        assert b < 0.6 * a  # converges (first order in dt for this ODE)
    # below the minimum depth nothing happens
    assert oracle.friction(1e-7, 0.05, 1.0, 1e-9, 0.0) == (1e-9, 0.0)


def test_hydrograph_piecewise_linear():
    assert oracle.hydrograph([0, 600, 1e9], [0, 500, 500], 300.0) == 250.0
    assert oracle.hydrograph([0, 600, 1e9], [0, 500, 500], 1e4) == 500.0
    assert oracle.hydrograph([10, 20], [1, 3], 0.0) == 1.0


# ------------------------------------------------------------------ invariants

def test_lake_at_rest_bitwise_fp64():
    """C-property: still water over a rough bed with dry islands stays bitwise still
    (Section "Hydrodynamics" numerics: modified-state bed treatment)."""
    s = W.fractal_lake(nx=40, ny=20, Lx=400.0, Ly=200.0, seed=11, relief=5.0, level=403.0)
    assert (s.H > s.z).any() and (s.H == s.z).any()
    o = oracle.Oracle(s)
    H0 = o.H.copy()
    o.step(2000)
    assert np.array_equal(o.H, H0)
    assert not o.qx.any() and not o.qy.any()


def test_lake_at_rest_open_boundaries():
    """Transmissive and (zero-discharge) inflow boundaries also keep still water still."""
    s = W.floodplain(nx=30, ny=12, Lx=300.0, Ly=120.0, seed=12, q_peak=0.0, outlet=W.TRANSMISSIVE)
    level = np.median(s.z) + 0.5
    s.H = np.maximum(s.z, level)
    o = oracle.Oracle(s)
    H0 = o.H.copy()
    o.step(500)
    assert np.array_equal(o.H, H0)
    assert not o.qx.any() and not o.qy.any()


def test_free_stream_preservation():
    """A uniform flow on a flat bed with transmissive boundaries everywhere stays
    uniform: sum_j l_ij n_ij = 0 for each closed triangle (Eq. 12)."""
    xy, tri, tag = W.rect_mesh(20, 10, 20.0, 10.0, jitter=0.2, seed=3,
                               side_tags=(W.TRANSMISSIVE,) * 4)
    n = len(tri)
    s = W.Scenario("uniform", xy, tri, np.zeros(n), np.zeros(n), tag, np.full(n, 1.5),
                   np.full(n, 1.2), np.full(n, -0.7), W.default_params())
    o = oracle.Oracle(s)
    o.step(50)
    assert np.max(np.abs(o.H - 1.5)) < 1e-13
    assert np.max(np.abs(o.qx - 1.2)) < 1e-13
    assert np.max(np.abs(o.qy + 0.7)) < 1e-13


def test_mass_closed_domain():
    """Closed domain: (V_n - V_0) / V_0 at round-off, wet/dry included."""
    s = W.dam_break(closed=True, h_right=0.0, manning=0.03)
    o = oracle.Oracle(s)
    v0 = o.volume()
    o.step(1500)
    assert abs(o.volume() - v0) / v0 < 1e-13
    s = W.random_state(W.dam_break(nx=40, ny=8, closed=True), seed=5)
    o = oracle.Oracle(s, cfl_mode=1)
    v0 = o.volume()
    o.step(300)
    assert abs(o.volume() - v0) / v0 < 1e-13


def test_mass_open_domain_balance():
    """Open domain with inflow and outflow: V_n - V_0 equals the boundary volume."""
    s = W.floodplain(nx=40, ny=16, Lx=500.0, Ly=200.0, seed=13, q_peak=50.0, ramp=60.0, outlet=W.TRANSMISSIVE)
    o = oracle.Oracle(s)
    v0 = o.volume()
    o.run_until(200.0)
    assert o.boundary_volume > 0
    assert abs(o.volume() - v0 - o.boundary_volume) / (v0 + o.boundary_volume) < 1e-12
    # with the outlet closed, the boundary volume is the hydrograph volume sum_n Q(t^n) dt^n:
    # a left Riemann sum of the ramp, just below its integral 50 * (200 - 30) = 8500 m^3
    s.edge_tag[s.edge_tag == W.TRANSMISSIVE] = W.WALL
    o = oracle.Oracle(s)
    v0 = o.volume()
    o.run_until(200.0)
    assert 8400.0 < o.boundary_volume <= 8500.0
    assert abs(o.volume() - v0 - o.boundary_volume) / (v0 + o.boundary_volume) < 1e-12


def test_mirror_symmetry():
    """run(mirror(mesh)) = mirror(run(mesh)) to round-off."""
    s = W.dam_break(nx=60, ny=6, jitter=0.15, seed=7, h_right=0.0)
    s.qy = np.random.default_rng(7).uniform(-0.1, 0.1, s.n_cells) * s.H
    m = W.mirror_x(s)
    a, b = oracle.Oracle(s), oracle.Oracle(m)
    a.step(120)
    b.step(120)
    assert abs(a.time - b.time) < 1e-12 * a.time
    assert np.max(np.abs(a.H - b.H)) < 1e-11
    assert np.max(np.abs(a.qx + b.qx)) < 1e-11
    assert np.max(np.abs(a.qy - b.qy)) < 1e-11


def test_rotation_90():
    """Exact coordinate swap (x, y) -> (-y, x): the rotated run equals the rotated state."""
    s = W.random_state(W.dam_break(nx=20, ny=8, jitter=0.2, seed=9), seed=9)
    r = W.rotate_90(s)
    a, b = oracle.Oracle(s), oracle.Oracle(r)
    a.step(40)
    b.step(40)
    assert abs(a.time - b.time) < 1e-12 * a.time
    assert np.max(np.abs(a.H - b.H)) < 1e-11
    assert np.max(np.abs(-a.qy - b.qx)) < 1e-11
    assert np.max(np.abs(a.qx - b.qy)) < 1e-11


def test_cfl_step_by_hand():
    """Eq. 21 on a uniform state of a regular right-isosceles mesh (legs a):
    rho = 2a/3 on the legs, sqrt(2) a/3 on the hypotenuse; lambda = |u.n| + sqrt(g h)."""
    a = 0.5
    xy, tri, tag = W.rect_mesh(10, 10, 10 * a, 10 * a, jitter=0.0, side_tags=(W.WALL,) * 4)
    n = len(tri)
    h, U, V = 1.3, 0.8, -0.3
    s = W.Scenario("u", xy, tri, np.zeros(n), np.zeros(n), tag, np.full(n, h), np.full(n, h * U),
                   np.full(n, h * V), W.default_params(cfl=0.9))
    c = math.sqrt(G * h)
    legs = [2 * a / 3 / (abs(U) + c), 2 * a / 3 / (abs(V) + c)]
    hyp = [math.sqrt(2) * a / 3 / (abs(U + V) / math.sqrt(2) + c),
           math.sqrt(2) * a / 3 / (abs(U - V) / math.sqrt(2) + c)]
    want = 0.9 * min(legs + hyp)
    got = oracle.Oracle(s).next_dt()
    assert abs(got - want) < 1e-14 * want
    # dt_max caps it; a dry domain without inflow takes dt_max
    s.H = s.z.copy()
    s.qx[:] = 0
    s.qy[:] = 0
    assert oracle.Oracle(s, dt_max=0.7).next_dt() == 0.7


# ------------------------------------------------------------------ closed-form flows

def test_steady_uniform_manning_flow():
    """Uniform flow on a slope (Eq. 2 with Manning's c_f, Table 1): friction balances the
    bed slope at the normal depth h_n = (q n / sqrt(S))^(3/5); starting there with
    q = Q/W, the state stays put (upstream half within 1 %, discharge within 2 %)."""
    L, Wd, S, n, Q = 1000.0, 20.0, 1e-3, 0.03, 20.0
    xy, tri, tag = W.rect_mesh(100, 4, L, Wd, jitter=0.0, side_tags=(W.INFLOW, W.TRANSMISSIVE, W.WALL, W.WALL))
    c = xy[tri].mean(axis=1)
    N = len(tri)
    z = S * (L - c[:, 0])
    hn = (Q / Wd * n / math.sqrt(S)) ** 0.6
    s = W.Scenario("uniform_flow", xy, tri, z, np.full(N, n), tag, z + hn, np.full(N, Q / Wd), np.zeros(N),
                   W.default_params(hydro_t=np.array([0.0, 1e9]), hydro_q=np.array([Q, Q])))
    o = oracle.Oracle(s)
    o.run_until(2000.0)
    up = c[:, 0] < 500
    assert abs(o.depth()[up].mean() - hn) < 0.01 * hn
    assert abs(o.qx[up].mean() - Q / Wd) < 0.02 * Q / Wd
    assert np.abs(o.qy[up]).max() < 0.05 * Q / Wd


def _l1_vs_exact(s, o, t, hL, uL, hR, uR, x0=50.0):
    x = _cells_x(s)
    he, ue = RX.sample((x - x0) / t, hL, uL, hR, uR)
    area = o.area()
    return np.sum(area * np.abs(o.depth() - he)) / area.sum(), he, ue


def test_stoker_numbers():
    """The Stoker closed form for h_L = 1, h_R = 0.1 (middle state, shock speed)."""
    hs, us = RX.star_state(1.0, 0.0, 0.1, 0.0)
    assert abs(hs - 0.396175) < 1e-6 and abs(us - 2.321355) < 1e-6
    assert abs(RX.shock_speed_right(1.0, 0.0, 0.1, 0.0) - 3.105134) < 1e-6


@pytest.mark.parametrize("h_right,t_end", [(0.1, 10.0), (0.0, 5.0)])
def test_dam_break_converges_to_closed_form(h_right, t_end):
    """Stoker (wet, t = 10 s) and Ritter (dry, t = 5 s, before the front leaves the
    100 m channel) dam breaks: the L1 depth error falls with refinement
    100 -> 200 -> 400 columns and the middle state / front position are right."""
    errs, lags = [], []
    for nx in (100, 200, 400):
        s = W.dam_break(nx=nx, ny=nx // 20, h_right=h_right, seed=1)
        o = oracle.Oracle(s)
        o.run_until(t_end)
        assert o.time == t_end
        assert o.depth().min() >= -1e-12
        e, he, ue = _l1_vs_exact(s, o, t_end, 1.0, 0.0, h_right, 0.0)
        errs.append(e)
        x = _cells_x(s)
        if h_right == 0:
            # exact wet extent at the 1e-3 m level: h = (2 c_L - xi)^2 / (9 g) = 1e-3
            front = 50 + (2 * math.sqrt(G) - math.sqrt(9 * G * 1e-3)) * t_end
            lags.append(front - x[o.depth() > 1e-3].max())
    assert errs[1] < 0.8 * errs[0] and errs[2] < 0.8 * errs[1]
    assert errs[2] < 0.01
    if h_right > 0:
        plateau = (x > 50 + 0.35 * t_end + 3) & (x < 50 + 3.105 * t_end - 3)
        assert abs(np.mean(o.depth()[plateau]) - 0.396175) < 2e-3
    else:
        # first-order smearing: the front lags, less on finer meshes
        assert lags[1] < lags[0] and lags[2] < lags[1] and 0 <= lags[2] < 5.0


def test_t5_two_rarefaction():
    """Section T5 (Eq. 22): two diverging rarefactions; star depth
    h* = (c - |u|/2)^2 / g = 0.271532 m with u* = 0; L1 error of h and q_x small."""
    p = GOLD["t5_two_rarefaction"]
    hs, us = RX.star_state(p["h_m"], p["qx_left"] / p["h_m"], p["h_m"], p["qx_right"] / p["h_m"])
    assert abs(hs - 0.271532) < 1e-6 and abs(us) < 1e-12
    s = W.two_rarefaction()
    assert s.n_cells == p["cells"] and s.params["cfl"] == p["cfl"]
    for t_end in p["t_end_s"]:
        o = oracle.Oracle(s)
        o.run_until(t_end)
        e, he, ue = _l1_vs_exact(s, o, t_end, 1.0, -3.0, 1.0, 3.0)
        assert e < 0.01
        x = _cells_x(s)
        centre = np.abs(x - 50) < 1.0
        assert abs(np.mean(o.depth()[centre]) - hs) < 0.02
        qe = he * ue
        assert np.sum(np.abs(o.qx - qe)) / len(qe) < 0.05


def test_thacker_moving_shoreline_converges():
    """Planar sloshing in a paraboloid (closed form): the L1 depth error at a quarter
    period falls with refinement."""
    a, h0, A = 3000.0, 10.0, 500.0
    om = math.sqrt(2 * G * h0) / a
    t = 0.25 * 2 * math.pi / om
    errs = []
    for nq in (48, 96, 192):
        s = W.thacker(nq=nq)
        o = oracle.Oracle(s)
        o.run_until(t)
        c = s.centroids()
        he, _, _ = W.thacker_exact(c[:, 0], c[:, 1], t)
        ar = o.area()
        errs.append(np.sum(ar * np.abs(o.depth() - he)) / ar.sum())
    assert errs[1] < 0.8 * errs[0] and errs[2] < 0.8 * errs[1]


@pytest.mark.slow
def test_t6_rest_level_paper_value():
    """Section T6: after the dam break over three humps, friction brings the basin to
    rest at h = 0.364 m (the value the paper prints).  Coarse mesh; the discrete rest
    level from mass balance must match the run and the paper's value."""
    p = GOLD["t6_three_humps"]
    s = W.three_humps(nx=75, ny=30)
    o = oracle.Oracle(s)
    v0 = o.volume()
    o.run_until(1500.0)
    assert abs(o.volume() - v0) / v0 < 1e-12
    area = o.area()
    # discrete rest level: sum_i |Omega_i| max(0, H - z_i) = V (bisection)
    lo, hi = 0.0, 3.0
    for _ in range(100):
        mid = 0.5 * (lo + hi)
        if np.sum(area * np.maximum(0.0, mid - s.z)) > v0:
            hi = mid
        else:
            lo = mid
    h_rest = 0.5 * (lo + hi)
    assert abs(h_rest - p["rest_h_m"]) < 2e-3
    wet = o.depth() > 0.05
    assert abs(np.median(o.H[wet]) - h_rest) < 5e-3
    assert np.max(np.hypot(o.qx, o.qy)) < 0.02
