"""Pins of the oracle's flood tracking (the hydrodynamic module's "Flood" outputs:
water front arrival time, maximum depth, flow velocity, specific discharge and bed
shear stress), against closed forms and invariants.

A plausible mistake fails one of them: a wrong threshold test or time level
(Ritter / Stoker arrival times, lake at rest), a maximum taken over the wrong
quantity (Stoker plateau, Ritter upstream), a wrong shear-stress law or exponent
(uniform Manning flow: tau = rho g h S), a missing update (invariants).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2102_12862_b300 import workloads as W

G = 9.81
RHO = 1000.0


def test_lake_at_rest_tracks_nothing():
    """Still water: the maxima are the initial values, bitwise; no velocity, discharge
    or shear; wet cells arrived at t = 0, dry ones never."""
    s = W.fractal_lake(nx=40, ny=20, Lx=400.0, Ly=200.0, seed=11, relief=5.0, level=403.0)
    o = oracle.Oracle(s)
    h0 = o.depth().copy()
    o.track(h_arrival=0.01)
    o.step(300)
    tr = o.tracking
    assert np.array_equal(tr["h_max"], h0)
    assert not tr["u_max"].any() and not tr["q_max"].any() and not tr["tau_max"].any()
    wet = h0 > 0.01
    assert np.all(tr["t_arrival"][wet] == 0.0)
    assert np.all(np.isnan(tr["t_arrival"][~wet]))


def _probe_error(nx, h_right, t_end, h_arr, exact_arrival):
    s = W.dam_break(nx=nx, ny=max(2, nx // 20), h_right=h_right, seed=1)
    o = oracle.Oracle(s)
    o.track(h_arrival=h_arr)
    o.run_until(t_end)
    x = s.centroids()[:, 0]
    return s, o, x


def test_ritter_arrival_times_converge():
    """Dry-bed dam break (h_L = 1 m): depth h reaches x at t = (x - 50) /
    (2 c_0 - 3 sqrt(g h)) (Ritter); arrival times of h = 0.05 m converge to it with
    refinement.  Upstream of the dam the depth only falls: h_max = 1 exactly."""
    h_arr, t_end = 0.05, 5.0
    c0 = math.sqrt(G)
    errs = []
    for nx in (100, 200, 400):
        s, o, x = _probe_error(nx, 0.0, t_end, h_arr, None)
        tr = o.tracking
        probe = (x > 55.0) & (x < 60.0)
        ta_exact = (x[probe] - 50.0) / (2 * c0 - 3 * math.sqrt(G * h_arr))
        assert np.all(np.isfinite(tr["t_arrival"][probe]))
        errs.append(np.mean(np.abs(tr["t_arrival"][probe] - ta_exact) / ta_exact))
        up = x < 49.0
        assert np.all(tr["h_max"][up] == 1.0)
        # beyond the exact wet extent at t_end nothing has arrived
        far = x > 50.0 + 2 * c0 * t_end + 2.0
        assert np.all(np.isnan(tr["t_arrival"][far]))
    assert errs[1] < errs[0] and errs[2] < errs[1]
    assert errs[2] < 0.02


def test_stoker_plateau_and_shock_arrival():
    """Wet-bed dam break (1 m / 0.1 m): behind the shock the depth is the middle state
    h_m = 0.396175 m until the rarefaction tail (speed 0.35 m/s) arrives, so h_max on
    the plateau is h_m; h = 0.2 m arrives with the shock, t = (x - 50) / 3.105134."""
    h_arr, t_end = 0.2, 10.0
    s, o, x = _probe_error(400, 0.1, t_end, h_arr, None)
    tr = o.tracking
    plateau = (x > 50 + 0.35 * t_end + 3) & (x < 50 + 3.105 * t_end - 3)
    assert abs(np.mean(tr["h_max"][plateau]) - 0.396175) < 2e-3
    ta_exact = (x[plateau] - 50.0) / 3.105134
    assert np.mean(np.abs(tr["t_arrival"][plateau] - ta_exact)) < 0.05
    ahead = x > 50 + 3.105 * t_end + 3
    assert np.all(np.isnan(tr["t_arrival"][ahead]))
    assert np.all(np.abs(tr["h_max"][ahead] - 0.1) < 1e-3)


def test_uniform_flow_shear_stress():
    """Uniform flow on a slope: the Manning shear stress rho g n^2 u^2 / h^(1/3) equals
    rho g h S at the normal depth (0.42 m, where h^(1/3) and h^(1/2) differ by 15 %);
    |q| = Q / W and |u| = q / h_n (within 5 %: the run still relaxes)."""
    L, Wd, S, n, Q = 1000.0, 20.0, 1e-3, 0.03, 5.0
    xy, tri, tag = W.rect_mesh(100, 4, L, Wd, jitter=0.0, side_tags=(W.INFLOW, W.TRANSMISSIVE, W.WALL, W.WALL))
    c = xy[tri].mean(axis=1)
    N = len(tri)
    z = S * (L - c[:, 0])
    hn = (Q / Wd * n / math.sqrt(S)) ** 0.6
    s = W.Scenario("uniform_flow", xy, tri, z, np.full(N, n), tag, z + hn, np.full(N, Q / Wd), np.zeros(N),
                   W.default_params(hydro_t=np.array([0.0, 1e9]), hydro_q=np.array([Q, Q])))
    o = oracle.Oracle(s)
    o.run_until(1500.0)
    o.track(h_arrival=0.01)
    o.run_until(2000.0)
    tr = o.tracking
    up = c[:, 0] < 500
    tau = RHO * G * hn * S
    assert abs(np.mean(tr["tau_max"][up]) - tau) < 0.05 * tau
    assert abs(np.mean(tr["q_max"][up]) - Q / Wd) < 0.05 * Q / Wd
    assert abs(np.mean(tr["u_max"][up]) - Q / Wd / hn) < 0.05 * Q / Wd / hn
    assert np.all(tr["t_arrival"][up] == 1500.0)


@pytest.mark.parametrize("seed", [3, 4])
def test_tracking_invariants(seed):
    """On a random wet/dry state with friction: the maxima bound the current values,
    never decrease, and arrival times lie in [t_0, t] and never change once set."""
    s = W.random_state(W.dam_break(nx=40, ny=6, seed=seed, manning=0.03), seed=seed)
    o = oracle.Oracle(s, cfl_mode=1)
    o.track(h_arrival=0.05)
    prev = {k: v.copy() for k, v in o.tracking.items()}
    for _ in range(6):
        o.step(15)
        tr = o.tracking
        h = o.depth()
        q = np.sqrt(o.qx * o.qx + o.qy * o.qy)  # the tracked form
        assert np.all(tr["h_max"] >= h) and np.all(tr["q_max"] >= q)
        for k in ("h_max", "u_max", "q_max", "tau_max"):
            assert np.all(tr[k] >= prev[k])
        a, pa = tr["t_arrival"], prev["t_arrival"]
        assert np.all(a[~np.isnan(pa)] == pa[~np.isnan(pa)])
        assert np.all((a[~np.isnan(a)] >= 0) & (a[~np.isnan(a)] <= o.time))
        assert np.all(np.isnan(a) <= (h <= 0.05))  # wet above the threshold => arrived
        prev = {k: v.copy() for k, v in tr.items()}
