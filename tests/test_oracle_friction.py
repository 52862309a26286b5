"""Pins of the oracle's friction closures of Table 1 beyond Manning (Chezy's
logarithmic law with K_s, Bezzola's three-branch law with y_R), against closed forms:
one step of uniform flow in a closed box (the interior sees only the friction split,
two semi-implicit stages with k(q) = |q| / (h^2 c_f^2), Eq. 2), in every branch of
each law, and the normal depth of uniform flow on a slope (q = h c_f (g h S)^(1/2)).

A plausible mistake fails one of them: a wrong branch threshold, coefficient or
logarithm base, c_f instead of c_f^2, the Manning form applied to the other laws.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2102_12862_b300 import workloads as W

G = 9.81


def cf_table1(law, h, r):
    """Table 1, written out here: Chezy (r = K_s), Bezzola (r = y_R)."""
    if law == 1:
        return 6.25 + math.log(h / r) if h > r else 6.25
    x = h / r
    if x > 2:
        return 2.5 * math.sqrt(1 - r / h) * math.log(10.9 * h / r)
    if x >= 0.5:
        return 1.25 * math.sqrt(x) * math.log(10.9 * h / r)
    return 1.5


@pytest.mark.parametrize("law,h,r", [(1, 0.8, 0.05), (1, 0.04, 0.05), (2, 0.9, 0.1), (2, 0.15, 0.1),
                                     (2, 0.04, 0.1)])
def test_one_step_in_a_box_is_the_friction_split(law, h, r):
    Lx, Ly, nx, ny = 20.0, 10.0, 20, 10
    xy, tri, tag = W.rect_mesh(nx, ny, Lx, Ly, jitter=0.0, side_tags=(W.WALL, W.WALL, W.WALL, W.WALL))
    N = len(tri)
    q0x, q0y = 0.6 * h, 0.2 * h
    s = W.Scenario("box", xy, tri, np.zeros(N), np.full(N, 0.03), tag, np.full(N, h), np.full(N, q0x),
                   np.full(N, q0y), W.default_params())
    o = oracle.Oracle(s)
    o.set_friction(law, r)
    dt = o.next_dt()
    o.step(1)
    c = s.centroids()
    inner = (c[:, 0] > 1.5) & (c[:, 0] < Lx - 1.5) & (c[:, 1] > 1.5) & (c[:, 1] < Ly - 1.5)
    cf = cf_table1(law, h, r)
    k = 1.0 / (h * h * cf * cf)
    a = dt * k * math.hypot(q0x, q0y)
    q1 = 1.0 / (1 + a)
    q2 = q1 / (1 + dt * k * math.hypot(q0x, q0y) * q1)
    fac = 0.5 * (1 + q2)
    assert fac < 1.0
    assert np.max(np.abs(o.qx[inner] - q0x * fac)) <= 1e-14 * q0x
    assert np.max(np.abs(o.qy[inner] - q0y * fac)) <= 1e-14 * q0y
    assert abs(oracle.friction_cf(law, h, r) - cf) <= 1e-15 * cf


@pytest.mark.slow
@pytest.mark.parametrize("law,r", [(1, 0.02), (2, 0.05)])
def test_normal_depth_on_a_slope(law, r):
    """Uniform flow q = 2 m^2/s on S = 0.002: the depth settles where friction balances
    gravity, q = h c_f(h) (g h S)^(1/2) (bisection here), within 2 %; the tracked bed shear stress rho u^2 / c_f^2 equals
    rho g h S there within 5 %."""
    L, Wd, S, q = 1000.0, 20.0, 0.002, 2.0
    lo, hi = 1e-3, 10.0
    for _ in range(100):
        mid = 0.5 * (lo + hi)
        if mid * cf_table1(law, mid, r) * math.sqrt(G * mid * S) > q:
            hi = mid
        else:
            lo = mid
    hn = 0.5 * (lo + hi)
    xy, tri, tag = W.rect_mesh(100, 4, L, Wd, jitter=0.0, side_tags=(W.INFLOW, W.TRANSMISSIVE, W.WALL, W.WALL))
    c = xy[tri].mean(axis=1)
    N = len(tri)
    z = S * (L - c[:, 0])
    s = W.Scenario("uniform_flow", xy, tri, z, np.full(N, 0.03), tag, z + hn, np.full(N, q), np.zeros(N),
                   W.default_params(hydro_t=np.array([0.0, 1e9]), hydro_q=np.array([q * Wd, q * Wd])))
    o = oracle.Oracle(s)
    o.set_friction(law, r)
    o.run_until(1500.0)
    up = (c[:, 0] > 200) & (c[:, 0] < 600)
    assert abs(np.mean(o.depth()[up]) / hn - 1.0) < 0.02
    # the tracked bed shear stress under the law: rho g h S in uniform flow
    o.track(0.01)
    o.run_until(1600.0)
    tau = 1000.0 * G * hn * S
    assert abs(np.mean(o.tracking["tau_max"][up]) / tau - 1.0) < 0.05
