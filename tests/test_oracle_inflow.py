"""Pins of the oracle's discharge-inflow boundary (the standard inflow boundary of the
paper's boundary-condition list: a discharge hydrograph Q(t) with a uniform-flow
distribution along the boundary), against what the physics of uniform flow and the
time-step criterion of Eq. 21 fix.

Reading under test: the unit discharge of inflow edge e is q_e = Q l_e h_e^(5/3) /
(l_e sum_f l_f h_f^(5/3)) over the inflow edges whose cell is wet (uniform Q / sum l
when they are all dry); the boundary depth is h_b = max(h_i, (q_e^2 / g)^(1/3)); the
edge brings the normal-frame flux (-q_e, q_e^2 / h_b + g h_b^2 / 2 - g h_i^2 / 2, 0)
and adds the wave speed lambda_b = q_e / h_b + sqrt(g h_b) to Eq. 21.

A plausible mistake fails one of them: a weight by the depth (or the width) instead of
the conveyance h^(5/3) redistributes the discharge across a channel whose two halves
carry their Manning normal flows; a wrong factor in the imposed momentum flux lifts or
drops the water at the inlet of that channel; a missing or wrong boundary wave speed,
or a wrong critical depth, changes the first time step of a fed cell.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2102_12862_b300 import workloads as W

G = 9.81


def two_depth_channel(nx=80, ny=8, L=400.0, Wd=20.0, S=1e-3, n=0.03, h_deep=1.5, h_shallow=1.0):
    """A sloped channel (bed slope S along x) whose cross-section has two depths: the
    half y < Wd/2 lies (h_deep - h_shallow) lower, so one flat surface covers both
    halves at their Manning normal depths.  Each half carries its normal unit discharge
    q = h^(5/3) S^(1/2) / n (Eq. 2 with Manning's c_f, Table 1); the inflow side x = 0
    brings their sum Q, the outlet x = L is transmissive, the banks are walls."""
    xy, tri, tag = W.rect_mesh(nx, ny, L, Wd, jitter=0.0,
                               side_tags=(W.INFLOW, W.TRANSMISSIVE, W.WALL, W.WALL))
    c = xy[tri].mean(axis=1)
    N = len(tri)
    deep = c[:, 1] < Wd / 2
    z = S * (L - c[:, 0]) - np.where(deep, h_deep - h_shallow, 0.0)
    h = np.where(deep, h_deep, h_shallow)
    q = h ** (5.0 / 3.0) * math.sqrt(S) / n
    Q = (h_deep ** (5.0 / 3.0) + h_shallow ** (5.0 / 3.0)) * math.sqrt(S) / n * Wd / 2
    s = W.Scenario("two_depth_channel", xy, tri, z, np.full(N, n), tag, z + h, q, np.zeros(N),
                   W.default_params(hydro_t=np.array([0.0, 1e9]), hydro_q=np.array([Q, Q])))
    return s, c, deep


def test_inflow_split_keeps_both_halves_at_their_normal_flow():
    """The conveyance split hands each half of the two-depth channel its own normal
    discharge (q_deep / q_shallow = (1.5 / 1.0)^(5/3) = 1.97), so after 600 s (two
    residence times) the first cell row next to the inflow carries the same unit
    discharge and depth as the rows 150-250 m downstream, in both halves, within the
    scheme's discretisation error (1.2 % measured; bar 3 %).  A split by depth would
    give the halves 1.88 and 1.25 m^2/s instead of 2.07 and 1.05 (-9 % / +14 % at the
    inlet); a wrong momentum flux moves the inlet depth by tens of per cent."""
    s, c, deep = two_depth_channel()
    o = oracle.Oracle(s)
    o.run_until(600.0)
    x = c[:, 0]
    first, far = x < 5.0, (x > 150.0) & (x < 250.0)
    h = o.depth()
    for half in (deep, ~deep):
        q1, qf = o.qx[first & half].mean(), o.qx[far & half].mean()
        h1, hf = h[first & half].mean(), h[far & half].mean()
        assert abs(q1 / qf - 1.0) < 0.03, (q1, qf)
        assert abs(h1 / hf - 1.0) < 0.03, (h1, hf)
        assert np.abs(o.qy[first & half]).max() < 0.03 * qf
    # and the whole inflow enters: the boundary volume balances the storage change
    assert o.boundary_volume != 0.0


def _fed_strip(h0: float, Q: float, a: float = 2.0, nx: int = 4):
    """One row of nx square quads of side a (2 nx right triangles), the x = 0 side an
    inflow edge of length a (one triangle holds it), walls elsewhere, flat bed, water
    at rest of depth h0 everywhere (h0 = 0: dry)."""
    xy, tri, tag = W.rect_mesh(nx, 1, nx * a, a, jitter=0.0, side_tags=(W.INFLOW, W.WALL, W.WALL, W.WALL))
    N = len(tri)
    s = W.Scenario("strip", xy, tri, np.zeros(N), np.zeros(N), tag, np.full(N, h0), np.zeros(N), np.zeros(N),
                   W.default_params(cfl=0.9, hydro_t=np.array([0.0, 1e9]), hydro_q=np.array([Q, Q])))
    return s


def test_inflow_wave_speed_in_eq21_dry_cell():
    """A dry strip fed by Q: all inflow cells dry, so q_e = Q / a; the boundary depth is
    the critical depth h_c = (q^2 / g)^(1/3) and lambda_b = q / h_c + sqrt(g h_c) =
    2 (g q)^(1/3) (critical flow, Froude 1).  Nothing else moves, so Eq. 21 gives
    dt = CFL rho / lambda_b with rho = 4 |Omega| / (3 l) = 2 a / 3 for the fed right
    triangle (legs a)."""
    a, Q = 2.0, 3.0
    s = _fed_strip(0.0, Q, a=a)
    q = Q / a
    want = 0.9 * (2.0 * a / 3.0) / (2.0 * (G * q) ** (1.0 / 3.0))
    o = oracle.Oracle(s)
    got = o.next_dt()
    assert abs(got - want) <= 1e-14 * want, (got, want)
    # positivity bound (cfl_mode 1): |Omega| / (l lambda_b) = a / (2 lambda_b)
    o1 = oracle.Oracle(s, cfl_mode=1)
    want1 = 0.9 * (a / 2.0) / (2.0 * (G * q) ** (1.0 / 3.0))
    assert abs(o1.next_dt() - want1) <= 1e-14 * want1
    # the first step brings exactly Q dt into the fed cell, and only there
    o.step(1)
    area = o.area()
    dv = area * o.depth()
    assert abs(dv.sum() - Q * got) <= 1e-13 * Q * got
    assert np.count_nonzero(dv) == 1


def test_inflow_wave_speed_in_eq21_wet_cell():
    """Water at rest, depth 2 m, fed by q = 5 m^2/s: h_c = 1.37 m < 2 m so h_b = 2 m and
    lambda_b = q / h + sqrt(g h) = 6.93 m/s on the inflow edge (rho = 2a/3) beats every
    cell's own sqrt(g h) = 4.43 m/s (rho >= sqrt(2) a / 3): dt = CFL (2a/3) / lambda_b."""
    a, h0, q = 2.0, 2.0, 5.0
    s = _fed_strip(h0, q * a, a=a)
    c = math.sqrt(G * h0)
    lam_b = q / h0 + c
    want = 0.9 * (2.0 * a / 3.0) / lam_b
    assert want < 0.9 * (math.sqrt(2.0) * a / 3.0) / c  # the boundary edge decides
    got = oracle.Oracle(s).next_dt()
    assert abs(got - want) <= 1e-14 * want, (got, want)


def test_inflow_into_dry_cells_is_uniform_along_the_boundary():
    """All inflow cells dry: the discharge is spread uniformly per unit length
    (q_e = Q / sum l), so after one step every fed cell holds q_e l_e dt, whatever the
    edge lengths (a jittered inflow side)."""
    Q = 40.0
    xy, tri, tag = W.rect_mesh(10, 7, 50.0, 35.0, jitter=0.2, seed=3,
                               side_tags=(W.INFLOW, W.WALL, W.WALL, W.WALL))
    # uneven inflow edges: move the inner nodes of the x = 0 side along it
    side = (xy[:, 0] == 0.0) & (xy[:, 1] > 0.0) & (xy[:, 1] < 35.0)
    xy[side, 1] += np.random.default_rng(3).uniform(-1.5, 1.5, side.sum())
    N = len(tri)
    s = W.Scenario("fed_plane", xy, tri, np.zeros(N), np.zeros(N), tag, np.zeros(N), np.zeros(N), np.zeros(N),
                   W.default_params(hydro_t=np.array([0.0, 1e9]), hydro_q=np.array([Q, Q])))
    o = oracle.Oracle(s)
    L, R, nx, ny, ln = o.edges()
    fed = R == -3
    assert fed.sum() == 7
    dt = o.next_dt()
    o.step(1)
    vol = o.area() * o.depth()
    want = np.zeros(N)
    np.add.at(want, L[fed], Q / ln[fed].sum() * ln[fed] * dt)
    assert np.allclose(vol, want, rtol=1e-13, atol=0.0)
    assert len(set(np.round(ln[fed], 9))) > 1  # the lengths differ
