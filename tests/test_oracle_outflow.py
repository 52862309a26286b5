"""Pins of the oracle's outflow boundaries (the h-Q relation and the weir of the paper's
standard-outflow list, with the parameters its appendix names: the h-Q table; the weir
height and Poleni factor) against what the physics fixes.

Reading under test: a weir edge lets q = (2/3) mu sqrt(2 g) eta^(3/2) per unit width
out, eta the head of the cell's surface over the crest (the crest taken at the cell's
bed if it lies below it); the h-Q boundary lets Q(S) out, the rating curve at the
length-weighted mean surface S of its wet cells, split over them by conveyance
l h^(5/3).  The edge flux is that of the boundary state on the cell's outgoing
characteristic (u_n + 2 sqrt(g h) carried from the cell) that carries q, q capped at
the critical discharge (u_n + 2 sqrt(g h))^3 / (27 g); nothing leaving: a wall.

A steady reservoir fed by Q fixes the head over a weir (Poleni) and the stage of an
h-Q outlet (the rating curve's inverse) through mass balance alone; a channel held at
its normal flow fixes the h-Q split between a deep and a shallow half; Ritter's
dam-break solution (critical flow at the dam site, u = c = 2/3 sqrt(g h0)) fixes the
discharge and the boundary wave speed of an outlet that could take more than the
water can bring.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2102_12862_b300 import workloads as W

G = 9.81


def basin(out_tag, Q=10.0, H0=1.4, nx=40, ny=4, L=200.0, Wd=20.0, z=0.0, n=0.03, inflow=True, cfl_mode=1):
    """A flat rectangular basin, inflow Q at x = 0 (or a wall), the outlet at x = L,
    walls along y; 5 m right triangles; Manning n damps the seiches."""
    tags = (W.INFLOW if inflow else W.WALL, out_tag, W.WALL, W.WALL)
    xy, tri, tag = W.rect_mesh(nx, ny, L, Wd, jitter=0.0, side_tags=tags)
    N = len(tri)
    p = W.default_params(cfl_mode=cfl_mode)
    if inflow:
        p = W.default_params(cfl_mode=cfl_mode, hydro_t=np.array([0.0, 1e9]), hydro_q=np.array([Q, Q]))
    return W.Scenario("basin", xy, tri, np.full(N, z), np.full(N, n), tag, np.full(N, H0), np.zeros(N),
                      np.zeros(N), p)


def outlet_cells(o, code):
    L, R, nx, ny, ln = o.edges()
    sel = R == code
    return L[sel], ln[sel]


def poleni_head(q, mu):
    return (q / ((2.0 / 3.0) * mu * math.sqrt(2.0 * G))) ** (2.0 / 3.0)


def energy(o):
    a, h = o.area(), o.depth()
    wet = h > 1e-6
    ke = np.zeros_like(h)
    ke[wet] = 0.5 * (o.qx[wet] ** 2 + o.qy[wet] ** 2) / h[wet]
    return float(np.sum(a * (ke + 0.5 * G * h * h)))


def test_weir_reservoir_steady_head_is_poleni():
    """Fed by Q = 10 m^3/s over 20 m, the basin settles where the weir lets Q out:
    Poleni's head eta = (q / ((2/3) mu sqrt(2g)))^(2/3) = 0.4302 m over the 1 m crest
    (mu = 0.6, q = 0.5 m^2/s), on every weir cell, and the outflow equals Q."""
    Q, Wd, crest, mu = 10.0, 20.0, 1.0, 0.6
    o = oracle.Oracle(basin(W.WEIR, Q=Q))
    o.set_outflow(weir_crest=crest, weir_poleni=mu)
    o.run_until(2400.0)
    cells, ln = outlet_cells(o, -5)
    eta = poleni_head(Q / Wd, mu)
    assert len(cells) == 4
    assert np.abs(o.H[cells] - crest - eta).max() < 1e-7 * eta
    _, qo = o.boundary_discharge()
    L, R, nx, ny, lens = o.edges()
    assert abs(float(np.sum(qo * lens)) - Q) < 1e-7 * Q


def test_weir_crest_below_the_bed_is_a_free_overfall():
    """A crest below the bed counts from the bed: the steady depth at the outlet is
    Poleni's head of the whole depth, h = (q / ((2/3) mu sqrt(2g)))^(2/3)."""
    Q, Wd, mu = 6.0, 20.0, 0.65
    o = oracle.Oracle(basin(W.WEIR, Q=Q, H0=0.5))
    o.set_outflow(weir_crest=-3.0, weir_poleni=mu)
    o.run_until(2400.0)
    cells, _ = outlet_cells(o, -5)
    h = o.depth()[cells]
    want = poleni_head(Q / Wd, mu)
    assert np.abs(h - want).max() < 1e-7 * want


def test_water_below_the_crest_stays_at_rest():
    """Water below the crest cannot leave: the weir is a wall and the basin stays a
    lake at rest, bitwise, over 500 steps (also with the positivity-free Eq. 21)."""
    for cfl_mode in (0, 1):
        s = basin(W.WEIR, H0=0.8, inflow=False, cfl_mode=cfl_mode)
        o = oracle.Oracle(s)
        o.set_outflow(weir_crest=1.0, weir_poleni=0.6)
        o.step(500)
        assert np.array_equal(o.H, s.H)
        assert not np.any(o.qx) and not np.any(o.qy)
        assert o.boundary_volume == 0.0


def test_weir_drain_dissipates_energy():
    """A closed basin draining over the weir loses energy every step and its surface
    never rises above where it started (the outlet adds nothing)."""
    s = basin(W.WEIR, H0=1.5, inflow=False)
    o = oracle.Oracle(s)
    o.set_outflow(weir_crest=1.0, weir_poleni=0.6)
    e_prev = energy(o)
    for _ in range(300):
        o.step(1)
        e = energy(o)
        assert e <= e_prev * (1.0 + 1e-12)
        e_prev = e
    assert o.H.max() <= 1.5 + 1e-12
    assert o.boundary_volume < 0.0


def _strip(h0, mu, nx=6, dx=2.0, dy=10.0, cfl_mode=0):
    """One row of nx quads dx x dy (dy >> dx, so the outlet edge -- a long leg -- has
    the smallest rho / lambda once the outlet speeds up the water), flat bed, water at
    rest of depth h0, walls except the weir at x = nx dx (crest far below the bed)."""
    xy, tri, tag = W.rect_mesh(nx, 1, nx * dx, dy, jitter=0.0, side_tags=(W.WALL, W.WEIR, W.WALL, W.WALL))
    N = len(tri)
    s = W.Scenario("strip", xy, tri, np.zeros(N), np.zeros(N), tag, np.full(N, h0), np.zeros(N), np.zeros(N),
                   W.default_params(cfl=0.9, cfl_mode=cfl_mode))
    o = oracle.Oracle(s)
    o.set_outflow(weir_crest=-10.0, weir_poleni=mu)
    return s, o


def test_outlet_taking_more_than_the_water_brings_passes_ritter_discharge():
    """Poleni with mu = 50 asks for far more than still water can deliver; the outlet
    passes the critical discharge of the characteristic, which for water at rest is
    Ritter's dam-site flow: h = 4 h0 / 9, u = c = (2/3) sqrt(g h0), q = (8/27) sqrt(g)
    h0^(3/2).  Its wave speed u + c = (4/3) sqrt(g h0) decides Eq. 21 on the outlet
    edge: dt = CFL rho / ((4/3) c0), rho = 4 |Omega| / (3 l); the first step lets
    exactly q l dt out."""
    h0 = 2.0
    s, o = _strip(h0, mu=50.0)
    c0 = math.sqrt(G * h0)
    area, l_out = 0.5 * 2.0 * 10.0, 10.0
    rho = 4.0 * area / (3.0 * l_out)
    want_dt = 0.9 * rho / (4.0 / 3.0 * c0)
    # every other edge of the strip allows more: its rho over c0
    L, R, nx, ny, lens = o.edges()
    assert 0.9 * (4.0 * area / (3.0 * lens.max())) / c0 > want_dt
    dt = o.next_dt()
    assert abs(dt - want_dt) <= 1e-14 * want_dt
    q = 8.0 / 27.0 * math.sqrt(G) * h0 ** 1.5
    v0 = o.volume()
    o.step(1)
    assert abs((v0 - o.volume()) - q * l_out * dt) <= 1e-12 * q * l_out * dt
    assert abs(o.boundary_volume + q * l_out * dt) <= 1e-12 * q * l_out * dt


def test_subcritical_outlet_wave_speed():
    """Below the cap the boundary state is the subcritical root s = sqrt(h_b) of
    2 sqrt(g) s^3 - w s^2 + q = 0 (w = 2 sqrt(g h0) for water at rest), taken here
    from numpy's polynomial roots: Eq. 21 on the outlet edge uses q / h_b + sqrt(g h_b)."""
    h0, mu = 2.0, 0.25
    s, o = _strip(h0, mu=mu)
    q = (2.0 / 3.0) * mu * math.sqrt(2.0 * G) * h0 ** 1.5  # crest far below: eta = h0
    w = 2.0 * math.sqrt(G * h0)
    assert q < w ** 3 / (27.0 * G)  # below the critical cap
    roots = np.roots([2.0 * math.sqrt(G), -w, 0.0, q])
    sb = max(r.real for r in roots if abs(r.imag) < 1e-12 and r.real > 0)
    hb = sb * sb
    assert q / hb < math.sqrt(G * hb)  # subcritical
    lam = q / hb + math.sqrt(G * hb)
    area, l_out = 10.0, 10.0
    want_dt = 0.9 * (4.0 * area / (3.0 * l_out)) / lam
    L, R, nx, ny, lens = o.edges()
    assert 0.9 * (4.0 * area / (3.0 * lens.max())) / math.sqrt(G * h0) > want_dt  # the outlet decides
    dt = o.next_dt()
    assert abs(dt - want_dt) <= 1e-13 * want_dt


RATING_S = np.array([1.0, 1.5, 2.0, 3.0])
RATING_Q = np.array([0.0, 8.0, 20.0, 50.0])


def test_hq_reservoir_steady_stage_inverts_the_rating():
    """Fed by Q = 10 m^3/s, the basin settles at the stage where the rating curve
    gives 10: S = 1.5 + 0.5 (10 - 8) / 12 = 1.5833 m on every outlet cell."""
    Q = 10.0
    o = oracle.Oracle(basin(W.HQ_OUTFLOW, Q=Q, H0=1.5))
    o.set_outflow(hq_stage=RATING_S, hq_discharge=RATING_Q)
    o.run_until(3600.0)
    cells, _ = outlet_cells(o, -4)
    S = 1.5 + 0.5 * (Q - 8.0) / 12.0
    assert np.abs(o.H[cells] - S).max() < 1e-7
    _, qo = o.boundary_discharge()
    L, R, nx, ny, lens = o.edges()
    assert abs(float(np.sum(qo * lens)) - Q) < 1e-7 * Q


def test_hq_split_keeps_both_halves_at_their_normal_flow():
    """A sloped channel whose deep half lies 0.5 m lower, fed by the sum of the two
    halves' Manning normal discharges, drains through an h-Q outlet whose rating curve
    is that normal-flow discharge as a function of the stage (41 points).  The
    conveyance split then hands each half its own normal discharge and the last cell
    row carries the same unit discharge and depth as the rows 150-250 m upstream, in
    both halves (bar 3 %); a split by depth would move them by ~10 %."""
    nx, ny, L, Wd, S0, n = 80, 8, 400.0, 20.0, 1e-3, 0.03
    h_deep, h_shallow = 1.5, 1.0
    xy, tri, tag = W.rect_mesh(nx, ny, L, Wd, jitter=0.0, side_tags=(W.INFLOW, W.HQ_OUTFLOW, W.WALL, W.WALL))
    c = xy[tri].mean(axis=1)
    N = len(tri)
    deep = c[:, 1] < Wd / 2
    z = S0 * (L - c[:, 0]) - np.where(deep, h_deep - h_shallow, 0.0)
    h = np.where(deep, h_deep, h_shallow)
    qn = h ** (5.0 / 3.0) * math.sqrt(S0) / n
    Q = (h_deep ** (5.0 / 3.0) + h_shallow ** (5.0 / 3.0)) * math.sqrt(S0) / n * Wd / 2
    s = W.Scenario("hq_channel", xy, tri, z, np.full(N, n), tag, z + h, qn, np.zeros(N),
                   W.default_params(cfl_mode=1, hydro_t=np.array([0.0, 1e9]), hydro_q=np.array([Q, Q])))
    o = oracle.Oracle(s)
    cells, _ = outlet_cells(o, -4)
    # the outlet cells' beds, per half, as the stage sees them (equal edge lengths)
    zd = z[cells][deep[cells]].mean()
    zs = z[cells][~deep[cells]].mean()
    stage = np.linspace(zs + 0.5, zs + 1.5, 41)
    rate = (np.maximum(stage - zd, 0) ** (5 / 3) + np.maximum(stage - zs, 0) ** (5 / 3)) * math.sqrt(S0) / n * Wd / 2
    o.set_outflow(hq_stage=stage, hq_discharge=rate)
    o.run_until(600.0)
    x = c[:, 0]
    last, far = x > L - 5.0, (x > 150.0) & (x < 250.0)
    hh = o.depth()
    for half in (deep, ~deep):
        q1, qf = o.qx[last & half].mean(), o.qx[far & half].mean()
        h1, hf = hh[last & half].mean(), hh[far & half].mean()
        assert abs(q1 / qf - 1.0) < 0.03, (q1, qf)
        assert abs(h1 / hf - 1.0) < 0.03, (h1, hf)


def test_dry_hq_outlet_lets_nothing_out():
    """No wet cell on the h-Q outlet: no stage, no discharge, the edges are walls."""
    s = basin(W.HQ_OUTFLOW, H0=0.0, inflow=False)
    o = oracle.Oracle(s)
    o.set_outflow(hq_stage=RATING_S, hq_discharge=RATING_Q)
    _, qo = o.boundary_discharge()
    assert not np.any(qo)
    o.step(5)
    assert o.boundary_volume == 0.0


def test_outflow_table_is_validated():
    o = oracle.Oracle(basin(W.HQ_OUTFLOW))
    with pytest.raises(oracle.OracleError):
        o.set_outflow(hq_stage=[1.0, 1.0], hq_discharge=[0.0, 1.0])  # not increasing
    with pytest.raises(oracle.OracleError):
        o.set_outflow(hq_stage=[1.0, 2.0], hq_discharge=[0.0, -1.0])  # negative discharge
    with pytest.raises(oracle.OracleError):
        o.set_outflow(hq_stage=[1.0], hq_discharge=[0.0])  # one point
    with pytest.raises(oracle.OracleError):
        o.set_outflow(weir_crest=1.0, weir_poleni=-0.5)
