"""Pins of the oracle's water-level boundary (the zhydrograph of the paper's standard
inflow and outflow lists, whose input is the water surface elevation) against what the
physics fixes.

Reading under test: the flux through a level edge is the HLLC flux between the inside
cell and a boundary state of depth h_b = max(0, Z_b(t) - z_i) (the imposed surface
over the cell's bed), normal velocity u_b = u_n + 2 sqrt(g h) - 2 sqrt(g h_b) (the
outgoing Riemann invariant carried from the cell; 0 next to a dry cell) and the cell's
tangential velocity; Eq. 21 adds the boundary state's |u_b| + sqrt(g h_b).

- Still water at the imposed level is the boundary state itself: it stays at rest,
  bitwise, on rough beds with dry cells.
- A level dropped at the outlet of a channel at rest drives a 1-rarefaction into it;
  for h_b >= 4/9 h0 the outlet state is (h_b, 2 (sqrt(g h0) - sqrt(g h_b))), so the
  discharge leaving is fixed until the wave returns (closed form).
- A basin opened to a higher level fills to it, mass balanced to round-off.
- Opened to its own level with a hump, the basin's available energy
  sum |Omega| (|q|^2 / (2 h) + g (H - Z_b)^2 / 2) decays (the positivity time step).
- A level raised at the inlet of a channel at rest drives a 2-shock into it, with the
  discharge and speed Rankine-Hugoniot fixes.
- A dry channel fed by a level stays positive and mass balanced.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2102_12862_b300 import workloads as W

G = 9.81


def channel(nx, ny, L, Wd, H0, z=0.0, n=0.0, level_side=1, cfl_mode=1, jitter=0.0, seed=0):
    """A flat rectangle with the level edges on the x = 0 (level_side 0) or x = L side
    (1), walls elsewhere."""
    tags = [W.WALL, W.WALL, W.WALL, W.WALL]
    tags[level_side] = W.WATER_LEVEL
    xy, tri, tag = W.rect_mesh(nx, ny, L, Wd, jitter=jitter, seed=seed, side_tags=tuple(tags))
    N = len(tri)
    zz = np.broadcast_to(np.asarray(z, dtype=np.float64), (N,)).copy()
    H = np.maximum(np.broadcast_to(np.asarray(H0, dtype=np.float64), (N,)), zz)
    return W.Scenario("level_channel", xy, tri, zz, np.full(N, n), tag, H, np.zeros(N), np.zeros(N),
                      W.default_params(cfl_mode=cfl_mode))


def available_energy(o, zb):
    a, h = o.area(), o.depth()
    wet = h > 1e-6
    ke = np.zeros_like(h)
    ke[wet] = 0.5 * (o.qx[wet] ** 2 + o.qy[wet] ** 2) / h[wet]
    return float(np.sum(a * (ke + 0.5 * G * (o.H - zb) ** 2)))


@pytest.mark.parametrize("cfl_mode", [0, 1])
def test_rest_at_the_imposed_level_is_bitwise(cfl_mode):
    """The fractal lake (rough bed, dry islands above the level) with one side at the
    lake's own level: 800 steps leave every value unchanged."""
    s = W.fractal_lake(nx=40, ny=20, Lx=400.0, Ly=200.0, seed=11)
    xy, tri, tag = W.rect_mesh(40, 20, 400.0, 200.0, jitter=0.1, seed=11,
                               side_tags=(W.WALL, W.WATER_LEVEL, W.WALL, W.WALL))
    s.edge_tag = tag
    s.params = W.default_params(cfl_mode=cfl_mode)
    o = oracle.Oracle(s)
    o.set_level([0.0], [403.0])
    H0 = o.H.copy()
    o.step(800)
    assert np.array_equal(o.H, H0)
    assert not o.qx.any() and not o.qy.any()
    assert o.time > 0


def test_level_drop_passes_the_rarefaction_discharge():
    """h0 = 1 m at rest, the outlet level dropped to 0.6 m: the 1-rarefaction's outlet
    state carries q = h_b 2 (sqrt(g h0) - sqrt(g h_b)) (subcritical: h_b > 4/9 h0) until
    its head, moving upstream at sqrt(g h0), has come back from the far wall."""
    h0, hb, L, Wd = 1.0, 0.6, 600.0, 10.0
    s = channel(240, 2, L, Wd, h0, level_side=1, cfl_mode=1)
    o = oracle.Oracle(s)
    o.set_level([0.0], [hb])
    q_exact = hb * 2.0 * (math.sqrt(G * h0) - math.sqrt(G * hb))
    # from the first seconds on (the outlet cells reach the outlet state within a few
    # steps) until the head, reaching x = 0 at L / sqrt(g h0) = 191 s, comes back
    for T in (10.0, 100.0):
        o.run_until(T)
        out = -o.boundary_volume  # volume that left
        assert out == pytest.approx(q_exact * Wd * T, rel=0.01), (T, out, q_exact * Wd * T)
    # the outlet cells hold the outlet state (first-order smearing over a few cells)
    L_, R_, _, _, _ = o.edges()
    cells = L_[R_ == -6]
    h_out = o.depth()[cells]
    assert np.all(np.abs(h_out - hb) < 0.03 * h0), h_out


def test_basin_fills_to_a_raised_level_mass_balanced():
    """A 200 x 20 m basin at 0.3 m (Manning n = 0.05) opened to a 0.4 m level on one
    side fills to it. The fixed level reflects, so the basin rings as a quarter-wave
    resonator (period 4 L / sqrt(g h), about 400 s) whose swing friction damps: the level
    averaged over two periods is the imposed one, the swing shrinks, and the volume gained
    equals the boundary volume to round-off at every instant."""
    s = channel(40, 4, 200.0, 20.0, 0.3, n=0.05, level_side=0, cfl_mode=1)
    o = oracle.Oracle(s)
    o.set_level([0.0], [0.4])
    a = o.area()
    v0 = o.volume()
    swing, mean = [], []
    for t in range(10, 2410, 10):
        o.run_until(float(t))
        assert o.volume() - v0 == pytest.approx(o.boundary_volume, abs=1e-11 * v0)
        swing.append(np.max(np.abs(o.H - 0.4)))
        mean.append(float(np.sum(a * o.H) / a.sum()))
    assert np.mean(mean[-80:]) == pytest.approx(0.4, abs=5e-4), np.mean(mean[-80:])
    assert max(swing[-80:]) < 0.5 * max(swing[40:120]), (max(swing[-80:]), max(swing[40:120]))
    assert o.boundary_volume == pytest.approx(0.1 * 200.0 * 20.0, rel=0.02)


def test_available_energy_decays():
    """A hump of 0.3 m on a basin at the boundary's level: the available energy never
    rises above its start (bar the kinetic energy water brings in, < 1 %), loses three
    quarters of it in 600 s (friction; the fixed level reflects the waves) and the
    basin settles towards the level."""
    s = channel(40, 4, 200.0, 20.0, 1.0, level_side=1, cfl_mode=1)
    c = s.centroids()
    s.H = s.H + 0.3 * np.exp(-((c[:, 0] - 80.0) / 20.0) ** 2)
    s.manning = np.full(len(s.z), 0.02)
    o = oracle.Oracle(s)
    o.set_level([0.0], [1.0])
    e0 = available_energy(o, 1.0)
    es = []
    for _ in range(60):
        o.run_until(o.time + 10.0)
        es.append(available_energy(o, 1.0))
    assert max(es) <= 1.01 * e0, (max(es), e0)
    assert max(b - a for a, b in zip(es, es[1:])) < 0.01 * e0
    assert es[-1] < 0.25 * e0, (es[-1], e0)
    assert np.max(np.abs(o.H - 1.0)) < 0.05


def test_raised_level_drives_the_rankine_hugoniot_shock():
    """h0 = 1 m at rest, the inlet level raised to 1.2 m: a 2-shock runs into the
    channel. Behind it the state is (h_b, u) with u = (h_b - h0) sqrt(g (h_b + h0) /
    (2 h_b h0)) (Rankine-Hugoniot from the state at rest), so the discharge entering is
    h_b u and the shock sits at S T, S = h_b u / (h_b - h0)."""
    h0, hb, L, Wd = 1.0, 1.2, 600.0, 10.0
    s = channel(240, 2, L, Wd, h0, level_side=0, cfl_mode=1)
    o = oracle.Oracle(s)
    o.set_level([0.0], [hb])
    u = (hb - h0) * math.sqrt(G * (hb + h0) / (2.0 * hb * h0))
    T = 100.0
    o.run_until(T)
    assert o.boundary_volume == pytest.approx(hb * u * Wd * T, rel=0.005)
    L_, R_, _, _, _ = o.edges()
    cells = L_[R_ == -6]
    assert np.all(np.abs(o.depth()[cells] - hb) < 1e-4 * hb)
    assert np.all(np.abs(o.qx[cells] - hb * u) < 1e-3 * hb * u)
    S = hb * u / (hb - h0)
    x = s.centroids()[:, 0]
    front = x[o.H > 0.5 * (h0 + hb)].max()
    assert abs(front - S * T) < 2 * L / 240, (front, S * T)


def test_dry_channel_fed_by_a_level_stays_positive_and_balanced():
    """A dry flat channel with a 0.5 m level at x = 0: water enters (first as a dam
    break into the dry cell), depths stay >= 0 and the volume gained is the boundary
    volume to round-off. The inflow here is supercritical, where a depth condition
    alone does not fix the state (the boundary type follows the flow regime), so only
    conservation and positivity are pinned."""
    h0, L, Wd = 0.5, 400.0, 10.0
    s = channel(160, 2, L, Wd, 0.0, level_side=0, cfl_mode=1)
    o = oracle.Oracle(s)
    o.set_level([0.0], [h0])
    v0 = o.volume()
    for T in (5.0, 20.0, 40.0):
        o.run_until(T)
        assert o.depth().min() >= 0.0
        assert o.volume() - v0 == pytest.approx(o.boundary_volume, abs=1e-12 * o.boundary_volume)
    assert o.boundary_volume > 0.5 * 8.0 / 27.0 * math.sqrt(G) * h0 ** 1.5 * Wd * 40.0  # half Ritter's


def test_level_series_and_wall_until_set():
    """Until a series is set the level edges are walls (a lake above any level stays
    put); a series that holds the lake's level until t = 50 s and then rises lets
    nothing in before and water in after."""
    s = channel(30, 3, 150.0, 15.0, 1.0, level_side=1, cfl_mode=1)
    o = oracle.Oracle(s)
    H0 = o.H.copy()
    o.step(50)
    assert np.array_equal(o.H, H0)  # a wall: at rest
    o2 = oracle.Oracle(s)
    o2.set_level([0.0, 50.0, 80.0], [1.0, 1.0, 1.3])
    o2.run_until(50.0)
    assert np.array_equal(o2.H, H0) and o2.boundary_volume == 0.0
    o2.run_until(200.0)
    assert o2.boundary_volume > 0.1 * 0.3 * 150.0 * 15.0
