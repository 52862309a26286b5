"""Pins of the oracle's external sources and sinks (Section "External inflow/outflow
discharge": S_h over regions, as a total discharge or a rain intensity, with the
Exact / Available / Infinity sink behaviours; added explicitly to continuity, the S
term of Eq. 12), against closed forms and invariants.

A plausible mistake fails one of them: a wrong unit conversion or sign (rain on a
lake at rest), the discharge spread over the wrong area (total discharge volume), a
sink that does not stop at the available water or one that does under Exact (sinks),
rain that does not drive the flow its mass balance fixes (a rained plane settling to
Manning's normal depth for q = i x).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2102_12862_b300 import workloads as W

TOTAL, INTENSITY = 0, 1
EXACT, AVAILABLE, INFINITY = 0, 1, 2


def const(v):
    return (np.array([0.0]), np.array([float(v)]))


def test_rain_on_lake_at_rest():
    """36 mm/h (1e-5 m/s) on a fully wet lake over fractal relief: the surface rises by
    i t everywhere, the water stays at rest bitwise, the added volume is i t A."""
    s = W.fractal_lake(nx=40, ny=20, Lx=400.0, Ly=200.0, seed=11, relief=5.0, level=406.0)
    o = oracle.Oracle(s)
    o.set_sources(np.zeros(o.n_cells), [INTENSITY], [EXACT], [const(36.0)])
    v0 = o.volume()
    o.run_until(200.0)
    assert np.max(np.abs(o.H - (406.0 + 1e-5 * 200.0))) <= 1e-11
    assert not o.qx.any() and not o.qy.any()
    a = o.area().sum()
    # the added volume is booked as |Omega| (H after - H before): each step rounds it at
    # the surface's ulp (~6e-14 m at 406 m) against dt i ~ 1e-5 m
    assert abs(o.source_volume - 1e-5 * 200.0 * a) <= 1e-7 * 1e-5 * 200.0 * a
    assert abs(o.volume() - v0 - o.source_volume) <= 1e-11 * v0


def test_rain_dilutes_species_on_a_lake_at_rest():
    """Eq. 8 with its source term off: rain brings water and no species.  On a lake at
    rest every cell's depth grows by i t while its species mass h phi stays, so phi(t) =
    phi0 h0 / (h0 + i t) cell by cell (closed form); a sink over part of the lake takes
    water and leaves the species (phi rises there by h0 / (h0 - s t)), and the species
    mass of the whole closed lake is unchanged to rounding."""
    s = W.fractal_lake(nx=40, ny=20, Lx=400.0, Ly=200.0, seed=11, relief=5.0, level=406.0)
    o = oracle.Oracle(s)
    h0 = o.depth().copy()
    assert h0.min() > 0.5
    rng = np.random.default_rng(5)
    phi0 = rng.uniform(0.2, 1.0, o.n_cells)
    o.set_scalars(np.stack([phi0 * h0, 0.5 * h0]))
    o.set_sources(np.zeros(o.n_cells), [INTENSITY], [EXACT], [const(36.0)])
    m0 = (o.area()[None, :] * o.hc).sum(axis=1)
    o.run_until(200.0)
    phi = o.concentration()
    assert np.max(np.abs(phi[0] - phi0 * h0 / (h0 + 1e-5 * 200.0))) <= 1e-12
    assert np.max(np.abs(phi[1] - 0.5 * h0 / (h0 + 1e-5 * 200.0))) <= 1e-12
    assert np.max(np.abs((o.area()[None, :] * o.hc).sum(axis=1) - m0) / m0) <= 1e-13
    # a sink of 36 mm/h on the cells with x < 200 m: the rest of the lake stays at rest,
    # so with the rain off their depth falls by s t and their phi rises accordingly
    o2 = oracle.Oracle(s)
    o2.set_scalars(np.stack([phi0 * h0]))
    x = s.centroids()[:, 0]
    region = np.where(x < 200.0, 0, -1)
    o2.set_sources(region, [INTENSITY], [EXACT], [const(-36.0)])
    o2.step(1)
    hs = o2.depth()
    # one step: the sink's cells lost dt s of water and none of their species
    sink = region == 0
    assert np.max(np.abs(o2.hc[0][sink] - (phi0 * h0)[sink])) <= 1e-12 * np.max(phi0 * h0)
    assert np.all(hs[sink] < h0[sink])


def test_total_discharge_volume():
    """A total discharge Q over a disk in a closed basin: the volume grows by Q t
    (constant Q) whatever the disk's cells; a linear ramp adds the step sum of Q(t^n),
    within first order of the integral."""
    s = W.dam_break(nx=60, ny=12, Lx=60.0, Ly=12.0, x_dam=30.0, closed=True, manning=0.02, seed=3)
    reg = W.disk_region(s, 45.0, 6.0, 3.0)
    assert (reg == 0).sum() > 10
    o = oracle.Oracle(s)
    o.set_sources(reg, [TOTAL], [EXACT], [const(3.0)])
    v0 = o.volume()
    o.run_until(20.0)
    assert abs(o.source_volume - 60.0) <= 1e-12 * 60.0
    assert abs(o.volume() - v0 - 60.0) <= 1e-11 * v0
    o2 = oracle.Oracle(s)
    o2.set_sources(reg, [TOTAL], [EXACT], [(np.array([0.0, 20.0]), np.array([0.0, 6.0]))])
    v0 = o2.volume()
    o2.run_until(20.0)
    assert abs(o2.volume() - v0 - o2.source_volume) <= 1e-11 * v0
    assert abs(o2.source_volume - 60.0) <= 0.01 * 60.0


def test_sinks():
    """Sinks on a disk in the shallow part (0.1 m) of a closed dam break: Available stops
    at the water the cells hold (no negative depth, removed volume below the
    prescription), Infinity empties the region every step, Exact takes the
    prescription even past the available water (the depth goes negative: the run
    fails), and a weak Exact sink removes exactly |Q| t."""
    s = W.dam_break(nx=60, ny=12, Lx=60.0, Ly=12.0, x_dam=30.0, closed=True, manning=0.02, seed=3)
    reg = W.disk_region(s, 45.0, 6.0, 3.0)
    inside = reg == 0
    strong = const(-1e6)  # mm/h: 0.28 m/s, the 0.1 m layer in ~0.4 s (the bore arrives after ~4 s)
    o = oracle.Oracle(s)
    o.set_sources(reg, [INTENSITY], [AVAILABLE], [strong])
    v0 = o.volume()
    a_reg = o.area()[inside].sum()
    emptied = False
    for _ in range(40):
        o.step(5)
        assert o.depth().min() >= 0.0
        emptied = emptied or bool(np.any(o.depth()[inside] == 0.0))
    assert emptied
    assert -o.source_volume < 1e6 / 3.6e6 * o.time * a_reg
    assert abs(o.volume() - v0 - o.source_volume) <= 1e-11 * v0
    oi = oracle.Oracle(s)
    oi.set_sources(reg, [INTENSITY], [INFINITY], [const(0.0)])
    for _ in range(10):
        oi.step(1)
        assert np.all(oi.depth()[inside] == 0.0)
    assert oi.source_volume < 0
    oe = oracle.Oracle(s)
    oe.set_sources(reg, [INTENSITY], [EXACT], [strong])
    oe.step(200)
    assert oe.depth()[inside].min() < -1e-3
    ow = oracle.Oracle(s)
    ow.set_sources(reg, [TOTAL], [EXACT], [const(-0.05)])
    v0 = ow.volume()
    ow.run_until(10.0)
    assert abs(ow.source_volume + 0.5) <= 1e-12 * 0.5
    assert abs(ow.volume() - v0 + 0.5) <= 1e-11 * v0


@pytest.mark.slow
def test_rain_on_a_plane_reaches_normal_depth():
    """Rain i = 100 mm/h on a dry plane (slope 0.1 %, Manning n = 0.03, 200 m x 10 m,
    outlet at the foot): the sheet the rain has gathered at x carries q = i x, and
    where the flow has settled (kinematic equilibrium at x = 100 m after ~1,000 s;
    upslope of the outlet, whose zero-gradient edge holds water back later) its depth
    is Manning's normal depth h(x) = (n i x / S^(1/2))^(3/5) -- a 10 % error in i
    shows as 6 %.  The discrete balance holds exactly: storage change = rain -
    outflow, and the rain booked is i A t."""
    s = W.rained_plane(slope=0.001)
    i = 100.0 / 3.6e6
    area = 200.0 * 10.0
    o = oracle.Oracle(s)
    o.set_sources(np.zeros(o.n_cells), [INTENSITY], [EXACT], [const(100.0)])
    o.run_until(1000.0)
    v1, b1, s1 = o.volume(), o.boundary_volume, o.source_volume
    o.run_until(1500.0)
    assert abs((o.volume() - v1) - (o.source_volume - s1) - (o.boundary_volume - b1)) <= 1e-12 * v1
    assert abs(o.source_volume - i * area * 1500.0) <= 1e-9 * i * area * 1500.0
    x = s.centroids()[:, 0]
    mid = (x > 30.0) & (x < 100.0)
    h_exact = (0.03 * i * x[mid] / math.sqrt(0.001)) ** 0.6
    assert np.mean(np.abs(o.depth()[mid] / h_exact - 1.0)) < 0.03
