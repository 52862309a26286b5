"""Pins of the oracle's passive-scalar advection (Section "Scalar advection-diffusion"
with the diffusion and source terms off), against what the paper and the mathematics
fix: the steady contact of Section T5 stays exactly in place, a uniform concentration
stays uniform under any flow, species mass is conserved in a closed domain, the
upwind contact flux keeps concentrations within their initial bounds, and an inflow
front travels at the flow velocity.

A plausible mistake fails one of them: the wrong side of the contact (boundedness,
front speed), the velocity instead of the concentration in the flux (uniform
concentration), a sign or a missing edge in the update (mass), a scalar that does not
follow the water's mass flux (T5, uniform concentration).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2102_12862_b300 import workloads as W


def test_t5_steady_contact_kept_exactly():
    """Section T5: phi = 1 left of x = 50 m, 0 right, under two diverging rarefactions;
    the exact solution keeps phi at its initial values (a steady contact)."""
    s = W.two_rarefaction()
    x = s.centroids()[:, 0]
    phi0 = np.where(x < 50.0, 1.0, 0.0)
    o = oracle.Oracle(s)
    o.set_scalars(phi0 * o.depth())
    o.run_until(2.5)
    wet = o.depth() > 1e-3
    assert wet.mean() > 0.9
    assert np.max(np.abs(o.concentration()[0][wet] - phi0[wet])) <= 1e-12


def test_uniform_concentration_stays_uniform():
    """Two species at 0.7 and 0.2 in a dam break with friction: phi stays uniform
    (the species flux is the water flux times phi)."""
    s = W.dam_break(manning=0.03)
    o = oracle.Oracle(s)
    h = o.depth()
    o.set_scalars(np.stack([0.7 * h, 0.2 * h]))
    o.step(300)
    wet = o.depth() > 1e-3
    phi = o.concentration()
    assert np.max(np.abs(phi[0][wet] - 0.7)) <= 1e-12
    assert np.max(np.abs(phi[1][wet] - 0.2)) <= 1e-12


def test_species_mass_conserved_closed_domain():
    s = W.random_state(W.dam_break(nx=60, ny=8, seed=5, closed=True), seed=5)
    o = oracle.Oracle(s, cfl_mode=1)
    rng = np.random.default_rng(5)
    o.set_scalars(rng.uniform(0, 1, (2, o.n_cells)) * np.maximum(o.depth(), 0))
    area = o.area()
    m0 = o.hc @ area
    o.step(200)
    m1 = o.hc @ area
    assert np.all(np.abs(m1 - m0) <= 1e-12 * np.abs(m0))


@pytest.mark.parametrize("seed", [6, 7])
def test_concentration_stays_within_bounds(seed):
    """Upwind contact fluxes under the CFL limit form a convex combination: phi in
    [0, 1] stays in [0, 1] (wet cells), also with wet/dry fronts and friction."""
    s = W.random_state(W.dam_break(nx=50, ny=6, seed=seed, manning=0.03), seed=seed)
    o = oracle.Oracle(s, cfl_mode=1)
    rng = np.random.default_rng(seed)
    o.set_scalars(rng.uniform(0, 1, (1, o.n_cells)) * np.maximum(o.depth(), 0))
    for _ in range(5):
        o.step(20)
        phi = o.concentration()[0][o.depth() > 1e-6]
        assert phi.min() >= -1e-12 and phi.max() <= 1 + 1e-12


def _uniform_channel(nx):
    L, Wd, S, n, Q = 1000.0, 20.0, 1e-3, 0.03, 20.0
    xy, tri, tag = W.rect_mesh(nx, 4, L, Wd, jitter=0.0, side_tags=(W.INFLOW, W.TRANSMISSIVE, W.WALL, W.WALL))
    c = xy[tri].mean(axis=1)
    N = len(tri)
    z = S * (L - c[:, 0])
    hn = (Q / Wd * n / math.sqrt(S)) ** 0.6
    s = W.Scenario("uniform_flow", xy, tri, z, np.full(N, n), tag, z + hn, np.full(N, Q / Wd), np.zeros(N),
                   W.default_params(hydro_t=np.array([0.0, 1e9]), hydro_q=np.array([Q, Q])))
    return s, c[:, 0], Q / Wd / hn


def test_inflow_front_moves_with_the_flow():
    """Uniform flow (velocity u = q / h_n): a concentration 1 entering clean water at
    x = 0 reaches x = u t; the 0.5 level of the first-order front is there within 1 %."""
    T = 300.0
    errs = []
    for nx in (50, 100, 200):
        s, x, u = _uniform_channel(nx)
        o = oracle.Oracle(s)
        o.set_scalars(np.zeros((1, o.n_cells)), c_in=[1.0])
        o.run_until(T)
        phi = o.concentration()[0]
        order = np.argsort(x)
        xs, ps = x[order], phi[order]
        k = np.argmax(ps < 0.5)
        front = np.interp(0.5, [ps[k], ps[k - 1]], [xs[k], xs[k - 1]])
        errs.append(abs(front - u * T))
        assert np.all(ps[xs < 0.5 * u * T] > 0.99)
        assert np.all(ps[xs > 1.5 * u * T] < 0.01)
    assert max(errs) < 0.01 * u * T


def t6_species(s):
    """Eq. 24's species: phi_1 = 0.5 upstream of the dam (x < 16 m), phi_2 = 0.1
    downstream (the second species' row prints "phi_1" for its downstream value; the
    rest values the paper gives, 0.386 and 0.023, fix the reading)."""
    x = s.centroids()[:, 0]
    h = np.maximum(s.H - s.z, 0.0)
    return np.stack([np.where(x < 16.0, 0.5, 0.0) * h, np.where(x < 16.0, 0.0, 0.1) * h])


@pytest.mark.slow
def test_t6_mixed_concentrations_paper_values():
    """Section T6: two species in the dam break over three humps (closed basin).  The
    paper's rest concentrations, phi_1 = 0.386 and phi_2 = 0.023, are the fully mixed
    values: species mass over water volume, which a conservative scheme keeps at every
    time.  Coarse mesh, 60 s (the bores have crossed the basin and mixed the species):
    the volume-weighted means equal the printed values to their three decimals, species
    mass is conserved, concentrations stay within their initial bounds."""
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))["t6_three_humps"]
    s = W.three_humps(nx=75, ny=30)
    o = oracle.Oracle(s)
    o.set_scalars(t6_species(s))
    area = o.area()
    m0 = o.hc @ area
    o.run_until(60.0)
    v = np.sum(area * o.depth())
    mean = (o.hc @ area) / v
    assert abs(mean[0] - gold["rest_phi1"]) <= 5e-4
    assert abs(mean[1] - gold["rest_phi2"]) <= 5e-4
    assert np.all(np.abs(o.hc @ area - m0) <= 1e-12 * m0)
    phi = o.concentration()[:, o.depth() > 1e-6]
    assert phi.min() >= -1e-12 and phi[0].max() <= 0.5 + 1e-12 and phi[1].max() <= 0.1 + 1e-12
    assert np.sum((phi[0] > 0.01) & (phi[1] > 0.01)) > 100  # the two species met
