"""Pins of the oracle's bed evolution (Section "Morphodynamics": Exner, Eq. 3 with
S_b = 0, the update of Eq. 13 with the HLL sediment flux of Eq. 14-16, the MPM-like
closure of Table 2, synchronous-decoupled with the water), against invariants, the
closed form of one step of uniform flow in a closed box, and the eigenvalues of the
one-dimensional shallow-water-Exner system.

A plausible mistake fails one of them: a missing edge in the update or a one-sided
flux (sediment conservation, boundary balance), a bed change that is not carried by
the free surface (water volume), transport below the threshold (threshold test), a
wrong sign, closure coefficient or exponent, Shields number, porosity factor or
direction (uniform flow in a closed box: what reaches the walls is exactly Table 2's
bedload), a wrong sign, celerity or factor in Eq. 16's speeds or a wrong dq_B/dq
(the speeds must bracket the waves of the coupled system, and their product gives back
the derivative of Table 2's law).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2102_12862_b300 import workloads as W

SAND = dict(porosity=0.4, s=2.65, d=0.001, alpha=8.0, m=1.5, theta_cr=0.047)


def test_closed_basin_conserves_sediment_and_water():
    """Dam break with friction in a closed basin over a rough bed: the bed moves, the
    sediment volume sum |Omega| z and the water volume sum |Omega| (H - z) stay."""
    s = W.random_state(W.dam_break(nx=60, ny=8, seed=4, closed=True, manning=0.03), seed=4, dry_frac=0.1)
    o = oracle.Oracle(s, cfl_mode=1)
    o.set_morpho(**SAND)
    area = o.area()
    z0, v0 = s.z.copy(), o.volume()
    o.step(300)
    dz = o.z - z0
    assert np.max(np.abs(dz)) > 1e-4
    assert abs(area @ dz) <= 1e-12 * (area @ np.abs(dz))
    assert abs(o.volume() - v0) <= 1e-12 * v0
    assert o.bed_outflow == 0.0


def test_below_threshold_nothing_moves():
    """theta_cr above every Shields number: the bed is bitwise unchanged and the water
    is bitwise the run without the module."""
    s = W.dam_break(manning=0.03)
    a, b = oracle.Oracle(s), oracle.Oracle(s)
    a.set_morpho(**dict(SAND, theta_cr=1e9))
    a.step(200)
    b.step(200)
    assert np.array_equal(a.z, s.z)
    assert np.array_equal(a.H, b.H) and np.array_equal(a.qx, b.qx) and np.array_equal(a.qy, b.qy)


def channel(bump: float, nx=200, ny=4, L=200.0, Wd=4.0, S=0.001, n=0.02, q=1.0):
    xy, tri, tag = W.rect_mesh(nx, ny, L, Wd, jitter=0.0, side_tags=(W.INFLOW, W.TRANSMISSIVE, W.WALL, W.WALL))
    c = xy[tri].mean(axis=1)
    N = len(tri)
    z = S * (L - c[:, 0]) + bump * np.exp(-((c[:, 0] - 80.0) / 6.0) ** 2)
    hn = (n * q / math.sqrt(S)) ** 0.6
    H = S * (L - c[:, 0]) + hn
    return W.Scenario("channel", xy, tri, z, np.full(N, n), tag, np.maximum(H, z), np.full(N, q), np.zeros(N),
                      W.default_params(hydro_t=np.array([0.0, 1e9]), hydro_q=np.array([q * Wd, q * Wd]))), hn


def test_open_channel_bed_balance():
    """Inflow fed at capacity, transmissive outlet: the bed volume change (1 - p) sum
    |Omega| dz equals what entered minus what left, to rounding."""
    s, _ = channel(0.05)
    o = oracle.Oracle(s)
    o.set_morpho(**SAND)
    z0 = s.z.copy()
    o.step(2000)
    area = o.area()
    change = (1 - SAND["porosity"]) * (area @ (o.z - z0))
    assert abs(change + o.bed_outflow) <= 1e-10 * max(abs(o.bed_outflow), area @ np.abs(o.z - z0))
    assert np.max(np.abs(o.z - z0)) > 1e-5


def mpm(h, u, n, P, g=9.81):
    """Table 2's MPM-like bedload magnitude for depth h, speed u, Manning n (Manning's
    bed shear stress rho g n^2 u^2 / h^(1/3) as the Shields number's numerator)."""
    theta = n * n * u * u / ((P["s"] - 1.0) * P["d"] * h ** (1.0 / 3.0))
    return P["alpha"] * max(theta - P["theta_cr"], 0.0) ** P["m"] * math.sqrt((P["s"] - 1.0) * g * P["d"] ** 3)


@pytest.mark.parametrize("angle", [0.0, 30.0])
def test_uniform_flow_in_a_closed_box_one_step(angle):
    """Flat bed, uniform depth 0.5 m and velocity 1.2 m/s (at an angle) in a closed box,
    one step: every edge between equal states carries exactly the cell's bedload, the
    walls none, so only the wall cells change -- the cells along the downstream walls
    gain dt q_B,n L_wall / (1 - p) of bed volume in total, the upstream ones lose as
    much, interior cells stay (Eq. 13 with Table 2's closure; q_B evaluated here)."""
    Lx, Ly, nx, ny = 40.0, 20.0, 40, 20
    xy, tri, tag = W.rect_mesh(nx, ny, Lx, Ly, jitter=0.0, side_tags=(W.WALL, W.WALL, W.WALL, W.WALL))
    N = len(tri)
    h0, sp, n = 0.5, 1.2, 0.03
    ux, uy = sp * math.cos(math.radians(angle)), sp * math.sin(math.radians(angle))
    s = W.Scenario("box", xy, tri, np.zeros(N), np.full(N, n), tag, np.full(N, h0), np.full(N, h0 * ux),
                   np.full(N, h0 * uy), W.default_params())
    o, plain = oracle.Oracle(s), oracle.Oracle(s)
    o.set_morpho(**SAND)
    dt = o.next_dt()
    o.step(1)
    plain.step(1)
    # the free surface moves with the bed: the water is the run without the module
    assert np.max(np.abs(o.depth() - plain.depth())) <= 1e-15
    assert np.array_equal(o.qx, plain.qx) and np.array_equal(o.qy, plain.qy)
    area = o.area()
    dz = o.z
    c = s.centroids()
    qb = mpm(h0, sp, n, SAND)
    assert qb > 0
    k = (1 - SAND["porosity"]) / dt
    qx, qy = qb * math.cos(math.radians(angle)), qb * math.sin(math.radians(angle))
    # per cell: each wall edge keeps back what would have left through it, l q_B . n
    L, R, enx, eny, ln = o.edges()
    expected = np.zeros(N)
    wall = R == -1
    np.add.at(expected, L[wall], ln[wall] * (qx * enx[wall] + qy * eny[wall]))
    got = k * area * dz
    assert np.max(np.abs(got - expected)) <= 1e-12 * qb * Lx / nx
    # interior cells stay; the east (and north) walls gain the bedload times their length
    assert np.max(np.abs(dz[expected == 0.0])) <= 1e-15
    east = c[:, 0] > Lx - 1.0
    assert abs(got[east].sum() - qx * Ly) <= 1e-12 * qb * Ly  # corner terms cancel


def _bedload_mpm(h, q, man, s_rel, d, alpha, m, theta_cr, g=9.81):
    """Table 2's MPM-like bedload |q_B| of a 1D flow of depth h and unit discharge q:
    Shields number theta = tau_b / ((rho_s - rho) g d) with Manning's bed shear stress
    tau_b = rho g n^2 u^2 / h^(1/3) (Eq. 2), u = q / h; |q_B| = alpha (theta -
    theta_cr)^m sqrt((s - 1) g d^3) above the threshold, 0 below."""
    u = q / h
    rho = 1000.0
    tau = rho * g * man * man * u * u / h ** (1.0 / 3.0)
    theta = tau / ((s_rel - 1.0) * rho * g * d)
    return alpha * max(theta - theta_cr, 0.0) ** m * math.sqrt((s_rel - 1.0) * g * d ** 3)


@pytest.mark.parametrize("porosity", [0.0, 0.4])
def test_eq16_speeds_bracket_the_waves_of_the_coupled_system(porosity):
    """Eq. 16 estimates the two slowest waves of the shallow-water-Exner system: in 1D,
    with U = (h, q, z), dU/dt + A dU/dx = 0 and
        A = [[0, 1, 0], [g h - u^2, 2 u, g h], [xi dq_B/dh, xi dq_B/dq, 0]],
    xi = 1 / (1 - p), whose eigenvalues are r1 < r2 < r3 (r1 ~ u - c, the bed wave r2,
    r3 ~ u + c in subcritical flow).  For an HLL flux the speeds must bound the waves
    they stand for: lambda_1 <= r1 and r2 <= lambda_2 <= r3.  The Jacobian is built here
    from Table 2's law with numerical derivatives (nothing from the oracle but the
    speeds), for random subcritical states above the threshold.  Also: the product
    lambda_1 lambda_2 = -(dq_B/dq) c^2, so the oracle's derivative, at fixed depth
    along the flow (Eq. 16's dq_B,n/dq_n), is read back and must equal the numerical
    derivative of the law.  The bracket is checked at porosity 0: Eq. 16 as printed has
    no 1 / (1 - p) (Eq. 3 has it), and with p = 0.4 strongly coupled states give
    lambda_1 above r1 (e.g. -1.043 against -1.073 m/s with a bed wave of 0.54 m/s); the
    derivative pin holds at every porosity."""
    g = 9.81
    rng = np.random.default_rng(16)
    s = W.dam_break(nx=6, ny=2, jitter=0.0)
    n_checked = 0
    for _ in range(400):
        h = rng.uniform(0.2, 3.0)
        fr = rng.uniform(0.15, 0.9)
        man = rng.uniform(0.02, 0.06)
        d = rng.uniform(5e-4, 5e-3)
        alpha, m, thcr, s_rel = rng.uniform(4.0, 12.0), rng.uniform(1.2, 2.0), rng.uniform(0.03, 0.06), 2.65
        c = math.sqrt(g * h)
        u = fr * c
        q = u * h
        if not _bedload_mpm(h, q, man, s_rel, d, alpha, m, thcr) > 0.0:
            continue
        sc = s.copy()
        sc.manning = np.full(s.n_cells, man)
        sc.H = sc.z + h
        sc.qx = np.full(s.n_cells, q)
        sc.qy = np.zeros(s.n_cells)
        o = oracle.Oracle(sc)
        o.set_morpho(porosity=porosity, s=s_rel, d=d, alpha=alpha, m=m, theta_cr=thcr)
        l1, l2 = o.morpho_speeds(3, 1.0, 0.0)
        eh, eq = 1e-6 * h, 1e-6 * q
        dqb_dh = (_bedload_mpm(h + eh, q, man, s_rel, d, alpha, m, thcr)
                  - _bedload_mpm(h - eh, q, man, s_rel, d, alpha, m, thcr)) / (2 * eh)
        dqb_dq = (_bedload_mpm(h, q + eq, man, s_rel, d, alpha, m, thcr)
                  - _bedload_mpm(h, q - eq, man, s_rel, d, alpha, m, thcr)) / (2 * eq)
        xi = 1.0 / (1.0 - porosity)
        A = np.array([[0.0, 1.0, 0.0], [g * h - u * u, 2 * u, g * h], [xi * dqb_dh, xi * dqb_dq, 0.0]])
        r = np.sort(np.linalg.eigvals(A).real)
        tol = 1e-9 * c
        if porosity == 0.0:
            assert l1 <= r[0] + tol, (l1, r)
            assert r[1] - tol <= l2 <= r[2] + tol, (l2, r)
        assert abs(-l1 * l2 / (c * c) - dqb_dq) <= 1e-5 * dqb_dq, (-l1 * l2 / (c * c), dqb_dq)
        n_checked += 1
    assert n_checked > 200
