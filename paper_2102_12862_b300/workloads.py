"""Seeded synthetic inputs: meshes, beds, roughness, boundary tags, initial states.

This module holds no arithmetic of the numerical method: it only builds inputs
(node coordinates, triangles, per-cell bed and Manning n, boundary tags, initial
H, q) and is the one module shared by the CUDA path's tests/benchmarks and the
oracle's tests.  Every generator is deterministic in its seed
(``numpy.random.default_rng``).

Workloads follow the paper's test shapes: a wet/dry dam break in a channel, a
floodplain fed by a discharge hydrograph (standing in for the Malpasset-type
field case of Section "T1", whose terrain data are not available), a lake at
rest on rough terrain, the two-rarefaction channel of Section "T5" and the
three-humps basin of Section "T6" (Eq. 23, Eq. 24).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

WALL, TRANSMISSIVE, INFLOW, HQ_OUTFLOW, WEIR, WATER_LEVEL = 0, 1, 2, 3, 4, 5


@dataclass
class Scenario:
    name: str
    xy: np.ndarray          # (n_nodes, 2) float64
    tri: np.ndarray         # (n_tri, 3) int32, counter-clockwise
    z: np.ndarray           # (n_tri,) float64 bed elevation per cell
    manning: np.ndarray     # (n_tri,) float64 Manning n per cell
    edge_tag: np.ndarray    # (n_tri, 3) uint8; edge k = (tri[k], tri[(k+1)%3]); used on boundary edges
    H: np.ndarray           # (n_tri,) float64 free-surface elevation
    qx: np.ndarray
    qy: np.ndarray
    params: dict = field(default_factory=dict)

    @property
    def n_cells(self) -> int:
        return int(self.tri.shape[0])

    def centroids(self) -> np.ndarray:
        return self.xy[self.tri].mean(axis=1)

    def copy(self) -> "Scenario":
        return Scenario(self.name, self.xy.copy(), self.tri.copy(), self.z.copy(), self.manning.copy(),
                        self.edge_tag.copy(), self.H.copy(), self.qx.copy(), self.qy.copy(), dict(self.params))


def default_params(**kw) -> dict:
    p = dict(cfl=0.9, g=9.81, h_min=1e-6, dt_max=1.0, cfl_mode=0,
             hydro_t=np.zeros(0), hydro_q=np.zeros(0))
    p.update(kw)
    return p


def rect_mesh(nx: int, ny: int, Lx: float, Ly: float, x0: float = 0.0, y0: float = 0.0,
              jitter: float = 0.1, seed: int = 0, side_tags=(TRANSMISSIVE, TRANSMISSIVE, WALL, WALL),
              alternate: bool = True):
    """Structured nx x ny quads on [x0, x0+Lx] x [y0, y0+Ly], each split in two triangles.

    Interior nodes are jittered by a seeded uniform +-jitter of the spacing along
    each axis.  The diagonal alternates per quad when ``alternate``.  side_tags
    gives the boundary tag of the (x-min, x-max, y-min, y-max) sides.
    Returns xy (n_nodes, 2), tri (2 nx ny, 3) int32 CCW, edge_tag (2 nx ny, 3) uint8.
    """
    rng = np.random.default_rng(seed)
    dx, dy = Lx / nx, Ly / ny
    I, J = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), indexing="ij")
    X = x0 + I * dx
    Y = y0 + J * dy
    if jitter > 0:
        interior = (I > 0) & (I < nx) & (J > 0) & (J < ny)
        jx = rng.uniform(-jitter, jitter, size=X.shape) * dx
        jy = rng.uniform(-jitter, jitter, size=Y.shape) * dy
        X = np.where(interior, X + jx, X)
        Y = np.where(interior, Y + jy, Y)
    xy = np.stack([X.ravel(), Y.ravel()], axis=1).astype(np.float64)
    nid = lambda i, j: i * (ny + 1) + j  # noqa: E731
    qi, qj = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
    qi, qj = qi.ravel(), qj.ravel()
    n00, n10, n01, n11 = nid(qi, qj), nid(qi + 1, qj), nid(qi, qj + 1), nid(qi + 1, qj + 1)
    diagA = ((qi + qj) % 2 == 0) if alternate else np.ones_like(qi, dtype=bool)
    # diagonal n00-n11: (n00,n10,n11), (n00,n11,n01); diagonal n10-n01: (n00,n10,n01), (n10,n11,n01)
    t1 = np.where(diagA[:, None], np.stack([n00, n10, n11], 1), np.stack([n00, n10, n01], 1))
    t2 = np.where(diagA[:, None], np.stack([n00, n11, n01], 1), np.stack([n10, n11, n01], 1))
    tri = np.empty((2 * len(qi), 3), dtype=np.int64)
    tri[0::2] = t1
    tri[1::2] = t2
    tri = tri.astype(np.int32)
    # boundary tags: an edge lies on a side if both its nodes do
    ni, nj = tri // (ny + 1), tri % (ny + 1)
    tag = np.zeros(tri.shape, dtype=np.uint8)
    for k in range(3):
        a, b = k, (k + 1) % 3
        ia, ib, ja, jb = ni[:, a], ni[:, b], nj[:, a], nj[:, b]
        tag[:, k] = np.where((ia == 0) & (ib == 0), side_tags[0], tag[:, k])
        tag[:, k] = np.where((ia == nx) & (ib == nx), side_tags[1], tag[:, k])
        tag[:, k] = np.where((ja == 0) & (jb == 0), side_tags[2], tag[:, k])
        tag[:, k] = np.where((ja == ny) & (jb == ny), side_tags[3], tag[:, k])
    return xy, tri, tag


def _centroids(xy, tri):
    return xy[tri].mean(axis=1)


# ----------------------------------------------------------------------------------------------
# dam breaks (channel 100 m x 10 m)
# ----------------------------------------------------------------------------------------------

def dam_break(nx: int = 200, ny: int = 10, h_left: float = 1.0, h_right: float = 0.1, seed: int = 1,
              jitter: float = 0.1, Lx: float = 100.0, Ly: float = 10.0, x_dam: float = 50.0,
              closed: bool = False, manning: float = 0.0) -> Scenario:
    """Wet (h_right > 0) or dry (h_right = 0) dam break on a flat frictionless bed.

    Reflective side walls; transmissive ends unless ``closed``.  Default: 200 x 10
    quads = 4,000 triangles, seed 1.
    """
    tags = (WALL, WALL, WALL, WALL) if closed else (TRANSMISSIVE, TRANSMISSIVE, WALL, WALL)
    xy, tri, tag = rect_mesh(nx, ny, Lx, Ly, jitter=jitter, seed=seed, side_tags=tags)
    c = _centroids(xy, tri)
    n = len(tri)
    z = np.zeros(n)
    H = np.where(c[:, 0] < x_dam, h_left, h_right).astype(np.float64)
    return Scenario("dam_break", xy, tri, z, np.full(n, float(manning)), tag, H, np.zeros(n), np.zeros(n),
                    default_params())


def two_rarefaction(ncells_x: int = 681, seed: int = 0, jitter: float = 0.0) -> Scenario:
    """Section "T5" (Eq. 22): 100 m x 0.1 m channel, h = 1, q_x = -3 left / +3 right
    of x = 50 m; 681 x 1 quads = 1,362 cells; walls at the sides, transmissive ends;
    CFL 0.95."""
    xy, tri, tag = rect_mesh(ncells_x, 1, 100.0, 0.1, jitter=jitter, seed=seed,
                             side_tags=(TRANSMISSIVE, TRANSMISSIVE, WALL, WALL))
    c = _centroids(xy, tri)
    n = len(tri)
    qx = np.where(c[:, 0] < 50.0, -3.0, 3.0)
    return Scenario("two_rarefaction", xy, tri, np.zeros(n), np.zeros(n), tag, np.ones(n), qx, np.zeros(n),
                    default_params(cfl=0.95))


def three_humps(nx: int = 150, ny: int = 60, seed: int = 0, jitter: float = 0.1) -> Scenario:
    """Section "T6": basin [0,75] x [-15,15] m, bed of Eq. 23, initial state of Eq. 24
    (h = 1 m for x < 16 m; free surface 0.125 m elsewhere), Manning n = 0.01, walls,
    CFL 0.95."""
    xy, tri, tag = rect_mesh(nx, ny, 75.0, 30.0, y0=-15.0, jitter=jitter, seed=seed,
                             side_tags=(WALL, WALL, WALL, WALL))
    c = _centroids(xy, tri)
    x, y = c[:, 0], c[:, 1]
    e1 = 1.0 - np.sqrt((x - 30.0) ** 2 + (y + 9.0) ** 2) / 8.0
    e2 = 1.0 - np.sqrt((x - 30.0) ** 2 + (y - 9.0) ** 2) / 8.0
    e3 = 3.0 - 3.0 * np.sqrt((x - 47.5) ** 2 + y ** 2) / 10.0
    z = np.maximum.reduce([np.zeros_like(x), e1, e2, e3])
    H = np.where(x < 16.0, z + 1.0, np.maximum(0.125, z))
    n = len(tri)
    return Scenario("three_humps", xy, tri, z, np.full(n, 0.01), tag, H, np.zeros(n), np.zeros(n),
                    default_params(cfl=0.95))


# ----------------------------------------------------------------------------------------------
# terrains
# ----------------------------------------------------------------------------------------------

def rained_plane(nx: int = 100, ny: int = 5, L: float = 200.0, Wd: float = 10.0, slope: float = 0.01,
                 manning: float = 0.03, seed: int = 0, jitter: float = 0.1) -> Scenario:
    """Tilted plane (the overland-flow setting of the "External inflow/outflow
    discharge" source): bed z = slope (L - x), initially dry, walls at x = 0 and at the
    sides, a transmissive outlet at x = L.  The rain is set separately (a source region
    covering every cell)."""
    xy, tri, tag = rect_mesh(nx, ny, L, Wd, jitter=jitter, seed=seed, side_tags=(WALL, TRANSMISSIVE, WALL, WALL))
    c = _centroids(xy, tri)
    z = slope * (L - c[:, 0])
    n = len(tri)
    # the positivity bound on dt: Eq. 21 as printed lets the thin sheet's depths fall
    # below zero here (as on the floodplain)
    return Scenario("rained_plane", xy, tri, z, np.full(n, manning), tag, z.copy(), np.zeros(n), np.zeros(n),
                    default_params(cfl_mode=1))


def disk_region(s: Scenario, x0: float, y0: float, r: float) -> np.ndarray:
    """Source region 0 on the cells whose centroid lies within r of (x0, y0), -1
    elsewhere."""
    c = _centroids(s.xy, s.tri)
    return np.where(np.hypot(c[:, 0] - x0, c[:, 1] - y0) <= r, 0, -1).astype(np.int32)


def _sinusoid_bed(rng, x, y, n_waves=8, amp=(0.5, 3.0), wl=(200.0, 2000.0)):
    A = rng.uniform(*amp, size=n_waves)
    L = rng.uniform(*wl, size=n_waves)
    th = rng.uniform(0, 2 * np.pi, size=n_waves)
    ph = rng.uniform(0, 2 * np.pi, size=n_waves)
    out = np.zeros_like(x)
    for k in range(n_waves):
        out += A[k] * np.sin(2 * np.pi * (x * np.cos(th[k]) + y * np.sin(th[k])) / L[k] + ph[k])
    return out


def _patch_map(rng, x, y, Lx, Ly, n_patches, lo, hi, chunk=1 << 18):
    """Nearest-seed (Voronoi) patches with a uniform value per patch."""
    sx = rng.uniform(0, Lx, n_patches)
    sy = rng.uniform(0, Ly, n_patches)
    val = rng.uniform(lo, hi, n_patches)
    out = np.empty_like(x)
    for s in range(0, len(x), chunk):
        d = (x[s:s + chunk, None] - sx[None, :]) ** 2 + (y[s:s + chunk, None] - sy[None, :]) ** 2
        out[s:s + chunk] = val[np.argmin(d, axis=1)]
    return out


def floodplain(nx: int = 1600, ny: int = 625, Lx: float = 5000.0, Ly: float = 2000.0, seed: int = 2,
               datum: float = 400.0, q_peak: float = 500.0, ramp: float = 600.0,
               n_range=(0.025, 0.06), jitter: float = 0.1, outlet: int = WALL) -> Scenario:
    """Floodplain fed by a discharge hydrograph (default 1600 x 625 quads = 2,000,000
    triangles on 5 km x 2 km, seed 2).

    Bed: datum + 1e-3 downstream slope + 8 seeded sinusoids (amplitude 0.5-3 m,
    wavelength 200-2000 m) + N(0, 0.05^2) per cell.  Manning n: 64 seeded patches,
    uniform in n_range.  A meandering main channel (cells within 40 m of
    y = Ly/2 + 300 sin(2 pi x / 2500 + phi)) is carved 3 m below the local bed and
    holds 2 m of water; everything else starts dry.  Inflow on the whole x = 0
    side, Q ramping 0 -> q_peak over ``ramp`` s then constant; the other sides are
    walls (``outlet`` sets the x = Lx side: a transmissive, zero-gradient outlet lets
    water in wherever the flow next to it turns inward, and on this terrain that
    inflow runs away after about 20 simulated minutes, so the default is a wall and the
    basin fills).  Time step: the positivity bound (cfl_mode 1), because with
    Eq. 21 as printed (cfl_mode 0) the depth goes negative near the inflow on this
    recipe (the oracle reaches -10 m on a 160 x 64 version).
    """
    rng = np.random.default_rng(seed)
    xy, tri, tag = rect_mesh(nx, ny, Lx, Ly, jitter=jitter, seed=seed,
                             side_tags=(INFLOW, outlet, WALL, WALL))
    c = _centroids(xy, tri)
    x, y = c[:, 0], c[:, 1]
    z = datum + 1e-3 * (Lx - x) + _sinusoid_bed(rng, x, y) + rng.normal(0.0, 0.05, size=len(x))
    man = _patch_map(rng, x, y, Lx, Ly, 64, *n_range)
    phi = rng.uniform(0, 2 * np.pi)
    yc = Ly / 2 + 0.15 * Ly * np.sin(2 * np.pi * x / 2500.0 + phi)
    chan = np.abs(y - yc) < 40.0
    z = np.where(chan, z - 3.0, z)
    H = np.where(chan, z + 2.0, z)
    n = len(tri)
    prm = default_params(hydro_t=np.array([0.0, ramp, 1e9]), hydro_q=np.array([0.0, q_peak, q_peak]), cfl_mode=1)
    return Scenario("floodplain", xy, tri, z, man, tag, H, np.zeros(n), np.zeros(n), prm)


def fractal_lake(nx: int = 1000, ny: int = 500, Lx: float = 2000.0, Ly: float = 1000.0, seed: int = 3,
                 datum: float = 400.0, relief: float = 5.0, level: float = 403.0, octaves: int = 8,
                 hurst: float = 0.7, jitter: float = 0.1) -> Scenario:
    """Lake at rest on fractal terrain (default 1000 x 500 quads = 1,000,000 tri).

    z = datum + spectral sum over ``octaves`` octaves (4 random directions each,
    amplitude 2^(-hurst o)), normalised to max|.| = relief; H = max(level, z)
    (cells above the level are dry); q = 0; walls; Manning n = 0.03.
    """
    rng = np.random.default_rng(seed)
    xy, tri, tag = rect_mesh(nx, ny, Lx, Ly, jitter=jitter, seed=seed, side_tags=(WALL, WALL, WALL, WALL))
    c = _centroids(xy, tri)
    x, y = c[:, 0], c[:, 1]
    f = np.zeros_like(x)
    base = 2.0 / max(Lx, Ly)
    for o in range(octaves):
        k = base * 2.0 ** o
        amp = 2.0 ** (-hurst * o)
        for _ in range(4):
            th = rng.uniform(0, 2 * np.pi)
            ph = rng.uniform(0, 2 * np.pi)
            f += amp * np.sin(2 * np.pi * k * (x * np.cos(th) + y * np.sin(th)) + ph)
    f *= relief / np.max(np.abs(f))
    z = datum + f
    H = np.maximum(level, z)
    n = len(tri)
    return Scenario("fractal_lake", xy, tri, z, np.full(n, 0.03), tag, H, np.zeros(n), np.zeros(n),
                    default_params())


def thacker(nq: int = 354, a: float = 3000.0, h0: float = 10.0, A: float = 500.0, half: float = 4000.0,
            datum: float = 0.0, jitter: float = 0.0, seed: int = 4, g: float = 9.81) -> Scenario:
    """Planar sloshing in a paraboloid (Thacker): bed z = datum - h0 (1 - r^2/a^2) on
    [-half, half]^2 (nq x nq quads), initial H = datum + (2 A h0 / a^2) x - h0 A^2/a^2,
    u = 0, v = A omega with omega = sqrt(2 g h0)/a, frictionless, walls.  Time step:
    the positivity bound (cfl_mode 1); Eq. 21 as printed drives the moving shoreline
    to negative depths (-3.9 m on 96 x 96 quads)."""
    xy, tri, tag = rect_mesh(nq, nq, 2 * half, 2 * half, x0=-half, y0=-half, jitter=jitter, seed=seed,
                             side_tags=(WALL, WALL, WALL, WALL))
    c = _centroids(xy, tri)
    x, y = c[:, 0], c[:, 1]
    z = datum - h0 * (1.0 - (x * x + y * y) / (a * a))
    Hs = datum + (2 * A * h0 / (a * a)) * x - h0 * A * A / (a * a)
    H = np.maximum(Hs, z)
    om = np.sqrt(2 * g * h0) / a
    wet = H > z
    n = len(tri)
    qy = np.where(wet, (H - z) * A * om, 0.0)
    return Scenario("thacker", xy, tri, z, np.zeros(n), tag, H, np.zeros(n), qy,
                    default_params(dt_max=10.0, cfl_mode=1))


def thacker_exact(x, y, t, a=3000.0, h0=10.0, A=500.0, datum=0.0, g=9.81):
    """Free surface, depth and velocity of the planar Thacker solution at time t."""
    om = np.sqrt(2 * g * h0) / a
    z = datum - h0 * (1.0 - (x * x + y * y) / (a * a))
    Hs = datum + (2 * A * h0 / (a * a)) * (x * np.cos(om * t) + y * np.sin(om * t)) - h0 * A * A / (a * a)
    h = np.maximum(0.0, Hs - z)
    return h, -A * om * np.sin(om * t), A * om * np.cos(om * t)


def ensemble_instance(k: int, base_seed: int = 5000, n_lo: float = 5e3, n_hi: float = 5e5,
                      size_override: int | None = None) -> Scenario:
    """Instance k of the batched ensemble: a jittered 5 km x 2 km rectangle with
    log-uniform cell count in [n_lo, n_hi], its own sinusoid bed, a main channel,
    uniform Manning n in [0.02, 0.07] and an inflow peak in [50, 1000] m^3/s."""
    rng = np.random.default_rng(base_seed + k)
    N = int(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi)))) if size_override is None else size_override
    ny = max(2, int(round(np.sqrt(N / 5.0))))
    nx = max(2, int(round(N / (2 * ny))))
    n_man = rng.uniform(0.02, 0.07)
    peak = rng.uniform(50.0, 1000.0)
    s = floodplain(nx=nx, ny=ny, seed=base_seed + k, q_peak=peak, n_range=(n_man, n_man))
    s.name = f"ensemble_{k}"
    return s


def random_state(s: Scenario, seed: int, dry_frac: float = 0.2, vel: float = 2.0,
                 depth=(0.01, 2.0), keep_bed: bool = False) -> Scenario:
    """Random valid state on a scenario's mesh: random bed (unless keep_bed), a
    fraction of dry cells (H = z), random depths, velocities and Manning n
    (unless keep_bed) elsewhere.  For short parity checks."""
    rng = np.random.default_rng(seed)
    n = s.n_cells
    out = s.copy()
    zr = rng.uniform(-1.0, 1.0, n)
    if not keep_bed:
        out.z = zr
    h = rng.uniform(*depth, n)
    dry = rng.random(n) < dry_frac
    h[dry] = 0.0
    tiny = (~dry) & (rng.random(n) < 0.05)
    h[tiny] = rng.uniform(0.0, 2e-6, tiny.sum())
    out.H = out.z + h
    out.qx = np.where(h > 0, h * rng.uniform(-vel, vel, n), 0.0)
    out.qy = np.where(h > 0, h * rng.uniform(-vel, vel, n), 0.0)
    mr = rng.uniform(0.0, 0.06, n)
    if not keep_bed:
        out.manning = mr
    return out


def mirror_x(s: Scenario) -> Scenario:
    """Mirror a scenario about x = 0 (node x -> -x, triangles reversed to stay CCW,
    tags follow their edges, q_x -> -q_x)."""
    out = s.copy()
    out.xy[:, 0] = -out.xy[:, 0]
    out.tri = s.tri[:, [0, 2, 1]].copy()
    # edge k of (v0, v2, v1): k=0 (v0,v2) = old edge 2; k=1 (v2,v1) = old 1; k=2 (v1,v0) = old 0
    out.edge_tag = s.edge_tag[:, [2, 1, 0]].copy()
    out.qx = -s.qx
    return out


def rotate_90(s: Scenario) -> Scenario:
    """Rotate a scenario by +90 degrees: (x, y) -> (-y, x), (qx, qy) -> (-qy, qx)."""
    out = s.copy()
    out.xy = np.stack([-s.xy[:, 1], s.xy[:, 0]], axis=1)
    out.qx = -s.qy
    out.qy = s.qx.copy()
    return out
