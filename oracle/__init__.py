"""FP64 CPU oracle for the explicit shallow-water step (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package.  It wraps ``bm_oracle.c`` (serial, edge loop, built with
``-O2 -ffp-contract=off``) through ctypes and shares no code with the CUDA path.

What the oracle computes follows BASEMENT v3 (arXiv 2102.12862): Eq. 1/Eq. 10
unknowns (H, q_x, q_y), the update of Eq. 12 with an HLLC flux and the
modified-state bed treatment (Section "Numerical solution", "Hydrodynamics"),
Manning friction (Eq. 2, Table 1) split off with a semi-implicit two-stage RK,
and the time step of Eq. 21.

The discharge-inflow split and boundary wave speed are pinned by
tests/test_oracle_inflow.py, the speeds of Eq. 16 by the coupled-system bracket in
tests/test_oracle_morpho.py; the wet/dry threshold logic by Ritter's dry-bed dam
break, the lake at rest with dry islands and wet/dry mass conservation.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bm_oracle.c")
_LIB_SERIAL = os.path.join(_HERE, "liboracle.so")
# A test that plants a mistake in the oracle compiles a mutated copy of the source
# (ORACLE_MUTANT_SRC) into a private library (ORACLE_MUTANT_LIB).
if os.environ.get("ORACLE_MUTANT_SRC"):
    _SRC = os.environ["ORACLE_MUTANT_SRC"]
    _LIB_SERIAL = os.environ["ORACLE_MUTANT_LIB"]
_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")
_lock = threading.Lock()
_libs: dict = {}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2 -ffp-contract=off); returns the .so path."""
    with _lock:
        if force or not os.path.exists(_LIB_SERIAL) or os.path.getmtime(_LIB_SERIAL) < os.path.getmtime(_SRC):
            tmp = _LIB_SERIAL + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                                   "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB_SERIAL)
    return _LIB_SERIAL


class _Params(C.Structure):
    _fields_ = [("cfl", C.c_double), ("g", C.c_double), ("h_min", C.c_double), ("dt_max", C.c_double),
                ("cfl_mode", C.c_int), ("hydro_t", C.POINTER(C.c_double)), ("hydro_q", C.POINTER(C.c_double)),
                ("hydro_n", C.c_int64)]


def _lib():
    if "serial" not in _libs:
        lib = C.CDLL(build())
        P = C.POINTER
        d, i64 = C.c_double, C.c_int64
        lib.orc_create.argtypes = [i64, P(d), i64, P(C.c_int32), P(d), P(d), P(C.c_uint8), P(_Params),
                                   P(C.c_void_p)]
        lib.orc_create.restype = C.c_int
        lib.orc_destroy.argtypes = [C.c_void_p]
        lib.orc_step.argtypes = [C.c_void_p, P(d), P(d), P(d), P(d), d, P(d)]
        lib.orc_step.restype = d
        lib.orc_run.argtypes = [C.c_void_p, P(d), P(d), P(d), P(d), d, i64, P(d)]
        lib.orc_run.restype = i64
        lib.orc_volume.argtypes = [C.c_void_p, P(d)]
        lib.orc_volume.restype = d
        lib.orc_next_dt.argtypes = [C.c_void_p, P(d), P(d), P(d), d]
        lib.orc_next_dt.restype = d
        lib.orc_hllc.argtypes = [d, d, d, d, d, d, d, P(d)]
        lib.orc_wave_speeds.argtypes = [d, d, d, d, d, P(d), P(d)]
        lib.orc_friction.argtypes = [d, d, d, d, d, P(d), P(d)]
        lib.orc_hydrograph.argtypes = [P(_Params), d]
        lib.orc_hydrograph.restype = d
        lib.orc_n_edges.argtypes = [C.c_void_p]
        lib.orc_n_edges.restype = i64
        lib.orc_cell_area.argtypes = [C.c_void_p, P(d)]
        lib.orc_edges.argtypes = [C.c_void_p, P(i64), P(i64), P(d), P(d), P(d)]
        lib.orc_track.argtypes = [C.c_void_p, P(d), P(d), P(d), d, d, d, C.c_int, P(d), P(d), P(d), P(d), P(d)]
        lib.orc_run_tracked.argtypes = [C.c_void_p, P(d), P(d), P(d), P(d), d, i64, P(d), d, d, P(d), P(d), P(d),
                                        P(d), P(d)]
        lib.orc_run_tracked.restype = i64
        lib.orc_run_scalars.argtypes = [C.c_void_p, P(d), P(d), P(d), P(d), d, i64, P(d), C.c_int, P(d), P(d)]
        lib.orc_run_scalars.restype = i64
        i32 = C.c_int32
        lib.orc_set_sources.argtypes = [C.c_void_p, i32, P(i32), P(i32), P(i32), P(i64), P(d), P(d)]
        lib.orc_set_sources.restype = C.c_int
        lib.orc_source_volume.argtypes = [C.c_void_p]
        lib.orc_source_volume.restype = d
        lib.orc_set_morpho.argtypes = [C.c_void_p, C.c_int, d, d, d, d, d, d]
        lib.orc_set_morpho.restype = C.c_int
        lib.orc_bed_outflow.argtypes = [C.c_void_p]
        lib.orc_bed_outflow.restype = d
        lib.orc_bed.argtypes = [C.c_void_p, P(d)]
        lib.orc_set_friction.argtypes = [C.c_void_p, C.c_int, P(d)]
        lib.orc_set_friction.restype = C.c_int
        lib.orc_cf.argtypes = [C.c_int, d, d]
        lib.orc_cf.restype = d
        lib.orc_morpho_speeds.argtypes = [C.c_void_p, P(d), P(d), P(d), i64, d, d, P(d), P(d)]
        lib.orc_morpho_speeds.restype = C.c_int
        lib.orc_set_outflow.argtypes = [C.c_void_p, i64, P(d), P(d), d, d]
        lib.orc_set_outflow.restype = C.c_int
        lib.orc_set_level.argtypes = [C.c_void_p, i64, P(d), P(d)]
        lib.orc_set_level.restype = C.c_int
        lib.orc_boundary_discharge.argtypes = [C.c_void_p, P(d), d, P(d), P(d)]
        lib.orc_boundary_discharge.restype = None
        _libs["serial"] = lib
    return _libs["serial"]


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class OracleError(RuntimeError):
    pass


class Oracle:
    """One mesh + one state, stepped on the CPU in FP64.

    ``scenario`` is any object with the attributes of ``workloads.Scenario``
    (xy, tri, z, manning, edge_tag, H, qx, qy, params).
    """

    def __init__(self, scenario, **overrides):
        lib = _lib()
        s = scenario
        prm = dict(s.params)
        prm.update(overrides)
        self._hydro_t = np.ascontiguousarray(prm.get("hydro_t", np.zeros(0)), dtype=np.float64)
        self._hydro_q = np.ascontiguousarray(prm.get("hydro_q", np.zeros(0)), dtype=np.float64)
        self.params = _Params(prm.get("cfl", 0.9), prm.get("g", 9.81), prm.get("h_min", 1e-6),
                              prm.get("dt_max", 1.0), int(prm.get("cfl_mode", 0)),
                              _dp(self._hydro_t), _dp(self._hydro_q), len(self._hydro_t))
        xy = np.ascontiguousarray(s.xy, dtype=np.float64)
        tri = np.ascontiguousarray(s.tri, dtype=np.int32)
        z = np.ascontiguousarray(s.z, dtype=np.float64)
        man = np.ascontiguousarray(s.manning, dtype=np.float64)
        tag = np.ascontiguousarray(s.edge_tag, dtype=np.uint8)
        h = C.c_void_p()
        rc = lib.orc_create(len(xy), _dp(xy), len(tri), tri.ctypes.data_as(C.POINTER(C.c_int32)), _dp(z), _dp(man),
                            tag.ctypes.data_as(C.POINTER(C.c_uint8)), C.byref(self.params), C.byref(h))
        if rc != 0:
            raise OracleError(f"orc_create failed with code {rc}")
        self._h = h
        self.n_cells = len(tri)
        self.z = z.copy()
        self.H = np.array(s.H, dtype=np.float64, copy=True)
        self.qx = np.array(s.qx if s.qx is not None else np.zeros(self.n_cells), dtype=np.float64, copy=True)
        self.qy = np.array(s.qy if s.qy is not None else np.zeros(self.n_cells), dtype=np.float64, copy=True)
        self.t = C.c_double(0.0)
        self.bvol = C.c_double(0.0)
        self.steps = 0
        self.tracking = None  # flood tracking record (see track())
        self.hc = None  # passive species q_c = h phi_c, K x n (see set_scalars())

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            _lib().orc_destroy(h)
            self._h = None

    def track(self, h_arrival: float, rho: float = 1000.0):
        """Start flood tracking from the current state (updated after every step):
        arrays t_arrival (NaN: not reached), h_max, u_max, q_max, tau_max."""
        n = self.n_cells
        self.tracking = {k: np.empty(n) for k in ("t_arrival", "h_max", "u_max", "q_max", "tau_max")}
        self._track_args = (float(h_arrival), float(rho))
        tr = self.tracking
        _lib().orc_track(self._h, _dp(self.H), _dp(self.qx), _dp(self.qy), self.t.value, float(h_arrival),
                         float(rho), 1, _dp(tr["t_arrival"]), _dp(tr["h_max"]), _dp(tr["u_max"]),
                         _dp(tr["q_max"]), _dp(tr["tau_max"]))

    def set_scalars(self, hc, c_in=None):
        """Advect K passive species with the water: hc (K x n) is q_c = h phi_c; c_in
        the inflow concentrations (K, default 0)."""
        self.hc = np.array(hc, dtype=np.float64, copy=True).reshape(-1, self.n_cells)
        k = self.hc.shape[0]
        self.c_in = np.zeros(k) if c_in is None else np.array(c_in, dtype=np.float64).reshape(k)

    def set_sources(self, region, kind, mode, series):
        """External sources / sinks S_h (see orc_set_sources): region (n,) of each
        cell (-1: none); per region kind (0: total discharge m^3/s, 1: intensity mm/h),
        mode (0: Exact, 1: Available, 2: Infinity) and series (t, v): points of v(t)."""
        reg = np.ascontiguousarray(region, dtype=np.int32).reshape(self.n_cells)
        kind = np.ascontiguousarray(kind, dtype=np.int32).reshape(-1)
        mode = np.ascontiguousarray(mode, dtype=np.int32).reshape(-1)
        nr = len(kind)
        if len(mode) != nr or len(series) != nr:
            raise OracleError("kind, mode and series need one entry per region")
        off = np.zeros(nr + 1, np.int64)
        for r, (t, v) in enumerate(series):
            off[r + 1] = off[r] + len(t)
        tt = np.ascontiguousarray(np.concatenate([np.asarray(t, float) for t, _ in series]) if nr else np.zeros(1))
        vv = np.ascontiguousarray(np.concatenate([np.asarray(v, float) for _, v in series]) if nr else np.zeros(1))
        rc = _lib().orc_set_sources(self._h, nr, reg.ctypes.data_as(C.POINTER(C.c_int32)),
                                    kind.ctypes.data_as(C.POINTER(C.c_int32)),
                                    mode.ctypes.data_as(C.POINTER(C.c_int32)),
                                    off.ctypes.data_as(C.POINTER(C.c_int64)), _dp(tt), _dp(vv))
        if rc != 0:
            raise OracleError(f"orc_set_sources failed with code {rc}")
        self.n_sources = nr

    def set_morpho(self, porosity=0.4, s=2.65, d=0.001, alpha=8.0, m=1.5, theta_cr=0.047, on=True):
        """Bed evolution (Exner, Eq. 3 / Eq. 13-16) with the MPM-like closure (Table 2),
        stepped with the water; z changes and H moves with it."""
        rc = _lib().orc_set_morpho(self._h, int(on), float(porosity), float(s), float(d), float(alpha), float(m),
                                   float(theta_cr))
        if rc != 0:
            raise OracleError(f"orc_set_morpho failed with code {rc}")
        self.morpho = bool(on)

    def set_friction(self, law: int, coef):
        """Friction closure of Table 1: 0 Manning (coef = n), 1 Chezy (coef = K_s),
        2 Bezzola (coef = y_R); coef per cell."""
        c = np.ascontiguousarray(np.broadcast_to(np.asarray(coef, dtype=np.float64), (self.n_cells,)))
        rc = _lib().orc_set_friction(self._h, int(law), _dp(c))
        if rc != 0:
            raise OracleError(f"orc_set_friction failed with code {rc}")

    def set_outflow(self, hq_stage=(), hq_discharge=(), weir_crest: float = 0.0, weir_poleni: float = 0.0):
        """Outflow laws of the h-Q edges (tag 3: rating curve through the (stage,
        discharge) table) and of the weir edges (tag 4: crest elevation, Poleni
        coefficient)."""
        s_ = np.ascontiguousarray(hq_stage, dtype=np.float64)
        q_ = np.ascontiguousarray(hq_discharge, dtype=np.float64)
        if s_.shape != q_.shape:
            raise OracleError("set_outflow: stage and discharge differ in length")
        rc = _lib().orc_set_outflow(self._h, len(s_), _dp(s_), _dp(q_), float(weir_crest), float(weir_poleni))
        if rc != 0:
            raise OracleError(f"orc_set_outflow failed with code {rc}")

    def set_level(self, t_pts, z_pts):
        """The water surface elevation Z_b(t) of the water-level edges (tag 5),
        piecewise linear through (t_pts, z_pts), constant beyond the ends; no points
        turns them back into walls."""
        t_ = np.ascontiguousarray(t_pts, dtype=np.float64)
        z_ = np.ascontiguousarray(z_pts, dtype=np.float64)
        if t_.shape != z_.shape:
            raise OracleError("set_level: times and levels differ in length")
        rc = _lib().orc_set_level(self._h, len(t_), _dp(t_), _dp(z_))
        if rc != 0:
            raise OracleError(f"orc_set_level failed with code {rc}")

    def boundary_discharge(self):
        """Per edge, the unit discharge entering through an inflow edge and the one
        leaving through an outflow edge at the current state (0 elsewhere)."""
        ne = _lib().orc_n_edges(self._h)
        qi, qo = np.empty(ne), np.empty(ne)
        _lib().orc_boundary_discharge(self._h, _dp(self.H), self.t.value, _dp(qi), _dp(qo))
        return qi, qo

    def morpho_speeds(self, i: int, nx: float, ny: float):
        """Eq. 16's (lambda_1, lambda_2) of cell i for the unit normal (nx, ny) at the
        current state, as the bed flux of the next step uses them (needs set_morpho)."""
        a, b = C.c_double(), C.c_double()
        rc = _lib().orc_morpho_speeds(self._h, _dp(self.H), _dp(self.qx), _dp(self.qy), int(i), float(nx), float(ny),
                                      C.byref(a), C.byref(b))
        if rc != 0:
            raise OracleError("orc_morpho_speeds: bed evolution is off or the cell index is out of range")
        return a.value, b.value

    @property
    def bed_outflow(self) -> float:
        """Solid sediment volume that left through the boundary (negative: entered)."""
        return _lib().orc_bed_outflow(self._h)

    @property
    def source_volume(self) -> float:
        """Volume the sources added (negative: sinks removed) since set_sources."""
        return _lib().orc_source_volume(self._h)

    def concentration(self):
        h = self.depth()
        return np.where(h > 0, self.hc / np.where(h > 0, h, 1.0), 0.0)

    def step(self, n: int = 1, t_end: float = math.inf) -> int:
        lib = _lib()
        if self.hc is not None:
            if self.tracking is not None:
                raise OracleError("scalars and flood tracking together are not supported by the oracle")
            k = lib.orc_run_scalars(self._h, _dp(self.H), _dp(self.qx), _dp(self.qy), C.byref(self.t),
                                    float(t_end), int(n), C.byref(self.bvol), self.hc.shape[0], _dp(self.hc),
                                    _dp(self.c_in))
            if k < 0:
                raise OracleError("orc_run_scalars: out of memory")
            self.steps += k
            self._sync_bed()
            return k
        if self.tracking is not None:
            tr = self.tracking
            k = lib.orc_run_tracked(self._h, _dp(self.H), _dp(self.qx), _dp(self.qy), C.byref(self.t),
                                    float(t_end), int(n), C.byref(self.bvol), *self._track_args,
                                    _dp(tr["t_arrival"]), _dp(tr["h_max"]), _dp(tr["u_max"]), _dp(tr["q_max"]),
                                    _dp(tr["tau_max"]))
        else:
            k = lib.orc_run(self._h, _dp(self.H), _dp(self.qx), _dp(self.qy), C.byref(self.t), float(t_end),
                            int(n), C.byref(self.bvol))
        self.steps += k
        self._sync_bed()
        return k

    def run_until(self, t_end: float, max_steps: int = 10**9) -> int:
        return self.step(max_steps, t_end)

    def _sync_bed(self):
        if getattr(self, "morpho", False):
            _lib().orc_bed(self._h, _dp(self.z))

    def next_dt(self) -> float:
        return _lib().orc_next_dt(self._h, _dp(self.H), _dp(self.qx), _dp(self.qy), self.t.value)

    def volume(self) -> float:
        return _lib().orc_volume(self._h, _dp(self.H))

    @property
    def time(self) -> float:
        return self.t.value

    @property
    def boundary_volume(self) -> float:
        return self.bvol.value

    def area(self) -> np.ndarray:
        a = np.empty(self.n_cells)
        _lib().orc_cell_area(self._h, _dp(a))
        return a

    def edges(self):
        lib = _lib()
        ne = lib.orc_n_edges(self._h)
        L = np.empty(ne, np.int64)
        R = np.empty(ne, np.int64)
        nx, ny, ln = np.empty(ne), np.empty(ne), np.empty(ne)
        lib.orc_edges(self._h, L.ctypes.data_as(C.POINTER(C.c_int64)), R.ctypes.data_as(C.POINTER(C.c_int64)),
                      _dp(nx), _dp(ny), _dp(ln))
        return L, R, nx, ny, ln

    def depth(self) -> np.ndarray:
        return self.H - self.z


def hllc(hL, uL, vL, hR, uR, vR, g=9.81):
    """HLLC flux (F_h, F_n, F_t) in the edge frame, as the oracle computes it."""
    out = (C.c_double * 3)()
    _lib().orc_hllc(hL, uL, vL, hR, uR, vR, g, out)
    return np.array(out[:])


def wave_speeds(hL, uL, hR, uR, g=9.81):
    """(S_L, S_R) wave-speed bounds the oracle's HLLC uses."""
    a, b = C.c_double(), C.c_double()
    _lib().orc_wave_speeds(hL, uL, hR, uR, g, C.byref(a), C.byref(b))
    return a.value, b.value


def friction(h, n, dt, qx, qy, g=9.81, h_min=1e-6):
    """One split friction step on (qx, qy) with depth h frozen."""
    a, b = C.c_double(qx), C.c_double(qy)
    _lib().orc_friction(h, n, g, dt, h_min, C.byref(a), C.byref(b))
    return a.value, b.value


def friction_cf(law, h, r):
    """c_f of a Table 1 closure (1 Chezy with K_s = r, 2 Bezzola with y_R = r)."""
    return _lib().orc_cf(int(law), float(h), float(r))


def hydrograph(t_pts, q_pts, t):
    tt = np.ascontiguousarray(t_pts, dtype=np.float64)
    qq = np.ascontiguousarray(q_pts, dtype=np.float64)
    p = _Params(0.9, 9.81, 1e-6, 1.0, 0, _dp(tt), _dp(qq), len(tt))
    return _lib().orc_hydrograph(C.byref(p), float(t))
