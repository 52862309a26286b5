"""Python binding of the C ABI in include/bm.h (ctypes; argument marshalling only).

The functions carry the C names (bm_mesh_create, bm_state_init, bm_step, ...);
every step of the shallow-water path runs in the CUDA kernels of libbm.so.  There
is no CPU fallback: loading fails loudly when the library is missing.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbm.so")

BM_OK, BM_EINVAL, BM_ENOMEM, BM_ECUDA, BM_ENONFINITE, BM_ENEGDEPTH, BM_ETIMEOUT, BM_EAGAIN, BM_EBUSY = range(9)
BM_FP64, BM_FP32_BULK = 0, 1
STATUS_NAMES = {0: "BM_OK", 1: "BM_EINVAL", 2: "BM_ENOMEM", 3: "BM_ECUDA", 4: "BM_ENONFINITE",
                5: "BM_ENEGDEPTH", 6: "BM_ETIMEOUT", 7: "BM_EAGAIN", 8: "BM_EBUSY"}


class BMError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class bm_params(C.Structure):
    _fields_ = [("cfl", C.c_double), ("g", C.c_double), ("h_min", C.c_double), ("dt_max", C.c_double),
                ("precision", C.c_int32), ("cfl_mode", C.c_int32), ("datum", C.c_double),
                ("hydro_t", C.POINTER(C.c_double)), ("hydro_q", C.POINTER(C.c_double)),
                ("hydro_n", C.c_int64)]


_lib = None
_P = C.POINTER
_d, _i64, _vp = C.c_double, C.c_int64, C.c_void_p

# name -> (restype, argtypes); the exported surface of include/bm.h
SIGNATURES = {
    "bm_params_default": (None, [_P(bm_params)]),
    "bm_last_error": (C.c_char_p, []),
    "bm_mesh_create": (C.c_int, [_P(_d), _i64, _P(C.c_int32), _i64, _P(_d), _P(_d), _P(C.c_uint8), _P(_vp)]),
    "bm_mesh_info": (C.c_int, [_vp, _P(_i64), _P(_i64), _P(_i64), _P(_i64), _P(_i64)]),
    "bm_mesh_destroy": (None, [_vp]),
    "bm_state_init": (C.c_int, [_vp, _P(bm_params), _P(_d), _P(_d), _P(_d), _P(_vp)]),
    "bm_state_destroy": (None, [_vp]),
    "bm_state_set_stream": (C.c_int, [_vp, _vp]),
    "bm_step": (C.c_int, [_vp, _i64]),
    "bm_step_async": (C.c_int, [_vp, _i64]),
    "bm_sync": (C.c_int, [_vp]),
    "bm_run_until": (C.c_int, [_vp, _d]),
    "bm_state_upload": (C.c_int, [_vp, _P(_d), _P(_d), _P(_d), _d]),
    "bm_state_download": (C.c_int, [_vp, _P(_d), _P(_d), _P(_d), _P(_d)]),
    "bm_state_stats": (C.c_int, [_vp, _P(_d), _P(_d), _P(_i64), _P(_d), _P(_d)]),
    "bm_step_timed": (C.c_int, [_vp, _i64, _P(_d), _P(_d)]),
}


def load_library(path: str = LIB_PATH):
    """Load libbm.so (built by paper_2102_12862_b300.build); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libbm.so not found at {path}: build it with `python -m paper_2102_12862_b300.build` "
                           "(the CUDA path has no CPU fallback)")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(st: int):
    if st != BM_OK:
        msg = load_library().bm_last_error().decode(errors="replace")
        raise BMError(st, msg)


def _dp(a):
    return None if a is None else a.ctypes.data_as(_P(_d))


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def make_params(**kw) -> tuple[bm_params, tuple]:
    """bm_params from keyword values (defaults from bm_params_default); returns the struct
    and the arrays it points into (keep them alive while the struct is used)."""
    lib = load_library()
    p = bm_params()
    lib.bm_params_default(C.byref(p))
    ht = _f64(kw.pop("hydro_t", np.zeros(0)))
    hq = _f64(kw.pop("hydro_q", np.zeros(0)))
    prec = kw.pop("precision", BM_FP64)
    if isinstance(prec, str):
        prec = {"fp64": BM_FP64, "fp32": BM_FP32_BULK, "fp32_bulk": BM_FP32_BULK}[prec.lower()]
    p.precision = prec
    for k, v in kw.items():
        if k == "datum" and v is None:
            v = math.nan
        setattr(p, k, v)
    p.hydro_n = len(ht)
    p.hydro_t = _dp(ht) if len(ht) else None
    p.hydro_q = _dp(hq) if len(hq) else None
    return p, (ht, hq)


# ---------------------------------------------------------------- same-name functions

def bm_mesh_create(xy, tri, z_bed, manning_n, edge_tag) -> int:
    lib = load_library()
    xy = _f64(xy).reshape(-1)
    tri = np.ascontiguousarray(tri, dtype=np.int32).reshape(-1)
    z = _f64(z_bed)
    n = _f64(manning_n)
    tag = np.ascontiguousarray(edge_tag, dtype=np.uint8).reshape(-1)
    out = _vp()
    _check(lib.bm_mesh_create(_dp(xy), len(xy) // 2, tri.ctypes.data_as(_P(C.c_int32)), len(tri) // 3, _dp(z),
                              _dp(n), tag.ctypes.data_as(_P(C.c_uint8)), C.byref(out)))
    return out.value


def bm_mesh_info(mesh: int) -> dict:
    v = [_i64() for _ in range(5)]
    _check(load_library().bm_mesh_info(mesh, *[C.byref(x) for x in v]))
    return dict(zip(["n_cells", "n_edges", "n_boundary", "n_inflow", "n_tiles"], [x.value for x in v]))


def bm_mesh_destroy(mesh: int):
    if mesh:
        load_library().bm_mesh_destroy(mesh)


def bm_state_init(mesh: int, params: bm_params, H, qx=None, qy=None) -> int:
    out = _vp()
    H, qx, qy = _f64(H), _f64(qx), _f64(qy)
    _check(load_library().bm_state_init(mesh, C.byref(params), _dp(H), _dp(qx), _dp(qy), C.byref(out)))
    return out.value


def bm_state_destroy(state: int):
    if state:
        load_library().bm_state_destroy(state)


def bm_state_set_stream(state: int, stream_ptr: int):
    _check(load_library().bm_state_set_stream(state, stream_ptr or None))


def bm_step(state: int, n_steps: int):
    _check(load_library().bm_step(state, int(n_steps)))


def bm_step_async(state: int, n_steps: int):
    _check(load_library().bm_step_async(state, int(n_steps)))


def bm_sync(state: int):
    _check(load_library().bm_sync(state))


def bm_run_until(state: int, t_end: float):
    _check(load_library().bm_run_until(state, float(t_end)))


def bm_state_upload(state: int, H, qx=None, qy=None, t: float = 0.0):
    H, qx, qy = _f64(H), _f64(qx), _f64(qy)
    _check(load_library().bm_state_upload(state, _dp(H), _dp(qx), _dp(qy), float(t)))


def bm_state_download(state: int, n_cells: int, H=None, qx=None, qy=None):
    """Download into the given float64 arrays (allocated if None); returns (H, qx, qy, t)."""
    H = np.empty(n_cells) if H is None else H
    qx = np.empty(n_cells) if qx is None else qx
    qy = np.empty(n_cells) if qy is None else qy
    t = _d()
    _check(load_library().bm_state_download(state, _dp(H), _dp(qx), _dp(qy), C.byref(t)))
    return H, qx, qy, t.value


def bm_state_stats(state: int, volume: bool = True) -> dict:
    t, dt, vol, bv = _d(), _d(), _d(), _d()
    steps = _i64()
    _check(load_library().bm_state_stats(state, C.byref(t), C.byref(dt), C.byref(steps),
                                         C.byref(vol) if volume else None, C.byref(bv)))
    return {"t": t.value, "dt_next": dt.value, "steps": steps.value, "volume": vol.value if volume else None,
            "boundary_volume": bv.value}


def bm_step_timed(state: int, n_steps: int) -> tuple[float, float]:
    """(summed step-kernel ms, total ms) of n_steps steps launched with per-kernel events."""
    k, t = _d(), _d()
    _check(load_library().bm_step_timed(state, int(n_steps), C.byref(k), C.byref(t)))
    return k.value, t.value


# ---------------------------------------------------------------- small owning wrappers

class Mesh:
    def __init__(self, xy, tri, z_bed, manning_n, edge_tag):
        self.handle = bm_mesh_create(xy, tri, z_bed, manning_n, edge_tag)
        self.info = bm_mesh_info(self.handle)
        self.n_cells = self.info["n_cells"]

    @classmethod
    def from_scenario(cls, s) -> "Mesh":
        return cls(s.xy, s.tri, s.z, s.manning, s.edge_tag)

    def close(self):
        if self.handle:
            bm_mesh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class State:
    """A device-resident state on a Mesh (keeps the mesh alive)."""

    def __init__(self, mesh: Mesh, H, qx=None, qy=None, **params):
        self.mesh = mesh
        self._p, self._keep = make_params(**params)
        self.handle = bm_state_init(mesh.handle, self._p, H, qx, qy)
        self.n_cells = mesh.n_cells

    @classmethod
    def from_scenario(cls, s, mesh: Mesh | None = None, **overrides) -> "State":
        prm = dict(s.params)
        prm.update(overrides)
        return cls(mesh or Mesh.from_scenario(s), s.H, s.qx, s.qy, **prm)

    def step(self, n: int = 1):
        bm_step(self.handle, n)

    def step_async(self, n: int = 1):
        bm_step_async(self.handle, n)

    def sync(self):
        bm_sync(self.handle)

    def run_until(self, t_end: float):
        bm_run_until(self.handle, t_end)

    def upload(self, H, qx=None, qy=None, t: float = 0.0):
        bm_state_upload(self.handle, H, qx, qy, t)

    def download(self):
        return bm_state_download(self.handle, self.n_cells)

    def stats(self, volume: bool = True) -> dict:
        return bm_state_stats(self.handle, volume)

    def step_timed(self, n: int) -> tuple[float, float]:
        return bm_step_timed(self.handle, n)

    def set_stream(self, stream_ptr: int):
        bm_state_set_stream(self.handle, stream_ptr)

    def close(self):
        if self.handle:
            bm_state_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
