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


class bm_server_opts(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_uint64), ("max_slots", C.c_int32), ("precision", C.c_int32),
                ("steps_per_round", C.c_int32), ("ctas_per_sm", C.c_int32)]


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
    "bm_mesh_layout": (C.c_int, [_vp, C.c_int32, _P(_i64), _P(_i64), _P(_i64)]),
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
    "bm_state_work": (C.c_int, [_vp, _P(_i64), _P(_i64)]),
    "bm_state_set_tile_skipping": (C.c_int, [_vp, C.c_int32]),
    "bm_step_timed": (C.c_int, [_vp, _i64, _P(_d), _P(_d)]),
    "bm_state_test_timeout": (C.c_int, [_vp]),
    "bm_state_set_launch": (C.c_int, [_vp, C.c_int]),
    "bm_state_set_schedule": (C.c_int, [_vp, C.c_int, C.c_int]),
    "bm_state_get_schedule": (C.c_int, [_vp, _P(C.c_int), _P(C.c_int)]),
    "bm_batch_set_schedule": (C.c_int, [_vp, C.c_int, C.c_int]),
    "bm_batch_get_schedule": (C.c_int, [_vp, _P(C.c_int), _P(C.c_int)]),
    "bm_state_set_slots": (C.c_int, [_vp, C.c_int]),
    "bm_state_get_slots": (C.c_int, [_vp, _P(C.c_int)]),
    "bm_batch_set_slots": (C.c_int, [_vp, C.c_int]),
    "bm_batch_get_slots": (C.c_int, [_vp, _P(C.c_int)]),
    "bm_state_set_claim": (C.c_int, [_vp, C.c_int]),
    "bm_state_get_claim": (C.c_int, [_vp, _P(C.c_int)]),
    "bm_batch_set_claim": (C.c_int, [_vp, C.c_int]),
    "bm_batch_get_claim": (C.c_int, [_vp, _P(C.c_int)]),
    "bm_batch_create": (C.c_int, [_P(_vp), C.c_int32, _P(_vp)]),
    "bm_batch_destroy": (None, [_vp]),
    "bm_batch_info": (C.c_int, [_vp, _P(C.c_int32), _P(_i64), _P(_i64)]),
    "bm_batch_set_stream": (C.c_int, [_vp, _vp]),
    "bm_batch_set_launch": (C.c_int, [_vp, C.c_int]),
    "bm_batch_step": (C.c_int, [_vp, _i64]),
    "bm_batch_step_async": (C.c_int, [_vp, _i64]),
    "bm_batch_sync": (C.c_int, [_vp]),
    "bm_batch_run_until": (C.c_int, [_vp, _P(_d)]),
    "bm_state_autotune": (C.c_int, [_vp, C.c_int, _P(C.c_int), _P(_d)]),
    "bm_batch_autotune": (C.c_int, [_vp, C.c_int, _P(C.c_int), _P(_d)]),
    "bm_volume_noalloc": (C.c_int, [_vp, _vp, _vp, _i64, _vp, _vp]),
    "bm_math_eval": (C.c_int, [C.c_int32, _vp, _vp, _i64]),
    "bm_state_track": (C.c_int, [_vp, C.c_double]),
    "bm_state_download_track": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "bm_state_set_scalars": (C.c_int, [_vp, C.c_int32, _vp, _vp]),
    "bm_state_download_scalars": (C.c_int, [_vp, _vp]),
    "bm_state_set_sources": (C.c_int, [_vp, C.c_int32, _vp, _vp, _vp, _vp, _vp, _vp]),
    "bm_state_set_morpho": (C.c_int, [_vp, C.c_int32, _d, _d, _d, _d, _d, _d]),
    "bm_state_download_bed": (C.c_int, [_vp, _vp]),
    "bm_state_set_friction": (C.c_int, [_vp, C.c_int32, _vp]),
    "bm_state_set_outflow": (C.c_int, [_vp, _vp, _vp, _i64, _d, _d]),
    "bm_state_set_level": (C.c_int, [_vp, _vp, _vp, _i64]),
    "bm_server_opts_default": (None, [_P(bm_server_opts)]),
    "bm_server_create": (C.c_int, [_P(bm_server_opts), _P(_vp)]),
    "bm_server_destroy": (None, [_vp]),
    "bm_submit": (C.c_int, [_vp, _vp, _P(bm_params), _P(_d), _P(_d), _P(_d), _d, _P(C.c_uint64)]),
    "bm_poll": (C.c_int, [_vp, C.c_uint64, _P(_d), _P(_d), _P(_d), _P(_d)]),
    "bm_submit_tracked": (C.c_int, [_vp, _vp, _P(bm_params), _P(_d), _P(_d), _P(_d), _d, _d, _P(C.c_uint64)]),
    "bm_poll_track": (C.c_int, [_vp, C.c_uint64, _P(_d), _P(_d), _P(_d), _P(_d), _P(_d)]),
    "bm_server_wait": (C.c_int, [_vp, C.c_uint64, _d]),
    "bm_server_stats": (C.c_int, [_vp, _P(_i64), _P(_i64), _P(_i64), _P(_d), _P(_d)]),
}



def _precision(prec) -> int:
    if isinstance(prec, str):
        return {"fp64": BM_FP64, "fp32": BM_FP32_BULK, "fp32_bulk": BM_FP32_BULK}[prec.lower()]
    return int(prec)

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
    p.precision = _precision(kw.pop("precision", BM_FP64))
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


def bm_mesh_layout(mesh: int, precision) -> dict:
    v = [_i64() for _ in range(3)]
    _check(load_library().bm_mesh_layout(mesh, _precision(precision), *[C.byref(x) for x in v]))
    return dict(zip(["max_tile_edges", "max_tile_halo", "record_bytes"], [x.value for x in v]))


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


TRACK_FIELDS = ("t_arrival", "h_max", "u_max", "q_max", "tau_max")


def bm_state_track(state: int, h_arrival: float):
    _check(load_library().bm_state_track(state, float(h_arrival)))


def bm_state_download_track(state: int, n_cells: int) -> dict:
    """The flood-tracking record in the caller's cell order (see bm_state_track)."""
    out = {k: np.empty(n_cells) for k in TRACK_FIELDS}
    _check(load_library().bm_state_download_track(state, *(_dp(out[k]) for k in TRACK_FIELDS)))
    return out


def bm_state_set_scalars(state: int, hc, c_in=None):
    """Passive species q_c = h phi_c: hc of shape (K, n_cells), K <= 5 (0 rows: none);
    c_in: K inflow concentrations (None: 0)."""
    hc = np.ascontiguousarray(np.atleast_2d(np.asarray(hc, dtype=np.float64)))
    k = hc.shape[0] if hc.size else 0
    ci = None if c_in is None else np.ascontiguousarray(np.asarray(c_in, dtype=np.float64).reshape(-1))
    if ci is not None and ci.size != k:
        raise ValueError("c_in needs one value per species")
    _check(load_library().bm_state_set_scalars(state, k, _dp(hc) if k else None, _dp(ci) if ci is not None else None))
    return hc, ci


def manning_from_strickler(k_str):
    """Strickler's coefficient k_str [m^(1/3)/s] as the Manning n the library takes:
    Table 1's Strickler law is Manning's with n = 1 / k_str."""
    return 1.0 / np.asarray(k_str, dtype=np.float64)


FRICTION_MANNING, FRICTION_CHEZY, FRICTION_BEZZOLA = 0, 1, 2
SOURCE_TOTAL, SOURCE_INTENSITY = 0, 1          # kind: m^3/s over the region, mm/h
SINK_EXACT, SINK_AVAILABLE, SINK_INFINITY = 0, 1, 2


def bm_state_set_sources(state: int, region, kind, mode, series):
    """External sources / sinks: region (n_cells,) of each cell (-1: none); per region
    kind, mode and series (t, v) of v(t)."""
    i32 = C.c_int32
    kind = np.ascontiguousarray(kind, dtype=np.int32).reshape(-1)
    mode = np.ascontiguousarray(mode, dtype=np.int32).reshape(-1)
    nr = len(kind)
    if len(mode) != nr or len(series) != nr:
        raise ValueError("kind, mode and series need one entry per region")
    reg = np.ascontiguousarray(region, dtype=np.int32).reshape(-1)
    off = np.zeros(nr + 1, np.int64)
    for r, (t, _) in enumerate(series):
        off[r + 1] = off[r] + len(t)
    tt = np.ascontiguousarray(np.concatenate([np.asarray(t, float) for t, _ in series]) if nr else np.zeros(1))
    vv = np.ascontiguousarray(np.concatenate([np.asarray(v, float) for _, v in series]) if nr else np.zeros(1))
    keep = (reg, kind, mode, off, tt, vv)
    _check(load_library().bm_state_set_sources(state, nr, reg.ctypes.data_as(_P(i32)), kind.ctypes.data_as(_P(i32)),
                                               mode.ctypes.data_as(_P(i32)), off.ctypes.data_as(_P(C.c_int64)),
                                               _dp(tt), _dp(vv)))
    return keep


def bm_state_download_scalars(state: int, n_species: int, n_cells: int) -> np.ndarray:
    """q_c of the state's species, shape (K, n_cells), caller cell order."""
    out = np.empty((n_species, n_cells))
    _check(load_library().bm_state_download_scalars(state, _dp(out)))
    return out


def bm_state_stats(state: int, volume: bool = True) -> dict:
    t, dt, vol, bv = _d(), _d(), _d(), _d()
    steps = _i64()
    _check(load_library().bm_state_stats(state, C.byref(t), C.byref(dt), C.byref(steps),
                                         C.byref(vol) if volume else None, C.byref(bv)))
    return {"t": t.value, "dt_next": dt.value, "steps": steps.value, "volume": vol.value if volume else None,
            "boundary_volume": bv.value}


def bm_state_work(state: int) -> tuple[int, int]:
    """(tiles the last step launch took, tiles of the state)."""
    nxt, tot = _i64(), _i64()
    _check(load_library().bm_state_work(state, C.byref(nxt), C.byref(tot)))
    return nxt.value, tot.value


def bm_state_set_tile_skipping(state: int, on: bool) -> None:
    _check(load_library().bm_state_set_tile_skipping(state, 1 if on else 0))


def bm_step_timed(state: int, n_steps: int) -> tuple[float, float]:
    """(summed step-kernel ms, total ms) of n_steps steps launched with per-kernel events."""
    k, t = _d(), _d()
    _check(load_library().bm_step_timed(state, int(n_steps), C.byref(k), C.byref(t)))
    return k.value, t.value


def bm_state_test_timeout(state: int):
    """One step launch whose bounded data wait runs out on purpose (diagnostics of the
    failure path); raises BMError(BM_ETIMEOUT).  Re-upload the state afterwards."""
    _check(load_library().bm_state_test_timeout(state))


def bm_state_set_launch(state: int, ctas_per_sm: int):
    _check(load_library().bm_state_set_launch(state, int(ctas_per_sm)))


def bm_volume_noalloc(H_dev: int, z_dev: int, area_dev: int, n_cells: int, volume_dev: int, stream_ptr: int = 0):
    """Volume of caller-owned device arrays (raw device pointers), no device allocation."""
    _check(load_library().bm_volume_noalloc(H_dev, z_dev, area_dev, int(n_cells), volume_dev, stream_ptr or None))


MATH_FUNCTIONS = {"rcbrt": 0, "rcbrt_lib": 1, "rcp": 2, "rcp_lib": 3, "rcbrt32": 4, "rcbrt32_lib": 5,
                  "cbrt": 6, "cbrt_lib": 7}


def bm_math_eval(fn: str, x) -> np.ndarray:
    """One of the step kernel's elementary functions (or the CUDA library's) on x."""
    xs = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    y = np.empty_like(xs)
    _check(load_library().bm_math_eval(MATH_FUNCTIONS[fn], xs.ctypes.data, y.ctypes.data, xs.size))
    return y


def bm_state_autotune(state: int, steps_per_trial: int = 20) -> tuple[int, float]:
    best, ms = C.c_int(), _d()
    _check(load_library().bm_state_autotune(state, int(steps_per_trial), C.byref(best), C.byref(ms)))
    return best.value, ms.value


def bm_batch_autotune(batch: int, steps_per_trial: int = 10) -> tuple[int, float]:
    best, ms = C.c_int(), _d()
    _check(load_library().bm_batch_autotune(batch, int(steps_per_trial), C.byref(best), C.byref(ms)))
    return best.value, ms.value


def bm_batch_create(states) -> int:
    arr = (_vp * len(states))(*[s.handle if hasattr(s, "handle") else s for s in states])
    out = _vp()
    _check(load_library().bm_batch_create(arr, len(states), C.byref(out)))
    return out.value


def bm_batch_destroy(batch: int):
    if batch:
        load_library().bm_batch_destroy(batch)


def bm_batch_info(batch: int) -> dict:
    m, c, t = C.c_int32(), _i64(), _i64()
    _check(load_library().bm_batch_info(batch, C.byref(m), C.byref(c), C.byref(t)))
    return {"n_members": m.value, "n_cells": c.value, "n_tiles": t.value}


def bm_batch_set_stream(batch: int, stream_ptr: int):
    _check(load_library().bm_batch_set_stream(batch, stream_ptr or None))


def bm_state_set_schedule(state: int, ctas_per_sm: int, static_sixteenths: int = -1):
    _check(load_library().bm_state_set_schedule(state, int(ctas_per_sm), int(static_sixteenths)))


def bm_state_get_schedule(state: int) -> tuple[int, int]:
    c, s = C.c_int(), C.c_int()
    _check(load_library().bm_state_get_schedule(state, C.byref(c), C.byref(s)))
    return c.value, s.value


def bm_batch_set_schedule(batch: int, ctas_per_sm: int, static_sixteenths: int = -1):
    _check(load_library().bm_batch_set_schedule(batch, int(ctas_per_sm), int(static_sixteenths)))


def bm_batch_get_schedule(batch: int) -> tuple[int, int]:
    c, s = C.c_int(), C.c_int()
    _check(load_library().bm_batch_get_schedule(batch, C.byref(c), C.byref(s)))
    return c.value, s.value


def bm_state_set_slots(state: int, slots: int):
    _check(load_library().bm_state_set_slots(state, int(slots)))


def bm_state_get_slots(state: int) -> int:
    k = C.c_int()
    _check(load_library().bm_state_get_slots(state, C.byref(k)))
    return k.value


def bm_batch_set_slots(batch: int, slots: int):
    _check(load_library().bm_batch_set_slots(batch, int(slots)))


def bm_batch_get_slots(batch: int) -> int:
    k = C.c_int()
    _check(load_library().bm_batch_get_slots(batch, C.byref(k)))
    return k.value


def bm_state_set_claim(state: int, mode: int):
    _check(load_library().bm_state_set_claim(state, int(mode)))


def bm_state_get_claim(state: int) -> int:
    k = C.c_int()
    _check(load_library().bm_state_get_claim(state, C.byref(k)))
    return k.value


def bm_batch_set_claim(batch: int, mode: int):
    _check(load_library().bm_batch_set_claim(batch, int(mode)))


def bm_batch_get_claim(batch: int) -> int:
    k = C.c_int()
    _check(load_library().bm_batch_get_claim(batch, C.byref(k)))
    return k.value


def bm_batch_set_launch(batch: int, ctas_per_sm: int):
    _check(load_library().bm_batch_set_launch(batch, int(ctas_per_sm)))


def bm_batch_step(batch: int, n_steps: int):
    _check(load_library().bm_batch_step(batch, int(n_steps)))


def bm_batch_step_async(batch: int, n_steps: int):
    _check(load_library().bm_batch_step_async(batch, int(n_steps)))


def bm_batch_sync(batch: int):
    _check(load_library().bm_batch_sync(batch))


def bm_batch_run_until(batch: int, t_end):
    te = _f64(np.atleast_1d(t_end))
    _check(load_library().bm_batch_run_until(batch, _dp(te)))


# ---------------------------------------------------------------- small owning wrappers

class Mesh:
    def __init__(self, xy, tri, z_bed, manning_n, edge_tag):
        self.handle = bm_mesh_create(xy, tri, z_bed, manning_n, edge_tag)
        self.z_bed = np.array(z_bed, dtype=np.float64)  # caller order (species concentrations)
        self.info = bm_mesh_info(self.handle)
        self.n_cells = self.info["n_cells"]

    @classmethod
    def from_scenario(cls, s) -> "Mesh":
        return cls(s.xy, s.tri, s.z, s.manning, s.edge_tag)

    def layout(self, precision="fp64") -> dict:
        return bm_mesh_layout(self.handle, precision)

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
        self.n_species = 0

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

    def track(self, h_arrival: float = 0.01):
        """Start flood tracking from the current state (updated with every step)."""
        bm_state_track(self.handle, h_arrival)

    def download_track(self) -> dict:
        return bm_state_download_track(self.handle, self.n_cells)

    def set_scalars(self, hc, c_in=None):
        """Carry passive species q_c = h phi_c (shape (K, n_cells), K <= 5), advected
        with every step from now on; c_in: their inflow concentrations."""
        hc, _ = bm_state_set_scalars(self.handle, hc, c_in)
        self.n_species = hc.shape[0] if hc.size else 0

    def set_sources(self, region, kind, mode, series):
        """External sources / sinks S_h over regions (see bm_state_set_sources):
        region (n_cells,) of each cell (-1: none); per region kind (SOURCE_TOTAL m^3/s,
        SOURCE_INTENSITY mm/h), mode (SINK_EXACT / SINK_AVAILABLE / SINK_INFINITY) and
        series (t, v) of v(t); no regions removes them."""
        bm_state_set_sources(self.handle, region, kind, mode, series)

    def set_morpho(self, porosity=0.4, s=2.65, d=0.001, alpha=8.0, m=1.5, theta_cr=0.047, on=True):
        """Bed evolution (Exner with the HLL sediment flux and the MPM-like closure;
        see bm_state_set_morpho), stepped with the water from now on (FP64 states)."""
        _check(load_library().bm_state_set_morpho(self.handle, int(on), float(porosity), float(s), float(d),
                                                  float(alpha), float(m), float(theta_cr)))

    def set_friction(self, law: int, coef):
        """Friction closure of Table 1: FRICTION_MANNING (coef = n), FRICTION_CHEZY
        (coef = K_s), FRICTION_BEZZOLA (coef = y_R); coef scalar or per cell."""
        c = np.ascontiguousarray(np.broadcast_to(np.asarray(coef, dtype=np.float64), (self.n_cells,)))
        _check(load_library().bm_state_set_friction(self.handle, int(law), _dp(c)))

    def set_outflow(self, hq_stage=(), hq_discharge=(), weir_crest: float = 0.0, weir_poleni: float = 0.0):
        """Outflow laws of the h-Q edges (tag 3: rating curve through the (stage,
        discharge) table) and of the weir edges (tag 4: crest elevation, Poleni
        coefficient); see bm_state_set_outflow."""
        st = np.ascontiguousarray(hq_stage, dtype=np.float64)
        dq = np.ascontiguousarray(hq_discharge, dtype=np.float64)
        if st.shape != dq.shape or st.ndim != 1:
            raise ValueError("set_outflow: hq_stage and hq_discharge must be 1-D and of equal length")
        _check(load_library().bm_state_set_outflow(self.handle, _dp(st) if len(st) else None,
                                                   _dp(dq) if len(dq) else None, len(st), float(weir_crest),
                                                   float(weir_poleni)))

    def set_level(self, t=(), z=()):
        """Water-level series of the level edges (tag 5): the imposed surface Z_b(t),
        piecewise linear through (t[k], z[k]); empty: the edges are walls. See
        bm_state_set_level."""
        tt = np.ascontiguousarray(t, dtype=np.float64)
        zz = np.ascontiguousarray(z, dtype=np.float64)
        if tt.shape != zz.shape or tt.ndim != 1:
            raise ValueError("set_level: t and z must be 1-D and of equal length")
        _check(load_library().bm_state_set_level(self.handle, _dp(tt) if len(tt) else None,
                                                 _dp(zz) if len(zz) else None, len(tt)))

    def download_bed(self) -> np.ndarray:
        """The bed elevation z (caller cell order)."""
        z = np.empty(self.n_cells)
        _check(load_library().bm_state_download_bed(self.handle, _dp(z)))
        return z

    def download_scalars(self) -> np.ndarray:
        return bm_state_download_scalars(self.handle, self.n_species, self.n_cells)

    def concentration(self) -> np.ndarray:
        """phi_c = q_c / h where h > 0, else 0 (shape (K, n_cells))."""
        hc = self.download_scalars()
        H, _, _, _ = self.download()
        h = H - self.mesh.z_bed
        return np.where(h > 0, hc / np.where(h > 0, h, 1.0), 0.0)

    def stats(self, volume: bool = True) -> dict:
        return bm_state_stats(self.handle, volume)

    def step_timed(self, n: int) -> tuple[float, float]:
        return bm_step_timed(self.handle, n)

    def work(self) -> tuple[int, int]:
        """(tiles the last step launch took, tiles of the state)."""
        return bm_state_work(self.handle)

    def set_tile_skipping(self, on: bool):
        bm_state_set_tile_skipping(self.handle, on)

    def test_timeout(self):
        bm_state_test_timeout(self.handle)

    def set_stream(self, stream_ptr: int):
        bm_state_set_stream(self.handle, stream_ptr)

    def set_launch(self, ctas_per_sm: int):
        bm_state_set_launch(self.handle, ctas_per_sm)

    def set_schedule(self, ctas_per_sm: int, static_sixteenths: int = -1):
        bm_state_set_schedule(self.handle, ctas_per_sm, static_sixteenths)

    def schedule(self) -> tuple[int, int]:
        """(CTAs per SM, static share of the tickets in sixteenths; -1 = default)."""
        return bm_state_get_schedule(self.handle)

    def set_slots(self, slots: int):
        """Tile slots of the step kernel's pipeline (2, 3 or 4)."""
        bm_state_set_slots(self.handle, slots)

    def slots(self) -> int:
        """The tile slots in force (3 while optional features are on)."""
        return bm_state_get_slots(self.handle)

    def set_claim(self, mode: int):
        """Work-item claiming: 0 ahead, 1 right after each issue, 2 once a slot is free,
        3 also once the tile before is past its edges; -1 the precision's default (FP64 3,
        FP32-bulk 2)."""
        bm_state_set_claim(self.handle, mode)

    def claim(self) -> int:
        return bm_state_get_claim(self.handle)

    def autotune(self, steps_per_trial: int = 20) -> tuple[int, float]:
        return bm_state_autotune(self.handle, steps_per_trial)

    def close(self):
        if self.handle:
            bm_state_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many states stepped by one launch per step (keeps the member States alive)."""

    def __init__(self, states):
        self.states = list(states)
        self.handle = bm_batch_create(self.states)
        self.info = bm_batch_info(self.handle)

    def step(self, n: int = 1):
        bm_batch_step(self.handle, n)

    def step_async(self, n: int = 1):
        bm_batch_step_async(self.handle, n)

    def sync(self):
        bm_batch_sync(self.handle)

    def run_until(self, t_end):
        te = np.broadcast_to(np.asarray(t_end, dtype=np.float64), (len(self.states),)).copy()
        bm_batch_run_until(self.handle, te)

    def set_stream(self, stream_ptr: int):
        bm_batch_set_stream(self.handle, stream_ptr)

    def set_launch(self, ctas_per_sm: int):
        bm_batch_set_launch(self.handle, ctas_per_sm)

    def set_schedule(self, ctas_per_sm: int, static_sixteenths: int = -1):
        bm_batch_set_schedule(self.handle, ctas_per_sm, static_sixteenths)

    def schedule(self) -> tuple[int, int]:
        return bm_batch_get_schedule(self.handle)

    def set_slots(self, slots: int):
        bm_batch_set_slots(self.handle, slots)

    def slots(self) -> int:
        return bm_batch_get_slots(self.handle)

    def set_claim(self, mode: int):
        bm_batch_set_claim(self.handle, mode)

    def claim(self) -> int:
        return bm_batch_get_claim(self.handle)

    def autotune(self, steps_per_trial: int = 10) -> tuple[int, float]:
        return bm_batch_autotune(self.handle, steps_per_trial)

    def close(self):
        if self.handle:
            bm_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- request server

def bm_server_create(precision=BM_FP32_BULK, hbm_budget_bytes: int = 0, max_slots: int = 0,
                     steps_per_round: int = 64, ctas_per_sm: int = 0) -> int:
    lib = load_library()
    o = bm_server_opts()
    lib.bm_server_opts_default(C.byref(o))
    if isinstance(precision, str):
        precision = _precision(precision)
    o.precision = precision
    o.hbm_budget_bytes = int(hbm_budget_bytes)
    o.max_slots = int(max_slots)
    o.steps_per_round = int(steps_per_round)
    o.ctas_per_sm = int(ctas_per_sm)
    out = _vp()
    _check(lib.bm_server_create(C.byref(o), C.byref(out)))
    return out.value


def bm_server_destroy(server: int):
    if server:
        load_library().bm_server_destroy(server)


def bm_submit(server: int, mesh: int, params: bm_params, H, qx=None, qy=None, t_end: float = 1.0) -> int:
    H, qx, qy = _f64(H), _f64(qx), _f64(qy)
    tk = C.c_uint64()
    _check(load_library().bm_submit(server, mesh, C.byref(params), _dp(H), _dp(qx), _dp(qy), float(t_end),
                                    C.byref(tk)))
    return tk.value


def bm_submit_tracked(server: int, mesh: int, params: bm_params, H, qx=None, qy=None, t_end: float = 1.0,
                      h_arrival: float = 0.01) -> int:
    H, qx, qy = _f64(H), _f64(qx), _f64(qy)
    tk = C.c_uint64()
    _check(load_library().bm_submit_tracked(server, mesh, C.byref(params), _dp(H), _dp(qx), _dp(qy), float(t_end),
                                            float(h_arrival), C.byref(tk)))
    return tk.value


def bm_poll_track(server: int, ticket: int, n_cells: int):
    """The finished run's flood-tracking record (dict), None while BM_EAGAIN."""
    out = {k: np.empty(n_cells) for k in TRACK_FIELDS}
    st = load_library().bm_poll_track(server, int(ticket), *(_dp(out[k]) for k in TRACK_FIELDS))
    if st == BM_EAGAIN:
        return None
    _check(st)
    return out


def bm_poll(server: int, ticket: int, n_cells: int):
    """(H, qx, qy, latency_s) when finished, None while BM_EAGAIN; raises on failure."""
    H, qx, qy = np.empty(n_cells), np.empty(n_cells), np.empty(n_cells)
    lat = _d()
    st = load_library().bm_poll(server, int(ticket), _dp(H), _dp(qx), _dp(qy), C.byref(lat))
    if st == BM_EAGAIN:
        return None
    _check(st)
    return H, qx, qy, lat.value


def bm_server_wait(server: int, ticket: int, timeout_s: float = 600.0):
    _check(load_library().bm_server_wait(server, int(ticket), float(timeout_s)))


def bm_server_stats(server: int) -> dict:
    q, r, c = _i64(), _i64(), _i64()
    cu, rb = _d(), _d()
    _check(load_library().bm_server_stats(server, C.byref(q), C.byref(r), C.byref(c), C.byref(cu), C.byref(rb)))
    return {"queued": q.value, "running": r.value, "completed": c.value, "cell_updates": cu.value,
            "resident_bytes": rb.value}


class Server:
    """Owning wrapper of a request server; keeps submitted meshes and params alive."""

    def __init__(self, precision="fp32", **opts):
        self.handle = bm_server_create(precision=precision, **opts)
        self.precision = precision
        self._keep = {}

    def submit(self, mesh: Mesh, H, qx=None, qy=None, t_end: float = 1.0, track=None, **params) -> int:
        """track: the flood-tracking arrival threshold (None: no tracking)."""
        params.setdefault("precision", self.precision)
        p, keep = make_params(**params)
        if track is None:
            tk = bm_submit(self.handle, mesh.handle, p, H, qx, qy, t_end)
        else:
            tk = bm_submit_tracked(self.handle, mesh.handle, p, H, qx, qy, t_end, track)
        self._keep[tk] = (mesh, p, keep)
        return tk

    def poll_track(self, ticket: int):
        """The finished run's tracking record; call before poll() / wait()."""
        return bm_poll_track(self.handle, ticket, self._keep[ticket][0].n_cells)

    def poll(self, ticket: int):
        mesh = self._keep[ticket][0]
        r = bm_poll(self.handle, ticket, mesh.n_cells)
        if r is not None:
            self._keep.pop(ticket, None)
        return r

    def wait(self, ticket: int, timeout_s: float = 600.0):
        bm_server_wait(self.handle, ticket, timeout_s)
        return self.poll(ticket)

    def stats(self) -> dict:
        return bm_server_stats(self.handle)

    def close(self):
        if self.handle:
            bm_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
