"""The C-ABI library loads and exports every entry point include/bm.h declares, and
host-side validation (which runs before any device call) rejects malformed input.
CPU only: no compute call reaches the GPU here."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2102_12862_b300 import bm
from paper_2102_12862_b300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")]


def declared_functions():
    names = set()
    for h in HEADERS:
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(?:bm_status|void|const char\s*\*)\s+(bm_\w+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    lib = bm.load_library()
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"
    assert set(names) <= set(bm.SIGNATURES) | set(getattr(bm, "EXTRA_SIGNATURES", {}))


def test_params_default():
    lib = bm.load_library()
    p = bm.bm_params()
    lib.bm_params_default(C.byref(p))
    assert p.cfl == 0.9 and p.g == 9.81 and p.h_min == 1e-6 and p.dt_max == 1.0
    assert p.precision == bm.BM_FP64 and p.cfl_mode == 0 and np.isnan(p.datum) and p.hydro_n == 0


def _mesh_args():
    s = W.dam_break(nx=4, ny=2)
    return [s.xy.copy(), s.tri.copy(), s.z.copy(), s.manning.copy(), s.edge_tag.copy()]


@pytest.mark.parametrize("mutate,msg", [
    (lambda a: a[1].__setitem__((0, 0), 10_000), "out of range"),
    (lambda a: a[1].__setitem__((0, 1), a[1][0, 0]), "degenerate"),
    (lambda a: a[4].fill(7), "tag"),
    (lambda a: a[4].fill(6), "tag"),
    (lambda a: a[3].__setitem__(0, -0.1), "n >= 0"),
    (lambda a: a[2].__setitem__(1, np.nan), "finite"),
    (lambda a: a[0].__setitem__((3, 0), np.inf), "non-finite"),
])
def test_mesh_validation_rejects(mutate, msg):
    args = _mesh_args()
    mutate(args)
    with pytest.raises(bm.BMError) as ei:
        bm.bm_mesh_create(*args)
    assert ei.value.status == bm.BM_EINVAL and msg in str(ei.value)


def test_mesh_lists_outflow_edges_after_the_inflow_edges():
    """Tags 3 (h-Q relation) and 4 (weir) are outflow edges; the mesh lists them after
    the inflow edges, and the tiles that hold them are boundary tiles."""
    xy, tri, tag = W.rect_mesh(20, 4, 100.0, 20.0, jitter=0.1, seed=1,
                               side_tags=(W.INFLOW, W.WEIR, W.HQ_OUTFLOW, W.WALL))
    N = len(tri)
    m = bm.Mesh(xy, tri, np.zeros(N), np.zeros(N), tag)
    info = m.info
    assert info["n_inflow"] == 4  # the x = 0 side
    assert info["n_boundary"] == 4 + 4 + 20 + 20


def test_mesh_takes_water_level_edges():
    """Tag 5 (water level) is a listed boundary edge too, after the outflow edges."""
    xy, tri, tag = W.rect_mesh(20, 4, 100.0, 20.0, jitter=0.1, seed=1,
                               side_tags=(W.INFLOW, W.WATER_LEVEL, W.HQ_OUTFLOW, W.WALL))
    N = len(tri)
    m = bm.Mesh(xy, tri, np.zeros(N), np.zeros(N), tag)
    assert m.info["n_inflow"] == 4
    assert m.info["n_boundary"] == 4 + 4 + 20 + 20


def test_mesh_rejects_non_manifold_and_flipped():
    xy = np.array([[0, 0], [1, 0], [0, 1], [1, 1], [0.5, -1.0]], float)
    # three triangles on edge (0,1)
    tri = np.array([[0, 1, 2], [1, 0, 4], [0, 1, 3]], np.int32)
    with pytest.raises(bm.BMError, match="more than two"):
        bm.bm_mesh_create(xy, tri, np.zeros(3), np.zeros(3), np.zeros((3, 3), np.uint8))
    # two overlapping triangles traversing (0,1) the same way
    tri = np.array([[0, 1, 2], [0, 1, 3]], np.int32)
    with pytest.raises(bm.BMError, match="same direction"):
        bm.bm_mesh_create(xy, tri, np.zeros(2), np.zeros(2), np.zeros((2, 3), np.uint8))


def test_empty_mesh_rejected():
    with pytest.raises(bm.BMError, match="n_tri"):
        bm.bm_mesh_create(np.zeros((3, 2)), np.zeros((0, 3), np.int32), np.zeros(0), np.zeros(0),
                          np.zeros((0, 3), np.uint8))


def test_params_validation_without_gpu():
    lib = bm.load_library()
    p, keep = bm.make_params(cfl=1.5)
    st = lib.bm_state_init(None, C.byref(p), None, None, None, C.byref(C.c_void_p()))
    assert st == bm.BM_EINVAL


@pytest.mark.parametrize("make", [
    lambda: W.dam_break(),
    lambda: W.floodplain(nx=120, ny=50, Lx=1200.0, Ly=500.0, seed=5),
    lambda: W.dam_break(nx=1000, ny=1, seed=6),  # a strip: tiles are long and thin
])
def test_mesh_layout_on_the_host(make):
    """Meshes are built and tiled without a GPU; the tile records respect the step
    kernel's limits (768 edges and halo cells per tile, 16-byte records)."""
    s = make()
    m = bm.Mesh.from_scenario(s)
    info = m.info
    assert info["n_cells"] == len(s.tri) and info["n_tiles"] == -(-len(s.tri) // 256)
    lay64, lay32 = m.layout("fp64"), m.layout("fp32")
    for lay, S in ((lay64, 8), (lay32, 4)):
        assert 0 < lay["max_tile_edges"] <= 768 and 0 <= lay["max_tile_halo"] <= 768
        assert lay["record_bytes"] % 16 == 0
        # every tile stores its 256 cells (1/area, slot) and each mesh edge at least once
        assert lay["record_bytes"] >= info["n_tiles"] * 256 * (S + 4) + info["n_edges"] * (4 + 3 * S)
    assert lay64["max_tile_edges"] == lay32["max_tile_edges"] and lay64["max_tile_halo"] == lay32["max_tile_halo"]
    with pytest.raises(bm.BMError, match="precision"):
        bm.bm_mesh_layout(m.handle, 7)


def test_math_eval_validates_before_any_device_work():
    lib = bm.load_library()
    assert lib.bm_math_eval(9, None, None, 1) == bm.BM_EINVAL
    assert lib.bm_math_eval(0, None, None, 4) == bm.BM_EINVAL
    assert lib.bm_math_eval(0, None, None, -1) == bm.BM_EINVAL
    assert lib.bm_math_eval(0, None, None, 0) == bm.BM_OK


def test_tracking_validates_before_any_device_work():
    lib = bm.load_library()
    assert lib.bm_state_track(None, 0.01) == bm.BM_EINVAL
    assert lib.bm_state_download_track(None, None, None, None, None, None) == bm.BM_EINVAL
