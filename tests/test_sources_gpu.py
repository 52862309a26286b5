"""External sources and sinks on the GPU (the per-step rate kernel and the S term of
Eq. 12 in the step kernel) against the oracle (Section "External inflow/outflow
discharge").

FP64: relative L-inf 1e-11 on h = H - z, q_x, q_y (normwise, as the state parity),
the lake at rest under rain kept bitwise at rest.  FP32-bulk: the lake rises by i t
within 1e-6 m and stays bitwise at rest; the rained plane's outflow and volume within
that mode's accuracy (1e-4 relative).  An Exact sink larger than the water ends the
run with BM_ENEGDEPTH, as the paper says such a run ends.
"""
import numpy as np
import pytest

import oracle
from paper_2102_12862_b300 import bm
from paper_2102_12862_b300 import workloads as W

pytestmark = pytest.mark.gpu
TOTAL, INTENSITY = bm.SOURCE_TOTAL, bm.SOURCE_INTENSITY
EXACT, AVAILABLE, INFINITY = bm.SINK_EXACT, bm.SINK_AVAILABLE, bm.SINK_INFINITY


def const(v):
    return (np.array([0.0]), np.array([float(v)]))


def rel_linf(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def both(s, region, kind, mode, series, precision="fp64", **kw):
    st = bm.State.from_scenario(s, precision=precision, **kw)
    o = oracle.Oracle(s, **kw)
    st.set_sources(region, kind, mode, series)
    o.set_sources(region, kind, mode, series)
    return st, o


def compare(s, st, o):
    tol = 1e-10 if o.steps > 400 else 1e-11
    H, qx, qy, t = st.download()
    assert abs(t - o.time) <= 1e-12 * max(1.0, o.time)
    for name, a, b in (("h", H - s.z, o.H - s.z), ("hu", qx, o.qx), ("hv", qy, o.qy)):
        if np.max(np.abs(b)) == 0.0:
            assert np.max(np.abs(a)) == 0.0, name
            continue
        e = rel_linf(a, b)
        assert e <= tol, f"{name}: rel Linf {e:.3e} ({o.steps} steps)"
    return H, qx, qy


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_rain_on_lake_at_rest(precision):
    s = W.fractal_lake(nx=60, ny=30, Lx=600.0, Ly=300.0, seed=11, relief=5.0, level=406.0)
    st, o = both(s, np.zeros(len(s.tri)), [INTENSITY], [EXACT], [const(36.0)], precision=precision)
    st.run_until(200.0)
    H, qx, qy, _ = st.download()
    assert not qx.any() and not qy.any()
    if precision == "fp64":
        o.run_until(200.0)
        compare(s, st, o)
    assert np.max(np.abs(H - (406.0 + 1e-5 * 200.0))) <= (1e-11 if precision == "fp64" else 1e-6)


@pytest.mark.parametrize("series", [const(3.0), (np.array([0.0, 10.0, 20.0]), np.array([0.0, 6.0, 1.0]))])
def test_total_discharge_on_a_disk(series):
    """A discharge over a disk in a closed dam break with friction (wet/dry fronts
    around the disk, two tiles' worth of region)."""
    s = W.dam_break(nx=60, ny=12, Lx=60.0, Ly=12.0, x_dam=30.0, closed=True, manning=0.02, seed=3)
    reg = W.disk_region(s, 45.0, 6.0, 3.0)
    st, o = both(s, reg, [TOTAL], [EXACT], [series])
    st.run_until(20.0)
    o.run_until(20.0)
    compare(s, st, o)
    assert abs(st.stats()["volume"] - o.volume()) <= 1e-11 * o.volume()


def sink_case(mode):
    s = W.dam_break(nx=60, ny=12, Lx=60.0, Ly=12.0, x_dam=30.0, closed=True, manning=0.02, seed=3)
    reg = W.disk_region(s, 45.0, 6.0, 3.0)
    # two regions: a strong sink (0.28 m/s) on the disk, a rain on every other cell
    reg2 = np.where(reg == 0, 0, 1).astype(np.int32)
    st, o = both(s, reg2, [INTENSITY, INTENSITY], [mode, EXACT], [const(-1e6), const(50.0)])
    return s, reg == 0, st, o


def test_sink_infinity():
    """Infinity empties the disk every step: element-wise parity over 200 steps."""
    s, inside, st, o = sink_case(INFINITY)
    for _ in range(5):
        st.step(40)
        o.step(40)
        H, _, _ = compare(s, st, o)
        assert np.all(H[inside] == s.z[inside])
        assert (H - s.z).min() >= 0.0


def test_sink_available():
    """Available takes at most the water a cell holds.  Where the prescription and the
    water nearly cancel, the film left is rounding-sized while the cell keeps its
    momentum, so its velocity (and the step Eq. 21 takes) amplifies rounding -- the
    thin-layer sensitivity of the state itself, here on purpose.  Element-wise parity
    over the first 40 steps (before the first such film on this case, where the two
    runs' step sizes part); 10 s later (same time on both sides) the depths stay
    non-negative, the disk is emptied and the volume matches the oracle's to 1e-6."""
    s, inside, st, o = sink_case(AVAILABLE)
    st.step(40)
    o.step(40)
    compare(s, st, o)
    t_end = o.time + 10.0
    st.run_until(t_end)
    o.run_until(t_end)
    H, _, _, _ = st.download()
    assert (H - s.z).min() >= 0.0
    assert np.any(H[inside] == s.z[inside])
    assert abs(st.stats()["volume"] - o.volume()) <= 1e-6 * o.volume()


def test_exact_sink_past_the_water_fails():
    s = W.dam_break(nx=60, ny=12, Lx=60.0, Ly=12.0, x_dam=30.0, closed=True, manning=0.02, seed=3)
    st = bm.State.from_scenario(s)
    st.set_sources(W.disk_region(s, 45.0, 6.0, 3.0), [INTENSITY], [EXACT], [const(-1e6)])
    with pytest.raises(bm.BMError) as ei:
        st.step(200)
    assert ei.value.status == bm.BM_ENEGDEPTH


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_rained_plane(precision):
    """Rain on an initially dry plane (wet/dry front from the crest down, transmissive
    outlet): FP64 element-wise; FP32-bulk stored volume and outflow within 1e-4."""
    s = W.rained_plane(slope=0.001)
    st, o = both(s, np.zeros(len(s.tri)), [INTENSITY], [EXACT], [const(100.0)], precision=precision)
    st.run_until(1500.0)
    o.run_until(1500.0)
    if precision == "fp64":
        compare(s, st, o)
    else:
        stats = st.stats()
        assert abs(stats["volume"] - o.volume()) <= 1e-4 * o.volume()
        assert abs(stats["boundary_volume"] - o.boundary_volume) <= 1e-4 * abs(o.boundary_volume) + 1e-6


def test_source_api_rules():
    s = W.dam_break(nx=40, ny=4, manning=0.02)
    st = bm.State.from_scenario(s)
    n = len(s.tri)
    with pytest.raises(bm.BMError, match="kind"):
        st.set_sources(np.zeros(n), [5], [EXACT], [const(1.0)])
    with pytest.raises(bm.BMError, match="increase strictly"):
        st.set_sources(np.zeros(n), [INTENSITY], [EXACT], [(np.array([1.0, 1.0]), np.array([1.0, 2.0]))])
    with pytest.raises(bm.BMError, match="out of range"):
        st.set_sources(np.full(n, 3), [INTENSITY], [EXACT], [const(1.0)])
    st.set_sources(np.zeros(n), [INTENSITY], [EXACT], [const(1.0)])
    st.step(3)
    st.set_sources(np.zeros(n), [], [], [])
    st.set_scalars(np.zeros((1, n)))  # species and sources may be set in either order
    st.set_sources(np.zeros(n), [INTENSITY], [EXACT], [const(1.0)])
    st.step(2)
