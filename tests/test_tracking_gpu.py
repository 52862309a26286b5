"""Flood tracking in the step kernel (front arrival time, maxima of depth, velocity,
specific discharge and bed shear stress) against the oracle's record.

FP64: maxima of depth and discharge within relative L-inf 1e-11 (normwise per field;
1e-10 after more than 400 steps, as the state parity), of velocity and shear stress
within 100 times that (they divide by thin depths), arrival times equal to the time parity bar
(the threshold decision may flip only where the depth lands within rounding of the
threshold: at most 2 cells, each within a step of the oracle's time).  FP32-bulk:
the record within that mode's accuracy (depth 1e-4 m L1).  The record is bitwise the
same alone and in a batch, and a cell copied through (dry, at rest) keeps its record.
"""
import numpy as np
import pytest

import oracle
from paper_2102_12862_b300 import bm
from paper_2102_12862_b300 import workloads as W

pytestmark = pytest.mark.gpu
FIELDS = ("h_max", "u_max", "q_max", "tau_max")


def rel_linf(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def compare_fp64(st, o, max_dt):
    # the state's own bar: 1e-11, or 1e-10 after more than 400 steps (as the state
    # parity tests; |u| = |q| / h carries the state's error divided by small depths)
    # |u| and the shear stress (~ |u|^2 / h^(1/3)) divide by the depth: in a thin
    # layer just above h_min the state's rounding differences grow by (max h) / h, so
    # those two fields get 100 times the bar
    tol = 1e-10 if o.steps > 400 else 1e-11
    g, r = st.download_track(), o.tracking
    for k in FIELDS:
        e = rel_linf(g[k], r[k])
        bar = tol * (100 if k in ("u_max", "tau_max") else 1)
        assert e <= bar, f"{k}: rel Linf {e:.3e} ({o.steps} steps)"
    # arrival times are step times: equal within the time parity bar (1e-12 relative)
    ga, ra = g["t_arrival"], r["t_arrival"]
    close = np.abs(ga - ra) <= 1e-12 * np.maximum(1.0, np.abs(ra))
    same = (np.isnan(ga) & np.isnan(ra)) | close
    assert (~same).sum() <= 2, f"{(~same).sum()} arrival times differ"
    both_set = ~same & ~np.isnan(ga) & ~np.isnan(ra)
    assert np.all(np.abs(ga[both_set] - ra[both_set]) <= max_dt)
    return g


def test_floodplain_fp64_matches_oracle():
    """Inflow hydrograph, transmissive outlet, walls and wet/dry fronts: tracking from
    t = 0 (threshold 0.05 m), 150 s of flood."""
    s = W.floodplain(nx=120, ny=50, Lx=1200.0, Ly=500.0, seed=22, q_peak=200.0, ramp=100.0,
                     outlet=W.TRANSMISSIVE)
    st = bm.State.from_scenario(s)
    o = oracle.Oracle(s)
    st.track(0.05)
    o.track(0.05)
    st.run_until(150.0)
    o.run_until(150.0)
    g = compare_fp64(st, o, max_dt=1.0)
    arrived = ~np.isnan(g["t_arrival"])
    assert arrived.sum() > np.sum(s.H - s.z > 0.05)  # the flood reached new cells
    assert np.nanmax(g["t_arrival"]) > 0


def test_dam_break_fp64_restart_and_shear():
    """Wet dam break with friction: 100 steps, then the record restarted mid-run and
    200 more steps on both sides (restart takes the current state and time)."""
    s = W.dam_break(manning=0.03)
    st = bm.State.from_scenario(s)
    o = oracle.Oracle(s)
    st.step(100)
    o.step(100)
    st.track(0.2)
    o.track(0.2)
    st.step(200)
    o.step(200)
    g = compare_fp64(st, o, max_dt=0.1)
    assert g["tau_max"].max() > 0
    t0 = o.tracking["t_arrival"]
    assert np.nanmin(t0) > 0  # the record began mid-run


def test_lake_at_rest_fp32_record_is_the_initial_state():
    """FP32-bulk lake at rest (datum 400 m): the record keeps the initial depth bitwise
    (the tile's cells are copied through or their depth is unchanged), no motion."""
    s = W.fractal_lake(nx=200, ny=100, Lx=400.0, Ly=200.0, seed=41)
    st = bm.State.from_scenario(s, precision="fp32")
    st.track(0.01)
    g0 = st.download_track()
    st.step(500)
    g = st.download_track()
    for k in ("t_arrival", "h_max"):
        assert np.array_equal(g[k], g0[k], equal_nan=True)
    assert not g["u_max"].any() and not g["q_max"].any() and not g["tau_max"].any()


def test_floodplain_fp32_within_its_accuracy():
    s = W.floodplain(nx=160, ny=64, Lx=1600.0, Ly=640.0, seed=23, q_peak=150.0, ramp=120.0)
    st = bm.State.from_scenario(s, precision="fp32")
    o = oracle.Oracle(s)
    st.track(0.05)
    o.track(0.05)
    st.run_until(200.0)
    o.run_until(200.0)
    g, r = st.download_track(), o.tracking
    area = o.area()
    assert np.sum(area * np.abs(g["h_max"] - r["h_max"])) / area.sum() <= 1e-4
    assert rel_linf(g["q_max"], r["q_max"]) <= 1e-3
    ga, ra = g["t_arrival"], r["t_arrival"]
    same_state = np.isnan(ga) == np.isnan(ra)
    assert same_state.mean() >= 0.999
    both_set = ~np.isnan(ga) & ~np.isnan(ra)
    assert np.mean(np.abs(ga[both_set] - ra[both_set]) <= 1.0) >= 0.99


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_record_equals_solo(precision):
    scs = [W.dam_break(manning=0.02), W.floodplain(nx=90, ny=33, Lx=900.0, Ly=330.0, seed=51, q_peak=120.0,
                                                    ramp=60.0)]
    solo = [bm.State.from_scenario(s, precision=precision) for s in scs]
    members = [bm.State.from_scenario(s, precision=precision) for s in scs]
    for st in solo + members:
        st.track(0.05)
    for st in solo:
        st.step(80)
    b = bm.Batch(members)
    b.step(80)
    for x, y in zip(solo, members):
        gx, gy = x.download_track(), y.download_track()
        for k in gx:
            assert np.array_equal(gx[k], gy[k], equal_nan=True), k


def test_download_without_tracking_is_an_error():
    st = bm.State.from_scenario(W.dam_break(nx=10, ny=2))
    with pytest.raises(bm.BMError, match="tracking is off"):
        st.download_track()
    with pytest.raises(bm.BMError, match="h_arrival"):
        st.track(-1.0)
