"""FP32-bulk precision mode: state, bed and geometry as FP32 offsets from an FP64
datum; thresholds through FP32 differences that are exact near the threshold;
time, dt and mass accumulators in FP64.

Gates (against the FP64 oracle on the same inputs): L1 depth error <= 1e-4 m,
lake at rest preserved (|u|, |v| <= 1e-6 m/s; here bitwise 0), relative mass
defect <= 1e-7.  Every test also records L-inf errors of h and velocity.
"""
import numpy as np
import pytest

import oracle
from paper_2102_12862_b300 import bm
from paper_2102_12862_b300 import workloads as W

pytestmark = pytest.mark.gpu


def errors(s, st, o):
    H, qx, qy, t = st.download()
    area = o.area()
    h, ho = H - s.z, o.H - s.z
    l1 = float(np.sum(area * np.abs(h - ho)) / area.sum())
    linf = float(np.max(np.abs(h - ho)))
    wet = (ho > 1e-3) & (h > 1e-3)
    du = np.abs(qx[wet] / h[wet] - o.qx[wet] / ho[wet]) if wet.any() else np.zeros(1)
    dv = np.abs(qy[wet] / h[wet] - o.qy[wet] / ho[wet]) if wet.any() else np.zeros(1)
    return {"l1_h": l1, "linf_h": linf, "l1_vel": float(np.mean(np.hypot(du, dv))),
            "linf_vel": float(max(du.max(), dv.max())), "t": t, "t_oracle": o.time}


def test_dam_break_fp32_vs_oracle():
    s = W.dam_break()
    st = bm.State.from_scenario(s, precision="fp32")
    o = oracle.Oracle(s)
    st.run_until(20.0)
    o.run_until(20.0)
    e = errors(s, st, o)
    assert e["t"] == 20.0
    assert e["l1_h"] <= 1e-4, e
    assert e["linf_h"] <= 5e-3, e


def test_floodplain_fp32_vs_oracle_and_mass():
    s = W.floodplain(nx=160, ny=64, Lx=1600.0, Ly=640.0, seed=23, q_peak=150.0, ramp=120.0)
    st = bm.State.from_scenario(s, precision="fp32")
    o = oracle.Oracle(s)
    v0 = st.stats()["volume"]
    st.run_until(240.0)
    o.run_until(240.0)
    e = errors(s, st, o)
    assert e["l1_h"] <= 1e-4, e
    stt = st.stats()
    defect = abs(stt["volume"] - v0 - stt["boundary_volume"]) / (v0 + stt["boundary_volume"])
    assert defect <= 1e-7, defect


def test_lake_at_rest_fp32_bitwise_high_datum():
    """Beds 395-405 m (datum 400): still water at 403 m stays bitwise still in FP32-bulk
    over 100,000 steps (the C-property survives because H and z are offsets from the
    same FP64 datum and the flux cancels exactly)."""
    s = W.fractal_lake(nx=200, ny=100, Lx=400.0, Ly=200.0, seed=41)
    st = bm.State.from_scenario(s, precision="fp32", datum=400.0)
    v0 = st.stats()["volume"]
    st.step(100_000)
    H, qx, qy, t = st.download()
    assert np.max(np.abs(H - s.H)) <= 1e-6
    assert np.max(np.abs(qx)) == 0.0 and np.max(np.abs(qy)) == 0.0
    assert abs(st.stats()["volume"] - v0) / v0 <= 1e-7


def test_thacker_fp32_datum_400():
    """Moving shoreline in a paraboloid 400 m above the datum origin: FP32-bulk stays
    within 1e-4 m (L1) of the FP64 oracle over a quarter period."""
    s = W.thacker(nq=96, datum=400.0)
    st = bm.State.from_scenario(s, precision="fp32", datum=400.0)
    o = oracle.Oracle(s)
    om = np.sqrt(2 * 9.81 * 10.0) / 3000.0
    t = 0.25 * 2 * np.pi / om
    st.run_until(t)
    o.run_until(t)
    e = errors(s, st, o)
    assert e["l1_h"] <= 1e-4, e


def test_fp32_auto_datum_and_roundtrip():
    s = W.dam_break(nx=20, ny=4)
    s.z = s.z + 400.0
    s.H = s.H + 400.0
    st = bm.State.from_scenario(s, precision="fp32")  # datum NaN -> min(z) = 400
    H, qx, qy, t = st.download()
    assert np.max(np.abs(H - s.H)) <= 1e-7  # offsets 1 and 0.1 round to FP32 near 1e-8


def test_fp32_downloaded_state_uploads_again():
    """A dry cell of an FP32-bulk state downloads as the datum plus its bed's FP32
    offset, which can lie below the FP64 bed by that rounding; uploading the download
    (a checkpoint resume) is accepted, keeps every dry cell's surface exactly and the
    wet ones to the rounding of the datum-plus-pair sum (1e-12 m), and continues as
    the run that never left the device (FP32-bulk accuracy)."""
    s = W.floodplain(nx=160, ny=64, Lx=1600.0, Ly=640.0, seed=23, q_peak=150.0, ramp=120.0)
    a = bm.State.from_scenario(s, precision="fp32")
    b = bm.State.from_scenario(s, precision="fp32")
    H0 = a.download()[0]  # a dry cell: the datum plus its bed's FP32 offset
    a.step(40)
    b.step(40)
    H, qx, qy, t = a.download()
    dry = (s.H - s.z <= 0.0) & (H == H0)  # dry at t = 0 and untouched since
    assert np.any(H[dry] < s.z[dry])  # the case under test occurs on this bed
    a.upload(H, qx, qy, t)
    H2, qx2, qy2, _ = a.download()
    assert np.array_equal(H2[dry], H[dry])
    assert np.max(np.abs(H2 - H)) <= 1e-12
    assert np.array_equal(qx2, qx) and np.array_equal(qy2, qy)
    a.step(30)
    b.step(30)
    A, B = a.download(), b.download()
    assert np.max(np.abs(A[0] - B[0])) <= 1e-5
    assert A[3] == B[3] or abs(A[3] - B[3]) <= 1e-9 * B[3]
