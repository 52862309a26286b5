"""Autotuner: picks a launch shape by timing trial steps, then restores the state,
so tuning does not change what the run computes."""
import numpy as np
import pytest

from paper_2102_12862_b300 import bm
from paper_2102_12862_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_autotune_restores_state(precision):
    s = W.floodplain(nx=240, ny=96, Lx=2400.0, Ly=960.0, seed=71)
    a = bm.State.from_scenario(s, precision=precision)
    b = bm.State.from_scenario(s, precision=precision)
    a.step(7)
    b.step(7)
    best, ms = a.autotune(5)
    assert best in (0, 1, 2, 3, 4, 6, 8) and ms > 0
    assert a.stats()["steps"] == 7
    a.step(11)
    b.step(11)
    for x, y in zip(a.download(), b.download()):
        assert np.array_equal(np.asarray(x), np.asarray(y))


def test_batch_autotune_keeps_end_times():
    scs = [W.ensemble_instance(k, size_override=n) for k, n in enumerate([2000, 7000, 4000])]
    sts = [bm.State.from_scenario(s, precision="fp32") for s in scs]
    b = bm.Batch(sts)
    best, ms = b.autotune(4)
    assert best in (0, 1, 2, 3, 4, 6, 8)
    b.run_until([5.0, 9.0, 3.0])
    assert [st.stats()["t"] for st in sts] == [5.0, 9.0, 3.0]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_schedule_does_not_change_results(precision):
    """Every launch shape and static share of the tickets gives bitwise the same run
    (the reductions are order-free), also after changing it mid-run."""
    s = W.floodplain(nx=200, ny=80, Lx=2000.0, Ly=800.0, seed=72)
    ref = bm.State.from_scenario(s, precision=precision)
    ref.step(60)
    R = ref.download()
    for ctas, s16 in [(0, 0), (1, 16), (2, 6), (0, 12)]:
        st = bm.State.from_scenario(s, precision=precision)
        st.set_schedule(ctas, s16)
        assert st.schedule() == (ctas, s16)
        st.step(30)
        st.set_schedule(1, -1)
        st.step(30)
        for x, y in zip(st.download(), R):
            assert np.array_equal(np.asarray(x), np.asarray(y))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_tile_slots_do_not_change_results(precision):
    """2, 3 and 4 tile slots (the plain step is built for each) give bitwise the same
    run, also when the count changes mid-run, alone and in a batch; a state with an
    optional feature runs 3 whatever was asked."""
    s = W.floodplain(nx=200, ny=80, Lx=2000.0, Ly=800.0, seed=74)
    ref = bm.State.from_scenario(s, precision=precision)
    ref.step(60)
    R = ref.download()
    for k in (2, 4, 3):
        st = bm.State.from_scenario(s, precision=precision)
        st.set_slots(k)
        assert st.slots() == k
        st.step(30)
        st.set_slots(2 if k != 2 else 4)
        st.step(30)
        for x, y in zip(st.download(), R):
            assert np.array_equal(np.asarray(x), np.asarray(y))
    a = bm.State.from_scenario(s, precision=precision)
    other = bm.State.from_scenario(W.floodplain(nx=90, ny=33, Lx=900.0, Ly=330.0, seed=75), precision=precision)
    b = bm.Batch([a, other])
    b.set_slots(4)
    assert b.slots() == 4
    b.step(60)
    for x, y in zip(a.download(), R):
        assert np.array_equal(np.asarray(x), np.asarray(y))
    t = bm.State.from_scenario(s, precision=precision)
    t.set_slots(2)
    t.track(0.05)
    assert t.slots() == 3
    for bad in (1, 5):
        with pytest.raises(bm.BMError):
            t.set_slots(bad)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_claiming_mode_does_not_change_results(precision):
    """Claiming items ahead (mode 0), right after an issue (mode 1) or once their slot is
    free (mode 2), with each slot count and static share, alone and in a batch, changed
    mid-run: bitwise the same run."""
    s = W.floodplain(nx=200, ny=80, Lx=2000.0, Ly=800.0, seed=76)
    ref = bm.State.from_scenario(s, precision=precision)
    assert ref.claim() == (3 if precision == "fp64" else 2) and ref.slots() == 2
    ref.step(60)
    R = ref.download()
    for mode, k, s16 in [(0, 3, -1), (0, 2, 0), (1, 4, 16), (1, 3, 0), (2, 2, -1), (2, 3, 16), (3, 2, -1), (3, 4, 0)]:
        st = bm.State.from_scenario(s, precision=precision)
        st.set_claim(mode)
        st.set_slots(k)
        st.set_schedule(0, s16)
        assert st.claim() == mode
        st.step(25)
        st.set_claim((mode + 1) % 4)
        st.step(35)
        for x, y in zip(st.download(), R):
            assert np.array_equal(np.asarray(x), np.asarray(y))
    a = bm.State.from_scenario(s, precision=precision)
    other = bm.State.from_scenario(W.floodplain(nx=90, ny=33, Lx=900.0, Ly=330.0, seed=77), precision=precision)
    b = bm.Batch([a, other])
    b.set_claim(2)
    assert b.claim() == 2
    b.step(60)
    for x, y in zip(a.download(), R):
        assert np.array_equal(np.asarray(x), np.asarray(y))
    for bad in (-2, 4):
        with pytest.raises(bm.BMError):
            a.set_claim(bad)


def test_set_schedule_rejects_bad_share():
    s = W.dam_break()
    st = bm.State.from_scenario(s)
    for bad in (-2, 17):
        with pytest.raises(bm.BMError):
            st.set_schedule(0, bad)


def _ms_per_step(st, n=200, reps=3):
    import torch
    stream = torch.cuda.Stream()
    st.set_stream(stream.cuda_stream)
    best = float("inf")
    for _ in range(reps):
        st.step(3)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st.step_async(n)
        e1.record(stream)
        torch.cuda.synchronize()
        st.sync()
        best = min(best, e0.elapsed_time(e1) / n)
    return best


@pytest.mark.parametrize("workload,precision", [("floodplain", "fp32"), ("lake", "fp64")])
def test_tuned_schedule_is_at_least_as_fast_as_the_default(workload, precision):
    """On two workloads (a 500,000-cell floodplain in FP32-bulk, a 250,000-cell wet lake
    in FP64) the autotuner's schedule steps at least as fast as the default (best of 3
    windows of 200 steps each; 5 % for timing noise)."""
    if workload == "floodplain":
        s = W.floodplain(nx=800, ny=312, Lx=5000.0, Ly=2000.0, seed=73)
    else:
        s = W.fractal_lake(nx=500, ny=250)
    tuned = bm.State.from_scenario(s, precision=precision)
    best, ms = tuned.autotune(20)
    ctas, s16 = tuned.schedule()
    assert best == ctas and -1 <= s16 <= 16 and tuned.slots() in (2, 3, 4) and tuned.claim() in (0, 1, 2, 3)
    default = bm.State.from_scenario(s, precision=precision)
    t_def, t_tun = _ms_per_step(default), _ms_per_step(tuned)
    assert t_tun <= 1.05 * t_def, (t_tun, t_def, (ctas, s16, tuned.slots(), tuned.claim()))
    # the tuned run (its trial steps undone) computes bitwise what the default run does
    for x, y in zip(tuned.download(), default.download()):
        assert np.array_equal(np.asarray(x), np.asarray(y))
