"""Batches: many uneven meshes stepped by one launch per step, each with its own dt.

Each member of a batch must end bitwise equal to the same state stepped alone (the
per-instance arithmetic and reduction order do not depend on the batch), for any
launch shape; run_until stops each member exactly at its own end time.
"""
import numpy as np
import pytest

import oracle
from paper_2102_12862_b300 import bm
from paper_2102_12862_b300 import workloads as W
from tests.test_parity_gpu import compare

pytestmark = pytest.mark.gpu


def scenarios():
    return [
        W.dam_break(),
        W.floodplain(nx=90, ny=33, Lx=900.0, Ly=330.0, seed=51, q_peak=120.0, ramp=60.0),
        W.random_state(W.dam_break(nx=37, ny=5, seed=52), seed=52),
        W.fractal_lake(nx=30, ny=17, Lx=300.0, Ly=170.0, seed=53),
        W.three_humps(nx=40, ny=16),
    ]


def states_for(scs, precision):
    # the random state (index 2) needs the positivity time step; the others keep their own
    return [bm.State.from_scenario(s, precision=precision, **({"cfl_mode": 1} if i == 2 else {}))
            for i, s in enumerate(scs)]


def equal_states(a, b):
    for x, y in zip(a.download(), b.download()):
        if not np.array_equal(np.asarray(x), np.asarray(y)):
            return False
    return True


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("ctas_per_sm", [0, 2])
def test_batch_equals_solo_bitwise(precision, ctas_per_sm):
    scs = scenarios()
    solo = states_for(scs, precision)
    batched = states_for(scs, precision)
    for s in solo:
        s.set_launch(ctas_per_sm)
        s.step(60)
    b = bm.Batch(batched)
    b.set_launch(ctas_per_sm)
    b.step(60)
    for k, (x, y) in enumerate(zip(solo, batched)):
        assert x.stats()["steps"] == y.stats()["steps"] == 60
        assert equal_states(x, y), f"member {k} differs from its solo run"


def test_batch_run_until_per_member_end_times():
    scs = scenarios()
    sts = states_for(scs, "fp64")
    b = bm.Batch(sts)
    t_end = np.array([3.0, 40.0, 0.5, 7.0, 2.0])
    b.run_until(t_end)
    for k, st in enumerate(sts):
        assert st.stats()["t"] == t_end[k]
    # members against the oracle, element by element on h = H - z, hu and hv (the
    # free surface sits ~400 m above the datum on the floodplain member, so H itself
    # would hide depth errors)
    for k in (1, 2, 4):
        o = oracle.Oracle(scs[k], **({"cfl_mode": 1} if k == 2 else {}))
        o.run_until(t_end[k])
        compare(scs[k], sts[k], o)
        assert sts[k].stats()["steps"] == o.steps
    # run_until listed only the running members towards the end; plain steps take
    # every member again
    before = [st.stats()["steps"] for st in sts]
    b.step(3)
    assert [st.stats()["steps"] for st in sts] == [n + 3 for n in before]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_launch_shape_does_not_change_results(precision):
    # 1,407 tiles: 1, 3 and 4 CTAs per SM give different static ticket assignments and
    # counter shares (and the default one more); the results are bitwise equal
    s = W.floodplain(nx=600, ny=300, Lx=3000.0, Ly=1500.0, seed=54, q_peak=300.0, ramp=30.0)
    ref = bm.State.from_scenario(s, precision=precision)
    ref.step(40)
    for shape in (1, 3, 4):
        b = bm.State.from_scenario(s, precision=precision)
        b.set_launch(shape)
        b.step(40)
        assert equal_states(ref, b), f"{shape} CTAs per SM"
        b.close()


def test_batch_rejects_mixed_precision_and_duplicates():
    s = W.dam_break(nx=10, ny=2)
    x = bm.State.from_scenario(s)
    y = bm.State.from_scenario(s, precision="fp32")
    with pytest.raises(bm.BMError, match="precision"):
        bm.Batch([x, y])
    with pytest.raises(bm.BMError, match="twice"):
        bm.Batch([x, x])


def test_fp32_batch_members_against_the_oracle():
    """FP32-bulk members of a batch against the FP64 oracle at the FP32-bulk bars: L1
    depth error <= 1e-4 m, relative mass defect (volume against initial volume plus
    boundary volume) <= 1e-7, and each member's time exactly its end time."""
    scs = [W.floodplain(nx=90, ny=33, Lx=900.0, Ly=330.0, seed=51, q_peak=120.0, ramp=60.0),
           W.dam_break(), W.three_humps(nx=40, ny=16)]
    sts = [bm.State.from_scenario(s, precision="fp32") for s in scs]
    v0 = [st.stats()["volume"] for st in sts]
    t_end = np.array([60.0, 8.0, 5.0])
    bm.Batch(sts).run_until(t_end)
    for k, (s, st) in enumerate(zip(scs, sts)):
        o = oracle.Oracle(s)
        o.run_until(t_end[k])
        H, qx, qy, t = st.download()
        assert t == t_end[k]
        area = o.area()
        l1 = float(np.sum(area * np.abs((H - s.z) - o.depth())) / area.sum())
        assert l1 <= 1e-4, (k, l1)
        stt = st.stats()
        defect = abs(stt["volume"] - v0[k] - stt["boundary_volume"]) / (v0[k] + abs(stt["boundary_volume"]))
        assert defect <= 1e-7, (k, defect)


def featured(precision):
    """Members with every optional feature, each on its own floodplain: two passive
    species under rain on a disk, rain on a disk (an external source), a log-law friction closure with flood
    tracking, and (FP64) bed evolution; plus a plain member."""
    scs = [W.floodplain(nx=100, ny=40, Lx=1000.0, Ly=400.0, seed=61 + k, q_peak=90.0, ramp=40.0) for k in range(5)]
    sts = [bm.State.from_scenario(s, precision=precision) for s in scs]
    hc = np.stack([np.maximum(scs[0].H - scs[0].z, 0.0) * 0.5, np.zeros(scs[0].n_cells)])
    sts[0].set_scalars(hc, [0.0, 1.0])
    # the species member also takes rain (species together with sources)
    sts[0].set_sources(W.disk_region(scs[0], 600.0, 200.0, 80.0), [bm.SOURCE_INTENSITY], [bm.SINK_EXACT],
                       [(np.array([0.0, 1e6]), np.array([90.0, 90.0]))])
    sts[1].set_sources(W.disk_region(scs[1], 700.0, 120.0, 60.0), [bm.SOURCE_INTENSITY], [bm.SINK_EXACT],
                       [(np.array([0.0, 1e6]), np.array([150.0, 150.0]))])
    sts[2].set_friction(bm.FRICTION_CHEZY, 25.0)
    sts[2].track(0.05)
    if precision == "fp64":
        sts[3].set_morpho(porosity=0.4, s=2.65, d=0.001)
    return scs, sts


def featured_pair(precision):
    return featured(precision)[1], featured(precision)[1]


def same_everything(a, b, precision, k):
    assert equal_states(a, b), k
    if k == 0:
        assert np.array_equal(a.download_scalars(), b.download_scalars())
    if k == 2:
        ta, tb = a.download_track(), b.download_track()
        for key in ta:
            assert np.array_equal(np.asarray(ta[key]), np.asarray(tb[key]), equal_nan=True), key
    if k == 3 and precision == "fp64":
        assert np.array_equal(a.download_bed(), b.download_bed())


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_with_every_feature_equals_solo(precision):
    """Members with species, sources, a log-law closure with tracking and bed evolution
    step in one batch: each ends bitwise equal to its solo run, for plain stepping and
    for run_until with per-member end times (the run's later launches list only the
    members still running, and the finished members' species and beds stay put)."""
    solo, inb = featured_pair(precision)
    b = bm.Batch(inb)
    for st in solo:
        st.step(40)
    b.step(40)
    for k, (x, y) in enumerate(zip(inb, solo)):
        same_everything(x, y, precision, k)
    ends = [30.0, 12.0, 25.0, 8.0, 40.0]
    for st, t in zip(solo, ends):
        st.run_until(t)
    b.run_until(ends)
    for k, (x, y) in enumerate(zip(inb, solo)):
        assert x.stats()["t"] == ends[k]
        same_everything(x, y, precision, k)


def test_batch_refuses_a_member_changed_after_it_was_made():
    s = W.floodplain(nx=60, ny=24, Lx=600.0, Ly=240.0, seed=66)
    a, c = bm.State.from_scenario(s), bm.State.from_scenario(s)
    b = bm.Batch([a, c])
    b.step(2)
    a.set_friction(bm.FRICTION_CHEZY, 30.0)
    with pytest.raises(bm.BMError, match="changed after bm_batch_create"):
        b.step(1)
    b2 = bm.Batch([a, c])  # made again: steps
    b2.step(2)
