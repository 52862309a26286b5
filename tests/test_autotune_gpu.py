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
