"""Failure detection on the GPU, in the forms that leave the device usable: a bounded
wait that runs out (a group of copies that is never issued, so its mbarrier never
completes) must end the launch with BM_ETIMEOUT after about a second, with every
issued copy retired, the state unchanged and the context usable; a re-uploaded state
then steps exactly like a fresh one.  (Non-finite results: test_parity_gpu.py.)"""
import time

import numpy as np
import pytest

from paper_2102_12862_b300 import bm
from paper_2102_12862_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_bounded_wait_runs_out_and_the_state_recovers(precision):
    s = W.dam_break(manning=0.02)
    st = bm.State.from_scenario(s, precision=precision)
    st.step(5)
    before = st.download()
    t0 = time.perf_counter()
    with pytest.raises(bm.BMError) as ei:
        st.test_timeout()
    wall = time.perf_counter() - t0
    assert ei.value.status == bm.BM_ETIMEOUT, ei.value
    assert 0.2 < wall < 30.0, wall  # the wait is bounded (about a second of SM clock)
    after = st.download()
    for x, y in zip(before, after):
        assert np.array_equal(np.asarray(x), np.asarray(y))
    assert st.stats(volume=False)["steps"] == 5
    # the status is sticky until the state is replaced
    with pytest.raises(bm.BMError) as ei:
        st.step(1)
    assert ei.value.status == bm.BM_ETIMEOUT
    st.upload(s.H, s.qx, s.qy, 0.0)
    st.step(20)
    ref = bm.State.from_scenario(s, mesh=st.mesh, precision=precision)
    ref.step(20)
    for x, y in zip(st.download(), ref.download()):
        assert np.array_equal(np.asarray(x), np.asarray(y))
