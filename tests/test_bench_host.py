"""Host-side arithmetic of bench.py's whole-run rate (no GPU)."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def test_step_weighted_is_the_trapezoid_over_the_run_steps():
    import bench
    snaps = [{"steps": 0}, {"steps": 100}, {"steps": 400}]
    steps, total = bench.step_weighted(snaps, [1.0, 3.0, 5.0])
    assert steps == 400
    # 100 steps at a mean of 2 ms, 300 at a mean of 4 ms
    assert total == pytest.approx(100 * 2.0 + 300 * 4.0)


def test_step_weighted_single_window_is_that_window():
    import bench
    steps, total = bench.step_weighted([{"steps": 7}], [0.25])
    assert (steps, total) == (1, 0.25)


def test_constant_time_per_step_gives_that_rate():
    import bench
    snaps = [{"steps": s} for s in (0, 15829, 50333, 104566)]
    steps, total = bench.step_weighted(snaps, [0.3] * 4)
    assert total / steps == pytest.approx(0.3)
