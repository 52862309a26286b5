"""The optional modules together on one state (flood tracking, external sources, bed
evolution, passive species) against the oracle stepping the same modules, and the
autotuner's trials undone for all of them.

Bars as for each module alone: FP64 state, bed change and tracking maxima within
relative L-inf 1e-11 (|u| and the shear stress 100 times that), species within the
state's bar.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2102_12862_b300 import bm
from paper_2102_12862_b300 import workloads as W

pytestmark = pytest.mark.gpu
SAND = dict(porosity=0.4, s=2.65, d=0.001, alpha=8.0, m=1.5, theta_cr=0.047)


def rel_linf(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def test_tracking_sources_and_bed_together_fp64():
    """A wet dam break with friction over sand, rain on a disk and flood tracking, 300
    steps: state, bed and tracking record against the oracle with the same modules.
    (On a dry floodplain fed by a flood the erodible bed amplifies rounding by orders
    of magnitude within a few hundred steps -- depths just above h_min at the front
    give the bedload, which grows like |u|^3, runaway values -- so the modules are
    checked together where the water covers the bed.)"""
    s = W.dam_break(nx=150, ny=12, manning=0.03, seed=9)
    reg = W.disk_region(s, 70.0, 5.0, 4.0)
    series = [(np.array([0.0, 5.0]), np.array([0.0, 3600.0]))]
    st = bm.State.from_scenario(s)
    o = oracle.Oracle(s)
    for x in (st, o):
        x.set_sources(reg, [bm.SOURCE_INTENSITY], [bm.SINK_EXACT], series)
        x.set_morpho(**SAND)
        x.track(0.2)
    st.step(300)
    o.step(300)
    tol = 1e-11
    z = st.download_bed()
    H, qx, qy, t = st.download()
    assert abs(t - o.time) <= 1e-12 * o.time
    errs = {name: rel_linf(a, b) for name, a, b in (("bed change", z - s.z, o.z - s.z), ("h", H - z, o.H - o.z),
                                                      ("hu", qx, o.qx), ("hv", qy, o.qy))}
    assert all(e <= tol for e in errs.values()), errs
    g, r = st.download_track(), o.tracking
    for k in ("h_max", "q_max"):
        assert rel_linf(g[k], r[k]) <= tol, k
    for k in ("u_max", "tau_max"):
        assert rel_linf(g[k], r[k]) <= 100 * tol, k
    assert np.max(np.abs(z - s.z)) > 1e-6
    assert np.max(g["h_max"][reg == 0] - (s.H - s.z)[reg == 0]) > 0


def test_species_with_bed_evolution_fp64():
    """A dam break with friction over sand carrying two species: the species kernel
    reads z^n before the bed moves; q_c, the bed and the state match the oracle."""
    s = W.dam_break(nx=150, ny=12, manning=0.03, seed=6)
    h0 = np.maximum(s.H - s.z, 0.0)
    x = s.centroids()[:, 0]
    hc = np.stack([np.where(x < 50, 0.8, 0.1) * h0, 0.3 * h0])
    st = bm.State.from_scenario(s)
    o = oracle.Oracle(s)
    for y in (st, o):
        y.set_scalars(hc)
        y.set_morpho(**SAND)
    st.step(300)
    o.step(300)
    g = st.download_scalars()
    for c in range(2):
        assert rel_linf(g[c], o.hc[c]) <= 1e-11
    z = st.download_bed()
    assert rel_linf(z - s.z, o.z - s.z) <= 1e-11
    assert np.max(np.abs(z - s.z)) > 1e-6


def test_autotune_undoes_its_trials_for_every_module():
    """The autotuner's trial steps are undone (state, tracking record, species, bed): a
    tuned state continues bitwise like an untuned one (results do not depend on the
    launch shape)."""
    s = W.dam_break(nx=120, ny=10, manning=0.03, seed=8)
    h0 = np.maximum(s.H - s.z, 0.0)
    runs = []
    for tune in (False, True):
        st = bm.State.from_scenario(s)
        st.set_scalars(0.5 * h0[None, :])
        st.track(0.05)
        st.set_morpho(**SAND)
        st.step(20)
        if tune:
            st.autotune(steps_per_trial=5)
        st.step(40)
        runs.append((st.download(), st.download_scalars(), st.download_track(), st.download_bed()))
    (a, ac, at, az), (b, bc, bt, bz) = runs
    for x, y in zip(a, b):
        assert np.array_equal(np.asarray(x), np.asarray(y))
    assert np.array_equal(ac, bc) and np.array_equal(az, bz)
    for k in at:
        assert np.array_equal(at[k], bt[k], equal_nan=True)
