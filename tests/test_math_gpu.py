"""The FP64 step's hand-written elementary functions against CUDA's own and against
numpy: 1/x by Newton-Raphson refinement of the hardware reciprocal estimate, x^(-1/3)
by Newton-Raphson refinement of a single-precision estimate (and x^(1/3) = x r^2),
and the FP32-bulk step's x^(-1/3) from the hardware base-2 logarithm and exponent."""
import numpy as np
import pytest

from paper_2102_12862_b300 import bm

pytestmark = pytest.mark.gpu


def _inputs(lo, hi, n=1 << 20, seed=5):
    rng = np.random.default_rng(seed)
    x = np.exp(rng.uniform(np.log(lo), np.log(hi), n))
    edges = np.array([lo, hi, 1.0, 2.0, 0.5, 3.0, 1e-6, 1e-3, 9.81, 1.0 + 2.0 ** -52, 2.0 - 2.0 ** -51])
    return np.concatenate([x, edges[(edges >= lo) & (edges <= hi)]])


def _ulps(a, ref):
    return np.abs(a - ref) / np.spacing(np.abs(ref))


def test_reciprocal_within_two_ulp():
    # the step divides by depths above h_min, wave-speed spans, 1 + 2a (>= 1) and
    # hydraulic depths: normal doubles of either sign
    x = _inputs(1e-12, 1e12)
    x = np.concatenate([x, -x[:1000]])
    ours = bm.bm_math_eval("rcp", x)
    lib = bm.bm_math_eval("rcp_lib", x)
    assert np.array_equal(lib, 1.0 / x)  # CUDA's division is the correctly rounded one
    assert _ulps(ours, lib).max() <= 2.0


def _rcbrt_ref(x):
    """x^(-1/3) rounded from extended precision."""
    return (1 / np.cbrt(x.astype(np.longdouble))).astype(np.float64)


def test_rcbrt_and_cbrt_fp64():
    x = _inputs(1e-30, 1e30)
    ref = _rcbrt_ref(x)
    lib = bm.bm_math_eval("rcbrt_lib", x)
    ours = bm.bm_math_eval("rcbrt", x)
    assert _ulps(lib, ref).max() <= 2.0
    assert _ulps(ours, ref).max() <= 3.0
    cref = np.cbrt(x.astype(np.longdouble)).astype(np.float64)
    assert _ulps(bm.bm_math_eval("cbrt_lib", x), cref).max() <= 1.0
    # x r^2 carries twice r's relative error plus two roundings: at most 2 * 3 + 2 ulp
    assert _ulps(bm.bm_math_eval("cbrt", x), cref).max() <= 8.0
    # outside the estimate's range the library is used
    far = np.array([1e-300, 1e-40, 1e40, 1e300])
    assert np.array_equal(bm.bm_math_eval("rcbrt", far), bm.bm_math_eval("rcbrt_lib", far))


def test_rcbrt_fp32_within_its_error_bound():
    # FP32-bulk evaluates x^(-1/3) of depths (m) in float: 2^(-log2(x)/3) from the
    # hardware approximations, against the library's rcbrtf (1 ulp) and the exact value
    x = _inputs(1e-6, 1e6).astype(np.float32).astype(np.float64)
    ref = _rcbrt_ref(x)
    eps32 = 2.0 ** -23
    lib = bm.bm_math_eval("rcbrt32_lib", x)
    ours = bm.bm_math_eval("rcbrt32", x)
    assert np.max(np.abs(lib - ref) / ref) <= 2 * eps32
    assert np.max(np.abs(ours - ref) / ref) <= 16 * eps32
