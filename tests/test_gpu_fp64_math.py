"""The FP64 stencil's reciprocal square root (the one-sided speeds, the midpoint predictor
and |grad| of the KNP update, Sec. 3.2.3) and reciprocal (the Step 4 weights), computed on
the FP32 and integer pipes, against exact rational arithmetic: within one unit in the last
place for positive doubles from the least subnormal to the largest finite double, and the
IEEE special cases."""
import math
from fractions import Fraction

import numpy as np
import pytest

from paper_1911_03225_gb300 import binding as B

pytestmark = pytest.mark.gpu

RSQRT, RCP = 0, 1


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def samples(lo_exp, hi_exp, count, seed):
    rng = np.random.default_rng(seed)
    x = np.ldexp(rng.uniform(1.0, 2.0, count), rng.integers(lo_exp, hi_exp, count))
    return x[x > 0]


SPECIAL = [5e-324, 1e-323, 2.225073858507201e-308, 2.2250738585072014e-308, 0.25, 1.0, 2.0, 3.0, 4.0,
           float(np.nextafter(1.0, 2.0)), float(np.nextafter(1.0, 0.0)), float(np.nextafter(4.0, 0.0))]


def test_fp64_rsqrt_within_one_ulp():
    x = np.concatenate([samples(-1074, 1024, 3000, 7), SPECIAL, [np.finfo(np.float64).max]])
    y = B.debug_fp64_math(RSQRT, x)
    bad = []
    for a, b in zip(x.tolist(), y.tolist()):
        # the exact a^(-1/2) lies strictly between b - ulp(b) and b + ulp(b)
        u = Fraction(math.ulp(b))
        lo, hi, X = Fraction(b) - u, Fraction(b) + u, Fraction(a)
        if not (lo > 0 and lo * lo * X < 1 < hi * hi * X):
            bad.append((a, b))
    assert not bad, bad[:5]


def test_fp64_reciprocal_within_one_ulp():
    # |x| up to 2^1021 and down to the subnormals whose reciprocal is finite; both signs
    x = np.concatenate([samples(-1023, 1022, 3000, 8), SPECIAL[2:]])
    x = np.concatenate([x, -x[::7]])
    y = B.debug_fp64_math(RCP, x)
    bad = []
    for a, b in zip(x.tolist(), y.tolist()):
        u = Fraction(math.ulp(b))
        lo, hi, X = abs(Fraction(b)) - u, abs(Fraction(b)) + u, abs(Fraction(a))
        if not (math.copysign(1.0, a) == math.copysign(1.0, b) and lo * X < 1 < hi * X):
            bad.append((a, b))
    assert not bad, bad[:5]


def test_fp64_special_values():
    y = B.debug_fp64_math(RSQRT, np.array([np.inf, np.nan]))
    assert y[0] == 0.0 and np.isnan(y[1])
    big = np.finfo(np.float64).max
    r = B.debug_fp64_math(RCP, np.array([np.inf, -np.inf, np.nan, 0.0, 5e-324, big, -big]))
    assert r[0] == 0.0 and r[1] == 0.0 and math.copysign(1.0, r[1]) < 0 and np.isnan(r[2])
    assert r[3] == np.inf and r[4] == np.inf
    np.testing.assert_array_equal(r[5:], 1.0 / np.array([big, -big]))   # subnormal results


def test_fp64_math_rejects_bad_arguments():
    with pytest.raises(B.FDMError) as e:
        B.debug_fp64_math(2, np.ones(4))
    assert e.value.status == B.FDM_ERR_INVALID_ARG
