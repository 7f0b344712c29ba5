"""The double-float (FP32X2) arithmetic on the device, by the scalar sequence
and by the packed-FP32-pair form the contraction kernels' merge loops run on
sm_100 and later, against exact rational dot products of the same
double-word operands.

Each operand x is stored as hi + lo (hi = fl32(x), lo = fl32(x - hi)); a
product is formed exactly as a double word (FMA error term plus both cross
terms; the lo*lo term, below 2^-48 relative, is dropped), added by TwoSum
into the high word with the errors gathered in the low word.  First-order
bound for K terms: |err| <= (K + 4) 2^-46 sum_k |a_k b_k|.
"""
from fractions import Fraction

import numpy as np
import pytest

from paper_2010_14962_gb300 import qtn

pytestmark = pytest.mark.gpu


def _dw(v):
    hi = np.float32(v)
    lo = np.float32(v - np.float64(hi))
    return Fraction(float(hi)) + Fraction(float(lo))


def _exact(a, b):
    re = im = Fraction(0)
    mag = 0.0
    for x, y in zip(a, b):
        xr, xi, yr, yi = _dw(x.real), _dw(x.imag), _dw(y.real), _dw(y.imag)
        re += xr * yr - xi * yi
        im += xr * yi + xi * yr
        mag += abs(x) * abs(y)
    return complex(float(re), float(im)), mag


@pytest.mark.parametrize("K", [2, 4, 32])
def test_double_float_dot_products(gpu, K):
    rng = np.random.default_rng(K)
    count = 96
    scale = rng.choice([1.0, 1e3, 1e-3], size=(count, K))
    a = (rng.normal(size=(count, K)) + 1j * rng.normal(size=(count, K))) * scale
    b = rng.normal(size=(count, K)) + 1j * rng.normal(size=(count, K))
    # a third of the items nearly cancel: b chosen so consecutive products cancel
    for i in range(0, count, 3):
        b[i, 1:] = -a[i, :-1] * b[i, :-1] / a[i, 1:] * (1 + 1e-7 * rng.normal(size=K - 1))
    s, m, packed = qtn.arith_check(a, b)
    print("packed pairs:", packed)
    worst_s = worst_m = 0.0
    for i in range(count):
        ref, mag = _exact(a[i], b[i])
        bound = (K + 4) * 2.0 ** -46 * mag
        worst_s = max(worst_s, abs(s[i] - ref) / mag)
        worst_m = max(worst_m, abs(m[i] - ref) / mag)
        assert abs(s[i] - ref) <= bound, (i, "scalar")
        assert abs(m[i] - ref) <= bound, (i, "merge loops")
    print(f"K={K}: worst |err| / sum|a b|: scalar {worst_s:.2e}, merge loops {worst_m:.2e}")
