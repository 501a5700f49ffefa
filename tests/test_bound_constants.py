"""The constants of the FP32 entropy decision's error bounds that follow
from the series of Delta H (host-side arithmetic, no GPU).

Delta H(alpha) = sum_{k>=2} c_k(alpha) M_k, c_k(alpha) = (-1)^k (alpha^k -
k alpha) / (k (k-1)), M_k = sum_i f_i x_i^k.  An error dx in every x_i moves
the computed k-th term by at most k |c_k| f |x|^(k-1) |dx|, so the bounds
need, for |x| <= 1/8 (the FP32 paths' limit):
  * Delta H(2): sum_{k>=3} k |c_k(2)| |x|^(k-3) <= 1 + 4 |x|;
  * Delta H(1): sum_{k>=2} k |c_k(1)| |x|^(k-1) = |x| / (1 - |x|);
and the chord test relies on c_2(2) = 0.
"""
import math

import numpy as np


def c(k, alpha):
    return (-1) ** k * (alpha ** k - k * alpha) / (k * (k - 1))


def test_c2_at_alpha_two_vanishes():
    assert c(2, 2.0) == 0.0


def test_first_order_factor_of_delta_h2():
    for x in np.linspace(0.0, 0.125, 257):
        s = sum(k * abs(c(k, 2.0)) * x ** (k - 3) for k in range(3, 400))
        assert s <= 1.0 + 4.0 * x, (x, s)
    # the factor is tight to within 4 % at the limit
    s = sum(k * abs(c(k, 2.0)) * 0.125 ** (k - 3) for k in range(3, 400))
    assert 1.44 < s < 1.45


def test_first_order_factor_of_delta_h1():
    for x in np.linspace(0.0, 0.125, 257):
        s = sum(k * abs(c(k, 1.0)) * x ** (k - 1) for k in range(2, 400))
        assert math.isclose(s, x / (1.0 - x), rel_tol=1e-12, abs_tol=1e-300)
