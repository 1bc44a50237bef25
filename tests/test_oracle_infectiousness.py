"""Pins for Eq. 1's infectiousness integral: the gamma density over one day.

For integer shape k the gamma CDF is the Erlang closed form
F(x) = 1 - exp(-x/theta) * sum_{m<k} (x/theta)^m / m!; for other shapes the
regularized incomplete gamma of scipy is the library routine."""
import math

import numpy as np
import pytest

import oracle
from paper_2110_04421_gb300 import workloads as W


def erlang_cdf(x, k, theta):
    if x <= 0:
        return 0.0
    y = x / theta
    return 1.0 - math.exp(-y) * sum(y**m / math.factorial(m) for m in range(k))


@pytest.mark.parametrize("k,theta", [(1, 1.0), (2, 3.0), (4, 1.25), (7, 0.8)])
def test_daily_integral_matches_erlang(k, theta):
    for t in range(1, 40):
        want = erlang_cdf(t, k, theta) - erlang_cdf(t - 1, k, theta)
        got = oracle.gamma_integral(t - 1.0, float(t), float(k), theta)
        assert abs(got - want) <= 1e-14 + 1e-12 * abs(want), (t, got, want)


@pytest.mark.parametrize("shape,scale", [(2.5, 2.0), (6.7, 0.9), (1.3, 4.0)])
def test_daily_integral_matches_incomplete_gamma(shape, scale):
    sp = pytest.importorskip("scipy.special")
    for t in range(1, 40):
        want = sp.gammainc(shape, t / scale) - sp.gammainc(shape, (t - 1) / scale)
        got = oracle.gamma_integral(t - 1.0, float(t), shape, scale)
        assert abs(got - want) <= 1e-10, (t, got, want)


def test_table_layout_and_day_zero():
    p = W.params_with(inf_shape=[4.0, 2.0, 3.0], inf_scale=[1.25, 2.0, 1.5], inf_len=30)
    g = dict(n=2, row_ptr=[np.zeros(3, np.uint32)], col=[np.zeros(0, np.uint32)])
    t64, t32 = oracle.Model(g, p).inf_table()
    assert t64.shape == (3, 30)
    assert np.all(t64[:, 0] == 0.0)               # nothing accrues before infection
    for c, (k, th) in enumerate([(4, 1.25), (2, 2.0), (3, 1.5)]):
        # telescoping: the table sums to F(L-1)
        assert abs(t64[c].sum() - erlang_cdf(29, k, th)) < 1e-13
        assert np.array_equal(t32[c], t64[c].astype(np.float32))
