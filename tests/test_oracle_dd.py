"""Double double arithmetic of the oracle against exact rational arithmetic,
and double double Newton refinement against an exact residual."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from workloads import configs, rng_for
from tests._checks import exact_residual

U2 = 2.0 ** -104  # double double unit roundoff, u^2 with u = 2^-53


def _rand_doubles(rng, k):
    return [float(v) for v in rng.normal(size=k) * 10.0 ** rng.integers(-20, 20, size=k)]


def _rand_dd(rng):
    hi = float(rng.normal() * 10.0 ** rng.integers(-5, 5))
    lo = float(hi * 2.0 ** -60 * rng.normal())
    s = hi + lo
    return (s, (hi - s) + lo)


def test_two_sum_and_two_prod_are_exact():
    rng = rng_for(70)
    a_s, b_s = _rand_doubles(rng, 500), _rand_doubles(rng, 500)
    for a, b in zip(a_s, b_s):
        hi, lo = oracle.dd_op("two_sum", a, b)
        assert hi == a + b
        assert Fraction(hi) + Fraction(lo) == Fraction(a) + Fraction(b)
        hi, lo = oracle.dd_op("two_prod", a, b)
        assert hi == a * b
        assert Fraction(hi) + Fraction(lo) == Fraction(a) * Fraction(b)


@pytest.mark.parametrize("op", ["dd_add", "dd_mul", "dd_div"])
def test_dd_ops_relative_error(op):
    rng = rng_for(71)
    worst = 0.0
    for _ in range(500):
        a, b = _rand_dd(rng), _rand_dd(rng)
        if op == "dd_add" and rng.random() < 0.5:
            b = (-a[0] * (1 + 1e-9), -a[1])  # cancellation
        fa = Fraction(a[0]) + Fraction(a[1])
        fb = Fraction(b[0]) + Fraction(b[1])
        exact = {"dd_add": fa + fb, "dd_mul": fa * fb, "dd_div": fa / fb}[op]
        hi, lo = oracle.dd_op(op, a, b)
        got = Fraction(hi) + Fraction(lo)
        scale = abs(fa) + abs(fb) if op == "dd_add" else abs(exact)
        worst = max(worst, float(abs(got - exact) / scale))
        assert abs(lo) <= abs(hi) * 2.0 ** -52
    assert worst <= 8 * U2, worst


def test_refinement_reaches_double_double_accuracy():
    """Refined regular endpoints of the dense n = 4 system satisfy f to about
    1e-28 when f is evaluated exactly at x_hi + x_lo."""
    w = configs.dense4()
    sys = w.systems[0]
    h = oracle.total_degree(sys, w.gammas[0])
    x, cls, st = oracle.track(h, threads=1)
    xh, xl, cls2, cond = oracle.refine(h, x, cls, st["cond"], st["stop"] == 0, cond_threshold=0.0)
    assert np.all(cls2 == oracle.REGULAR)
    assert np.any(xl != 0)
    for p in range(4):
        before = exact_residual(sys, x[p], np.zeros_like(x[p]))
        after = exact_residual(sys, xh[p], xl[p])
        assert after <= 1e-28, (p, before, after)
