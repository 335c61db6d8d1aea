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


# ------------------------------------------------------------ double double path tracking (Section 5, Table 2)

def test_dd_tracker_dense4_reaches_double_double_accuracy():
    """The whole path in double double: the same 16 regular endpoints as the
    double tracker (1e-10), with the same step counts (the readings are the
    same), and each endpoint x_hi + x_lo a root of f to 1e-28 in exact
    rational arithmetic."""
    from workloads import configs
    from tests._checks import exact_residual, same_set
    w = configs.dense4()
    s, g = w.systems[0], w.gammas[0]
    h = oracle.total_degree(s, g)
    xh, xl, c, st = oracle.track_dd(h, threads=1)
    x, c2, st2 = oracle.track(h, threads=1)
    assert np.all(c == oracle.REGULAR) and np.all(c2 == oracle.REGULAR)
    ok, err = same_set(xh, x, 1e-10)
    assert ok, err
    assert np.array_equal(st["n_accept"] + st["n_reject"], st2["n_accept"] + st2["n_reject"])
    for p in range(16):
        assert exact_residual(s, xh[p], xl[p]) <= 1e-28


def test_dd_tracker_univariate_and_cyclic5():
    """A degree 6 polynomial: the double double endpoints are its companion
    matrix eigenvalues (1e-12) and roots to 1e-28 exactly; cyclic 5: the
    double tracker's classes and regular set, every regular endpoint a root
    to 1e-28."""
    from workloads import cyclic, rng_for, unit_gamma, univariate
    from tests._checks import exact_residual, same_set
    rng = rng_for(91)
    c = rng.normal(size=7) + 1j * rng.normal(size=7)
    s = univariate(c)
    h = oracle.total_degree(s, unit_gamma(rng))
    xh, xl, cls, st = oracle.track_dd(h, threads=1)
    assert np.all(cls == oracle.REGULAR)
    comp = np.roots(c[::-1])
    ok, err = same_set(xh, comp[:, None], 1e-12)
    assert ok, err
    for p in range(6):
        assert exact_residual(s, xh[p], xl[p]) <= 1e-28
    s5 = cyclic(5)
    h5 = oracle.total_degree(s5, unit_gamma(rng_for(92)))
    xh, xl, cls, st = oracle.track_dd(h5)
    x, c2, _ = oracle.track(h5)
    assert np.array_equal(np.bincount(cls, minlength=4), np.bincount(c2, minlength=4))
    ok, err = same_set(xh[cls == 0], x[c2 == 0], 1e-10)
    assert ok, err
    reg = np.where(cls == 0)[0]
    for p in reg[:10]:
        assert exact_residual(s5, xh[p], xl[p]) <= 1e-28
