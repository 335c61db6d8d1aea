"""Quad double arithmetic of the oracle against exact rational arithmetic,
and quad double path tracking (Section 5, Table 2: the solver in quad double,
"quality up") against the double tracker and exact residuals."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from workloads import configs, cyclic, rng_for, unit_gamma, univariate
from tests._checks import exact_residual_parts, same_set

U4 = 2.0 ** -200  # a margin above the 2^-212 of four doubles


def _rand_qd(rng):
    """Four doubles of decreasing magnitude, each below the last bit of the
    one before (the sum is known exactly as a rational)."""
    v = float(rng.normal() * 10.0 ** rng.integers(-5, 5))
    out = [v]
    for _ in range(3):
        v = float(v * 2.0 ** -54 * rng.normal())
        out.append(v)
    return np.array(out)


def _exact(x):
    return sum(Fraction(float(v)) for v in x)


@pytest.mark.parametrize("op", ["qd_add", "qd_mul", "qd_div"])
def test_qd_ops_relative_error(op):
    rng = rng_for(700)
    worst = 0.0
    for _ in range(400):
        a, b = _rand_qd(rng), _rand_qd(rng)
        if op == "qd_add" and rng.random() < 0.5:
            b = -a * (1 + 2.0 ** -30)  # cancellation of the leading bits
            b[1:] = rng.normal(size=3) * abs(a[0]) * 2.0 ** -80
        fa, fb = _exact(a), _exact(b)
        exact = {"qd_add": fa + fb, "qd_mul": fa * fb, "qd_div": fa / fb}[op]
        got_parts = oracle.qd_op(op, a, b)
        got = _exact(got_parts)
        scale = abs(fa) + abs(fb) if op == "qd_add" else abs(exact)
        worst = max(worst, float(abs(got - exact) / scale))
        for k in range(3):  # decreasing, non-overlapping parts
            assert abs(got_parts[k + 1]) <= abs(got_parts[k]) * 2.0 ** -50 or got_parts[k + 1] == 0.0
    assert worst <= U4, worst


def test_qd_tracker_dense4_reaches_quad_double_accuracy():
    """The whole path in quad double: the double tracker's 16 regular
    endpoints (1e-10) with the same step counts, each endpoint a root of f to
    1e-58 in exact rational arithmetic."""
    w = configs.dense4()
    s, g = w.systems[0], w.gammas[0]
    h = oracle.total_degree(s, g)
    xq, c, st = oracle.track_qd(h, threads=4)
    x, c2, st2 = oracle.track(h, threads=1)
    assert np.all(c == oracle.REGULAR) and np.all(c2 == oracle.REGULAR)
    ok, err = same_set(xq[:, :, 0], x, 1e-10)
    assert ok, err
    assert np.array_equal(st["n_accept"] + st["n_reject"], st2["n_accept"] + st2["n_reject"])
    for p in range(16):
        assert exact_residual_parts(s, xq[p]) <= 1e-58


def test_qd_tracker_univariate_roots_and_double_double_agreement():
    """A degree 6 polynomial: the quad double endpoints are its companion
    eigenvalues (1e-12), roots to 1e-58 exactly, and agree with the double
    double tracker's endpoints to its accuracy (1e-28)."""
    rng = rng_for(701)
    c = rng.normal(size=7) + 1j * rng.normal(size=7)
    s = univariate(c)
    h = oracle.total_degree(s, unit_gamma(rng))
    xq, cls, st = oracle.track_qd(h, threads=4)
    assert np.all(cls == oracle.REGULAR)
    ok, err = same_set(xq[:, :, 0], np.roots(c[::-1])[:, None], 1e-12)
    assert ok, err
    xh, xl, cd, _ = oracle.track_dd(h, threads=4)
    for p in range(6):
        assert exact_residual_parts(s, xq[p]) <= 1e-58
        dd_val = complex(xh[p, 0]) + complex(xl[p, 0])
        q_val = sum(complex(v) for v in xq[p, 0])
        assert abs(dd_val - q_val) <= 1e-28 * (1 + abs(q_val))


def test_qd_tracker_cyclic5_classes_equal_double():
    h5 = oracle.total_degree(cyclic(5), unit_gamma(rng_for(702)))
    xq, cls, st = oracle.track_qd(h5)
    x, c2, _ = oracle.track(h5)
    assert np.array_equal(np.bincount(cls, minlength=4), np.bincount(c2, minlength=4))
    ok, err = same_set(xq[cls == 0][:, :, 0], x[c2 == 0], 1e-10)
    assert ok, err
    for p in np.where(cls == 0)[0][:5]:
        assert exact_residual_parts(cyclic(5), xq[p]) <= 1e-58
