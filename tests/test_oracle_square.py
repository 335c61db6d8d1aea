"""Pins of the squaring of Section 2.1 (oracle.square, then the oracle's
tracker) against closed forms.

* Underdetermined: the sphere x1^2 + x2^2 + x3^2 = 1 cut by two random
  hyperplanes is a line meeting a quadric: two points, the roots of the
  quadratic (d.d) s^2 + 2 (p.d) s + (p.p - 1) = 0 along the line p + s d.
* Overdetermined: x1 = 1, x2 = 2, x1 x2 = 2 with one new unknown s and
  multipliers l_i: the square system has the solution (1, 2, 0) and one
  more, s = (l2 + 2 l1 - l3) / (l1 l2), x1 = 1 - l1 s, x2 = 2 - l2 s.
"""
import numpy as np

import oracle
from workloads import PolySystem, rng_for, unit_gamma
from tests._checks import same_set


def test_underdetermined_sphere_meets_a_line_twice():
    rng = rng_for(82)
    sphere = PolySystem(1, 3, np.array([4]), np.array([[2, 0, 0], [0, 2, 0], [0, 0, 2], [0, 0, 0]], np.uint8),
                        np.array([1, 1, 1, -1], complex), name="sphere")
    c = rng.normal(size=(2, 4)) + 1j * rng.normal(size=(2, 4))
    S = oracle.square(sphere, c)
    x, cls, st = oracle.track(oracle.total_degree(S, unit_gamma(rng)), threads=1)
    assert np.bincount(cls, minlength=4)[0] == 2
    # the line: A x = -b with A = c[:, 1:], b = c[:, 0]
    A, b = c[:, 1:], c[:, 0]
    p = np.linalg.lstsq(A, -b, rcond=None)[0]
    d = np.cross(A[0], A[1])  # A d = 0 (bilinear cross product)
    roots = np.roots([d @ d, 2 * (p @ d), p @ p - 1])
    expect = np.array([p + s * d for s in roots])
    ok, err = same_set(x[cls == 0], expect, 1e-10)
    assert ok, err


def test_overdetermined_gains_a_slack_unknown():
    rng = rng_for(83)
    over = PolySystem(3, 2, np.array([2, 2, 2]), np.array([[1, 0], [0, 0], [0, 1], [0, 0], [1, 1], [0, 0]], np.uint8),
                      np.array([1, -1, 1, -2, 1, -2], complex), name="over")
    lam = rng.normal(size=(3, 1)) + 1j * rng.normal(size=(3, 1))
    S = oracle.square(over, lam)
    assert (S.n_eq, S.n_var) == (3, 3)
    x, cls, st = oracle.track(oracle.total_degree(S, unit_gamma(rng)), threads=1)
    l1, l2, l3 = lam[:, 0]
    s = (l2 + 2 * l1 - l3) / (l1 * l2)
    expect = np.array([[1, 2, 0], [1 - l1 * s, 2 - l2 * s, s]])
    ok, err = same_set(x[cls == 0], expect, 1e-10)
    assert ok, err
