"""Pins of the oracle's coefficient-parameter homotopy (Section 2.3: the
solutions of a random coefficient system start the paths to the target
system), and the root count of the random-coefficient copies of cyclic 7.

The copies of cyclic 7 with random coefficients keep its supports, so for
generic coefficients they have as many isolated roots as the first copy
(the root count of a generic member of a family of systems with fixed
supports is the same for every generic member).  Two of the eight copies of
the benchmark batch give 917 regular endpoints under the total-degree
homotopy instead of 924.  Continuation from the 924 roots of the first copy
reaches 924 distinct regular roots of each of them; the 7 the total-degree
homotopy misses form one orbit of x -> w x (w^7 = 1) of norm about 114.
At such a root the start system's term (1-t) gamma (x_i^{d_i} - 1) is of
size (1-t) 114^7 ~ 2e14 (1-t), so the total-degree path reaches it only
when 1 - t is near 1e-14, the resolution of t in double precision: those
paths stall there (h < h_min) while still moving and are counted at
infinity.  The library tracks the same readings and finds the same 917.
"""
import numpy as np
import pytest

import oracle
from workloads import configs, random_dense, rng_for, unit_gamma
from tests._checks import match_sets, min_pair_distance, relative_residual, same_set

RTOL = 1e-10


def _regular(sys, gamma):
    h = oracle.total_degree(sys, gamma)
    x, c, st = oracle.track(h)
    return x[c == 0], np.bincount(c, minlength=4)


def test_parameter_homotopy_between_equal_systems_keeps_every_root():
    """With g = f the homotopy is ((1-t) gamma + t) f, which vanishes at the
    roots of f for every t: each path stays at its start."""
    sys = random_dense(3, 2, rng_for(20))
    R, cnt = _regular(sys, unit_gamma(rng_for(21)))
    assert cnt[0] == 8
    h = oracle.parameter_homotopy(sys, sys.coefs, unit_gamma(rng_for(22)))
    x, c, st = oracle.track(h, starts=R, threads=1)
    assert np.all(c == 0)
    assert np.max(np.abs(x - R)) <= 1e-12 * (1 + np.abs(R).max())


def test_parameter_homotopy_reaches_the_total_degree_roots():
    """From the 924 roots of one random cyclic 7 copy to another: the same
    regular set as the total-degree homotopy of the target finds."""
    w = configs.cyclic7_batch()
    R1, cnt1 = _regular(w.systems[1], w.gammas[1])
    R2, cnt2 = _regular(w.systems[2], w.gammas[2])
    assert cnt1[0] == cnt2[0] == 924
    h = oracle.parameter_homotopy(w.systems[2], w.systems[1].coefs, unit_gamma(rng_for(23)))
    x, c, st = oracle.track(h, starts=R1)
    assert np.bincount(c, minlength=4)[0] == 924
    ok, err = same_set(x[c == 0], R2, RTOL)
    assert ok, err


@pytest.mark.parametrize("copy", [7, 8])
def test_random_cyclic7_copies_have_924_roots(copy):
    """Copies 7 and 8 of the batch: 924 distinct regular roots by
    continuation from copy 1, a superset of the 917 the total-degree
    homotopy reaches; the 7 others are one orbit of x -> w x of norm > 100."""
    w = configs.cyclic7_batch()
    R1, cnt1 = _regular(w.systems[1], w.gammas[1])
    s = w.systems[copy]
    Rt, cnt = _regular(s, w.gammas[copy])
    assert cnt1[0] == 924 and cnt[0] == 917
    h = oracle.parameter_homotopy(s, w.systems[1].coefs, unit_gamma(rng_for(24)))
    x, c, st = oracle.track(h, starts=R1)
    R = x[c == 0]
    assert len(R) == 924
    assert relative_residual(s, R).max() <= 1e-12
    assert min_pair_distance(R) > 1e-6
    ra, rb, rel = match_sets(Rt, R)
    assert len(ra) == 917 and rel.max() <= RTOL
    extra = np.setdiff1d(np.arange(924), rb)
    X = R[extra]
    assert len(X) == 7 and np.all(np.abs(X).max(axis=1) > 100)
    w7 = np.exp(2j * np.pi / 7)
    ok, err = same_set(X, X[0][None, :] * w7 ** np.arange(7)[:, None], 1e-9)
    assert ok, err


@pytest.mark.parametrize("copy", [1, 7])
def test_gamma_invariance_random_cyclic7_copies(copy):
    """The regular endpoint set of a random copy does not depend on gamma."""
    w = configs.cyclic7_batch()
    s = w.systems[copy]
    Ra, ca = _regular(s, w.gammas[copy])
    Rb, cb = _regular(s, unit_gamma(rng_for(25)))
    assert np.array_equal(ca, cb)
    ok, err = same_set(Ra, Rb, RTOL)
    assert ok, err
