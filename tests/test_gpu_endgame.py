"""The Cauchy endgame on the GPU (phc_endgame through the C ABI) against the
oracle's: per path the same cycle number, and where there is an estimate
the same point within 1e-10; the double root, triple root and Example 4.1
cases of tests/test_oracle_endgame.py, a regular system and a batch handle."""
import numpy as np
import pytest

import oracle
import paper_1804_03807_gb300 as P
from workloads import configs, membership_example, rng_for, unit_gamma, univariate

pytestmark = pytest.mark.gpu
R, Q = 0.3 + 0.7j, -1.2 + 0.4j


def _poly(roots):
    c = np.array([1.0 + 0j])
    for z in roots:
        c = np.polymul(c, [1, -z])
    return univariate(c[::-1])


def _compare(sys, gamma):
    h = P.phc_make_homotopy(sys, gamma)
    r, cyc = P.endgame(h)
    xg, cg = r.x.cpu().numpy().T, cyc.cpu().numpy()
    xo, co, _ = oracle.endgame(oracle.total_degree(sys, gamma))
    assert np.array_equal(cg, co), (cg, co)
    ok = co > 0
    if ok.any():
        d = np.max(np.abs(xg[ok] - xo[ok]), axis=1) / (1 + np.max(np.abs(xo[ok]), axis=1))
        assert d.max() <= 1e-10, d.max()
    return xg, cg


def test_endgame_singular_roots_and_example_4_1():
    g = unit_gamma(rng_for(61))
    for mult in (2, 3):
        xg, cg = _compare(_poly([R] * mult + [Q]), g)
        assert sorted(cg.tolist()) == [1] + [mult] * mult
        assert np.abs(xg[cg == mult, 0] - R).max() <= 1e-12
    xg, cg = _compare(membership_example(), unit_gamma(rng_for(62)))
    assert (cg == 2).sum() == 2 and np.abs(xg[cg == 2] - np.array([2, 0])).max() <= 1e-12


def test_endgame_regular_system_and_batch_handle():
    w = configs.dense4()
    xg, cg = _compare(w.systems[0], w.gammas[0])
    assert np.all(cg == 1)
    wb = configs.cyclic_batch(4, 1, seed=805)
    hb = P.phc_make_homotopy_batch(wb.systems, wb.gammas)
    r, cyc = P.endgame(hb)
    Pn = wb.systems[0].bezout()
    for s_i, (s, g) in enumerate(zip(wb.systems, wb.gammas)):
        xo, co, _ = oracle.endgame(oracle.total_degree(s, g))
        assert np.array_equal(cyc.cpu().numpy()[s_i * Pn:(s_i + 1) * Pn], co)
