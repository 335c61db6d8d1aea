"""Pins of the oracle's Cauchy endgame against closed forms and Example 4.1.

* (x - r)^2 (x - q): the two paths that meet the double root r go around
  t = 1 as a 2-cycle (c = 2) and the mean of their loop samples is r to
  1e-12, where the double precision tracker stops at about 1e-8; the simple
  root q has c = 1.  (x - r)^3 (x - q): c = 3.
* Example 4.1: (x1 - 1)(x1 - 2), (x1 - 1) x2^2 has the double isolated point
  (2, 0) ("which occurs with multiplicity two"): two paths reach it with
  c = 2; the paths to the line x1 = 1 have c = 1; a path that runs to
  infinity closes around a pole and gets no estimate (c = 0).
* A regular system (dense n = 4, degree 2): c = 1 on every path, the
  estimates are the tracker's regular endpoints.
"""
import json
import os

import numpy as np

import oracle
from workloads import configs, membership_example, rng_for, unit_gamma, univariate
from tests._checks import relative_residual, same_set

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_examples.json")))
R, Q = 0.3 + 0.7j, -1.2 + 0.4j


def _poly(roots):
    c = np.array([1.0 + 0j])
    for z in roots:
        c = np.polymul(c, [1, -z])
    return univariate(c[::-1])


def test_double_and_triple_roots():
    g = unit_gamma(rng_for(61))
    for mult in (2, 3):
        s = _poly([R] * mult + [Q])
        h = oracle.total_degree(s, g)
        x, cyc, st = oracle.endgame(h)
        at_r = np.abs(x[:, 0] - R) < 1e-6
        assert at_r.sum() == mult and np.all(cyc[at_r] == mult)
        assert np.abs(x[at_r, 0] - R).max() <= 1e-12
        assert np.all(cyc[~at_r] == 1) and np.abs(x[~at_r, 0] - Q).max() <= 1e-12
        xt, ct, _ = oracle.track(h, threads=1)
        assert np.abs(xt[at_r, 0] - R).max() > 1e-10  # the tracker alone is far less accurate there


def test_example_4_1_double_point():
    gold = GOLDEN["example_4_1_membership"]
    s = membership_example()
    h = oracle.total_degree(s, unit_gamma(rng_for(62)))
    x, cyc, st = oracle.endgame(h)
    at_p = np.max(np.abs(x - np.array(gold["test_point"])), axis=1) < 1e-6
    assert at_p.sum() == gold["point_multiplicity"] and np.all(cyc[at_p] == 2)
    assert np.max(np.abs(x[at_p] - np.array(gold["test_point"]))) <= 1e-12
    on_line = (cyc > 0) & ~at_p
    assert np.all(cyc[on_line] == 1) and np.abs(x[on_line, 0] - 1).max() <= 1e-12
    assert (cyc == 0).sum() >= 1 and np.all(st["relres"][cyc == 0] > 1e-10)


def test_regular_system_has_cycle_one():
    w = configs.dense4()
    s, g = w.systems[0], w.gammas[0]
    h = oracle.total_degree(s, g)
    x, cyc, _ = oracle.endgame(h)
    xt, ct, _ = oracle.track(h, threads=1)
    assert np.all(cyc == 1) and np.all(ct == oracle.REGULAR)
    ok, err = same_set(x, xt, 1e-10)
    assert ok, err
    assert relative_residual(s, x).max() <= 1e-12
