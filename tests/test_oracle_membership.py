"""Pins of the oracle's homotopy membership test and the filters of
Section 4 against what the paper fixes.

* Example 4.1: the system (x1 - 1)(x1 - 2), (x1 - 1) x2^2 has the line
  x1 = 1 and the double point (2, 0).  The line has degree 1, so its
  embedding for dimension 1 has one generic point; moving the hyperplane
  through (2, 0) carries it to a point of the line, not to (2, 0); moved
  through a point of the line, it lands on that point.
* Example 4.2 (Figures 4 and 5): the cascade of Example 3.1 filtered from
  the top down leaves the witness sets of one 3-dimensional set of degree 1
  (x1 = 1), one 2-dimensional set of degree 1 (x1 = 2, x2 = 1) and twelve
  lines (degree 12), and exactly the four isolated points (3,2,2,1),
  (3,3,2,1), (4,3,2,1), (4,2,2,1): every singular candidate lies on a
  higher-dimensional set.  The number of paths of a filter stage is the
  number of points tested times the degree of the set (Corollary 4.3's
  proof: n_k d_k paths).
"""
import json
import os

import numpy as np
import pytest

import oracle
from workloads import embedding_constants, membership_example, multistep_example, rng_for, unit_gamma
from tests._checks import same_set

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_examples.json")))


def _solve_embedded(sys, D, seed):
    rng = rng_for(seed)
    g, hy = embedding_constants(rng, sys.n_eq, sys.n_var, D)
    E = oracle.embed(sys, D, g, hy)
    h = oracle.total_degree(E, unit_gamma(rng))
    x, c, st = oracle.track(h, threads=1)
    x, _, c, _ = oracle.refine(h, x, c, st["cond"], st["stop"] == 0)
    return E, x, c


@pytest.mark.parametrize("seed", [71, 72])
def test_example_4_1_membership(seed):
    sys = membership_example()
    E, x, c = _solve_embedded(sys, 1, seed)
    gold = GOLDEN["example_4_1_membership"]
    W = x[(c == oracle.REGULAR) & oracle.slack_zero(x, 2)]
    assert len(W) == gold["line_degree"]  # the line x1 = 1 has degree 1
    assert abs(W[0, 0] - 1) <= 1e-10
    pts = np.array([gold["test_point"], [1, 5], [1, 0.3 - 2j]], dtype=complex)
    on, ends = oracle.membership(E, 2, 1, W, pts)
    assert on.tolist() == [gold["on_line"], True, True]  # (2, 0) is not on the line (Example 4.1)
    for z, (xe, ce) in zip(pts[1:], ends[1:]):
        assert np.max(np.abs(xe[0] - np.concatenate([z, [0]]))) <= 1e-10 * (1 + np.abs(z).max())
    # moved through (2, 0): the generic point stays on the line, on the moved hyperplane
    xe, ce = ends[0]
    assert ce[0] == oracle.REGULAR and abs(xe[0, 0] - 1) <= 1e-10 and abs(xe[0, 2]) <= 1e-10


def _cascade_levels(seed):
    """Endpoints of the top stage and of every cascade stage of Example 3.1
    (refined), as levels {k: (E_k, x, cls)}."""
    sys = multistep_example()
    n, D = 4, 3
    E, x, c = _solve_embedded(sys, D, seed)
    levels = {D: (E, x, c)}
    X = x[(c == oracle.REGULAR) & ~oracle.slack_zero(x, n + D - 1)]
    for k in range(D, 0, -1):
        Enext, xk, ck, st = oracle.cascade_stage(E, n, n, k, X, threads=1)
        hk = oracle.total_degree(Enext, 1.0)
        xk, _, ck, _ = oracle.refine(hk, xk, ck, st["cond"], st["stop"] == 0)
        levels[k - 1] = (Enext, xk, ck)
        if k > 1:
            X = xk[(ck == oracle.REGULAR) & ~oracle.slack_zero(xk, n + k - 2)]
        E = Enext
    return levels


@pytest.mark.parametrize("seed", [41, 42])
def test_example_4_2_filter(seed):
    gold = GOLDEN["example_3_1_cascade"]
    gold_f = GOLDEN["example_4_2_filter"]
    levels = _cascade_levels(seed)
    witness, isolated, stages = oracle.filter_candidates(levels, 4)
    # degrees of the 3-, 2- and 1-dimensional sets: 1, 1, 12
    assert {str(k): len(w) for k, w in witness.items()} == gold_f["witness_degrees"]
    assert len(isolated) == gold_f["isolated_regular"]
    ok, err = same_set(isolated, np.array(gold["isolated_points"], dtype=complex), 1e-10)
    assert ok, err
    # every stage tracks (points tested) x (degree) paths
    deg = {3: 1, 2: 1, 1: 12}
    for level, dim, paths, removed in stages:
        assert paths % deg[dim] == 0 and removed <= paths // deg[dim]
    print("filter stages (level, dimension, paths, removed):", stages)
