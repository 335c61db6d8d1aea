"""Pins of the oracle's polyhedral homotopies (Section 2.2): mixed cells,
mixed volumes, the binomial start systems and the tracked paths.

What fixes the answers, independently of the oracle's own code:
* closed forms: a dense system's mixed volume is its Bezout number; one
  equation in one unknown of degree d has mixed volume d;
* the paper: the top dimensional system of Example 3.1 (three slack
  variables) has mixed volume 61 (tests/golden/paper_examples.json);
* Bernstein's count by another method: a system with coefficients in general
  position has as many isolated roots in (C*)^n as its mixed volume, and the
  oracle's total-degree homotopy counts them independently;
* invariance: the mixed volume does not depend on the lifting;
* brute force: every choice of two points per support checked exactly must
  give the cells the pruned search gives;
* the binomial solutions solve their binomial systems, |det D| of them,
  pairwise distinct; the polyhedral paths end at the roots the total-degree
  homotopy finds.
"""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import mixed as M
from workloads import (PolySystem, cyclic, embedding_constants, multistep_example, random_dense, random_lifting,
                       rng_for, unit_gamma, with_random_coefficients)
from tests._checks import match_sets, min_pair_distance, relative_residual

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_examples.json")))


def _mv(sys, seed):
    return M.mixed_volume(M.mixed_cells(sys, random_lifting(rng_for(seed), sys.n_terms)))


def _tiny_sparse(rng, n, terms):
    """n equations in n unknowns, each with `terms` distinct random monomials
    of degree <= 2 (the constant term included)."""
    from itertools import product
    mons = [e for e in product(range(3), repeat=n) if sum(e) <= 2]
    exps, tpe = [], []
    for _ in range(n):
        pick = [0] + list(rng.choice(np.arange(1, len(mons)), size=terms - 1, replace=False))
        exps.extend(mons[k] for k in pick)
        tpe.append(terms)
    return PolySystem(n, n, np.array(tpe), np.array(exps, dtype=np.uint8),
                      rng.standard_normal(len(exps)) + 1j * rng.standard_normal(len(exps)), name="tiny")


@pytest.mark.parametrize("n,deg", [(1, 5), (2, 3), (3, 2)])
def test_mixed_volume_of_a_dense_system_is_its_bezout_number(n, deg):
    sys = random_dense(n, deg, rng_for(300 + n))
    assert _mv(sys, 301) == deg ** n


def test_mixed_volume_of_example_3_1_top_system_is_the_papers_61():
    g = GOLDEN["example_3_1_top_mixed_volume"]
    rng = rng_for(310)
    gammas, hyper = embedding_constants(rng, 4, 4, g["top_dim"])
    E = oracle.embed(multistep_example(), g["top_dim"], gammas, hyper)
    assert _mv(E, 311) == g["mixed_volume"]


@pytest.mark.parametrize("n", [4, 5])
def test_mixed_volume_counts_the_roots_the_total_degree_homotopy_finds(n):
    """Random coefficients on the cyclic n-roots supports: the total-degree
    homotopy's regular endpoints number the mixed volume (16 and 70)."""
    g = with_random_coefficients(cyclic(n), rng_for(320 + n))
    h = oracle.total_degree(g, unit_gamma(rng_for(321)))
    _, cls, _ = oracle.track(h)
    assert _mv(g, 322) == int(np.sum(cls == 0)) == {4: 16, 5: 70}[n]


def test_mixed_volume_does_not_depend_on_the_lifting():
    g = with_random_coefficients(cyclic(5), rng_for(330))
    a = M.mixed_cells(g, random_lifting(rng_for(331), g.n_terms))
    b = M.mixed_cells(g, random_lifting(rng_for(332), g.n_terms))
    assert {c.pairs for c in a} != {c.pairs for c in b}  # other subdivisions
    assert M.mixed_volume(a) == M.mixed_volume(b) == 70


@pytest.mark.parametrize("seed", [340, 341, 342])
def test_pruned_search_finds_exactly_the_cells_of_brute_force(seed):
    rng = rng_for(seed)
    sys = _tiny_sparse(rng, 2 + seed % 2, 4)
    lift = random_lifting(rng, sys.n_terms)
    assert M.mixed_cells(sys, lift) == M.mixed_cells_brute(sys, lift)
    g = cyclic(4)
    lift = random_lifting(rng_for(seed + 10), g.n_terms)
    assert M.mixed_cells(g, lift) == M.mixed_cells_brute(g, lift)


def test_a_tie_on_a_lower_facet_is_reported():
    """Lifting zero puts every point of a support at the same level."""
    g = cyclic(3)
    with pytest.raises(ValueError, match="general position"):
        M.mixed_cells_brute(g, np.zeros(g.n_terms, dtype=np.int32))


def test_cell_powers_vanish_on_the_cell_and_are_at_least_one_elsewhere():
    g = with_random_coefficients(cyclic(5), rng_for(350))
    lift = random_lifting(rng_for(351), g.n_terms)
    for cell in M.mixed_cells(g, lift):
        p = M.cell_powers(g, lift, cell)
        on = np.zeros(g.n_terms, bool)
        on[[t for pr in cell.pairs for t in pr]] = True
        assert np.all(p[on] == 0.0)
        assert np.all(p[~on] >= 1.0) and p[~on].min() == 1.0


def test_binomial_start_solutions_solve_their_binomial_systems():
    g = with_random_coefficients(cyclic(5), rng_for(360))
    lift = random_lifting(rng_for(361), g.n_terms)
    for cell in M.mixed_cells(g, lift):
        Y = M.binomial_starts(g, cell)
        assert Y.shape[0] == cell.volume
        assert min_pair_distance(Y) > 1e-6
        for (a, b) in cell.pairs:
            ea, eb = g.exps[a].astype(int), g.exps[b].astype(int)
            ta = g.coefs[a] * np.prod(Y ** ea, axis=1)
            tb = g.coefs[b] * np.prod(Y ** eb, axis=1)
            assert np.max(np.abs(ta + tb) / (np.abs(ta) + np.abs(tb))) < 1e-12


@pytest.mark.parametrize("n", [4, 5])
def test_polyhedral_paths_end_at_the_roots_of_the_total_degree_homotopy(n):
    g = with_random_coefficients(cyclic(n), rng_for(370 + n))
    lift = random_lifting(rng_for(371), g.n_terms)
    starts, x, cls, stats, cell_of = M.track_polyhedral(g, lift)
    assert np.all(cls == 0)  # no polyhedral path diverges
    assert np.max(relative_residual(g, x)) < 1e-12
    h = oracle.total_degree(g, unit_gamma(rng_for(372)))
    xt, ct, _ = oracle.track(h)
    reg = xt[ct == 0]
    assert reg.shape[0] == x.shape[0]
    _, _, r = match_sets(x, reg)
    assert r.max() < 1e-9


def test_polyhedral_divergence_bound_is_relative_to_the_start():
    """Section 2.2 fixes no divergence bound.  A polyhedral path starts at a
    binomial solution in its cell's scaled coordinates, which may lie beyond
    diverge_norm (1e6) without the path diverging, so its bound is diverge_norm
    x max(1, ||y(0)||); the other homotopies keep diverge_norm.  y - 1e7 with
    both terms on the cell (no power of t) is a path that stays at its start
    1e7: it reaches t = 1 in the 18 steps of a path whose steps are all
    accepted and ends beyond the endpoint bound (at infinity).  The
    total-degree path of the same equation from x - 1 grows from 1 to 1e7 and
    stops when it passes 1e6."""
    s = PolySystem(1, 1, np.array([2]), np.array([[1], [0]], dtype=np.uint8), np.array([1.0, -1e7]))
    x, cls, st = oracle.track(oracle.polyhedral_homotopy(s, np.array([0.0, 0.0])), starts=np.array([[1e7]]),
                              threads=1)
    assert st["stop"][0] == 0 and st["t"][0] == 1.0 and st["n_accept"][0] == 18
    assert cls[0] == 2 and x[0, 0] == 1e7
    x, cls, st = oracle.track(oracle.total_degree(s, unit_gamma(rng_for(480))), threads=1)
    assert st["stop"][0] == 1 and st["t"][0] < 1.0 and cls[0] == 2
    assert 1e6 < abs(x[0, 0]) < 1e7
