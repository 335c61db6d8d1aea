"""Pin of the oracle's endpoint measures (condition number and relative
residual) against a computation from their definitions with numpy.

At t = 1 the homotopy is the target system, so with J = f_x(x) (the
Jacobian from the definition of f, not the oracle's evaluator),
s_i = 1 + scale_i (scale_i: the sum over the terms of equation i of
|c|_1 |x^a|_1) and ||x|| = max_j max(|Re x_j|, |Im x_j|):
  cond   = max_j sum_i |(J^-1)_ji|_1 s_i / (1 + ||x||)
  relres = max_i |f_i(x)|_1 / s_i.
J^-1 comes from numpy's inverse (LAPACK), so a transposed accumulation, a
dropped scale or a wrong norm in the oracle would show here.
"""
import numpy as np
import pytest

import oracle
from workloads import PolySystem, cyclic, embedding_constants, random_dense, rng_for, univariate, unit_gamma
from tests._checks import eval_system, jacobian, term_scales


def reference(sys, x):
    J = jacobian(sys, x)
    s = 1.0 + term_scales(sys, x)
    Ji = np.linalg.inv(J)
    a1 = np.abs(Ji.real) + np.abs(Ji.imag)
    nx = np.max(np.maximum(np.abs(x.real), np.abs(x.imag)))
    cond = np.max(a1 @ s) / (1.0 + nx)
    f = eval_system(sys, x)[0]
    relres = np.max((np.abs(f.real) + np.abs(f.imag)) / s)
    return cond, relres


def _points(n, rng, k=4):
    return [(rng.normal(size=n) + 1j * rng.normal(size=n)) * rng.uniform(0.3, 3.0) for _ in range(k)]


@pytest.mark.parametrize("sys", [random_dense(3, 3, rng_for(11)), cyclic(5), random_dense(4, 2, rng_for(12))])
def test_end_measures_total_degree_homotopy(sys):
    h = oracle.total_degree(sys, unit_gamma(rng_for(13)))
    for x in _points(sys.n_var, rng_for(14)):
        c, r = oracle.end_measures(h, x)
        cr, rr = reference(sys, x)
        assert abs(c - cr) <= 1e-10 * cr
        assert abs(r - rr) <= 1e-12 * max(rr, 1e-300) + 1e-300


def test_end_measures_parameter_homotopy_uses_the_target():
    sys = random_dense(3, 2, rng_for(15))
    rng = rng_for(16)
    c0 = rng.normal(size=sys.n_terms) + 1j * rng.normal(size=sys.n_terms)
    h = oracle.parameter_homotopy(sys, c0, unit_gamma(rng))
    for x in _points(3, rng):
        c, r = oracle.end_measures(h, x)
        cr, rr = reference(sys, x)
        assert abs(c - cr) <= 1e-10 * cr and abs(r - rr) <= 1e-12 * rr


def test_end_measures_cascade_homotopy_drops_the_scaled_hyperplane():
    """At t = 1 the cascade homotopy E_k -> E_{k-1} has hyperplane k reduced
    to its slack term z_k."""
    base = cyclic(4)
    rng = rng_for(17)
    g, hy = embedding_constants(rng, 4, 4, 1)
    E = oracle.embed(base, 1, g, hy)
    h = oracle.cascade_homotopy(E, 4, 4, 1)
    # E with the last equation reduced to z_1
    tpe = np.array(E.terms_per_eq).copy()
    keep = np.ones(E.n_terms, bool)
    last = int(np.sum(tpe[:-1]))
    for q in range(last, E.n_terms):
        e = E.exps[q]
        keep[q] = e[4] == 1 and e[:4].sum() == 0
    tpe[-1] = int(keep[last:].sum())
    R = PolySystem(E.n_eq, E.n_var, tpe, E.exps[keep], E.coefs[keep], name="E1-at-t1")
    for x in _points(5, rng):
        c, r = oracle.end_measures(h, x)
        cr, rr = reference(R, x)
        assert abs(c - cr) <= 1e-10 * cr and abs(r - rr) <= 1e-12 * rr


def test_end_measures_near_a_double_root():
    """(x - 1)(x - 1 - e)(x + 2): at the root x = 1 the condition number
    grows like 1/e (here the closed form |3|/|e * 3| up to the scales)."""
    for e in (1e-3, 1e-6):
        coefs = np.polymul(np.polymul([1, -1], [1, -1 - e]), [1, 2])[::-1]
        sys = univariate(coefs)
        h = oracle.total_degree(sys, 1.0)
        x = np.array([1.0 + 0j])
        c, r = oracle.end_measures(h, x)
        cr, rr = reference(sys, x)
        assert abs(c - cr) <= 1e-9 * cr
        # f'(1) = -3 e, so |J^-1|_1 = 1 / (3 e); s = 1 + sum |c|
        s = 1.0 + np.sum(np.abs(coefs.real) + np.abs(coefs.imag))
        assert abs(c - s / (3 * e) / 2.0) <= 1e-6 * c
