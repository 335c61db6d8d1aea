"""Test-side checks that are independent of both the oracle and the GPU path:
direct polynomial evaluation from the definition, endpoint-set matching and
exact rational evaluation."""
from __future__ import annotations

from fractions import Fraction

import numpy as np
from scipy.optimize import linear_sum_assignment


def eval_system(sys, X: np.ndarray) -> np.ndarray:
    """f(x) for every row of X [P, n] from f_i = sum_t c_t prod_j x_j^a_tj."""
    X = np.atleast_2d(X)
    P = X.shape[0]
    out = np.zeros((P, sys.n_eq), np.complex128)
    off = 0
    for i in range(sys.n_eq):
        m = int(sys.terms_per_eq[i])
        a = sys.exps[off:off + m].astype(np.int64)  # [m, n]
        c = sys.coefs[off:off + m]
        mon = np.prod(X[:, None, :] ** a[None, :, :], axis=2)  # [P, m]
        out[:, i] = mon @ c
        off += m
    return out


def relative_residual(sys, X: np.ndarray) -> np.ndarray:
    """max_i |f_i(x)| / (1 + sum_t |c_t| |x^a_t|) per row."""
    X = np.atleast_2d(X)
    res = np.zeros(X.shape[0])
    off = 0
    for i in range(sys.n_eq):
        m = int(sys.terms_per_eq[i])
        a = sys.exps[off:off + m].astype(np.int64)
        c = sys.coefs[off:off + m]
        mon = np.prod(X[:, None, :] ** a[None, :, :], axis=2)
        f = mon @ c
        scale = np.abs(mon) @ np.abs(c)
        res = np.maximum(res, np.abs(f) / (1.0 + scale))
        off += m
    return res


def match_sets(A: np.ndarray, B: np.ndarray):
    """Optimal one-to-one matching of the rows of A and B (complex [P, n]) by
    distance; returns (row_a, row_b, relative distance per pair)."""
    A = np.atleast_2d(A)
    B = np.atleast_2d(B)
    if A.shape[0] == 0 or B.shape[0] == 0:
        return np.zeros(0, int), np.zeros(0, int), np.zeros(0)
    D = np.max(np.abs(A[:, None, :] - B[None, :, :]), axis=2)
    scale = 1.0 + np.maximum(np.max(np.abs(A), axis=1)[:, None], np.max(np.abs(B), axis=1)[None, :])
    R = D / scale
    ra, rb = linear_sum_assignment(R)
    return ra, rb, R[ra, rb]


def same_set(A: np.ndarray, B: np.ndarray, rtol: float) -> tuple[bool, float]:
    """True when A and B have equal size and match one-to-one within rtol."""
    if A.shape[0] != B.shape[0]:
        return False, float("inf")
    if A.shape[0] == 0:
        return True, 0.0
    _, _, r = match_sets(A, B)
    return bool(r.max() <= rtol), float(r.max())


def min_pair_distance(A: np.ndarray) -> float:
    """Smallest distance between two distinct rows (path-jumping guard)."""
    if A.shape[0] < 2:
        return float("inf")
    D = np.max(np.abs(A[:, None, :] - A[None, :, :]), axis=2)
    D[np.arange(A.shape[0]), np.arange(A.shape[0])] = np.inf
    return float(D.min())


def frac_complex(z_hi: complex, z_lo: complex = 0.0):
    return (Fraction(z_hi.real) + Fraction(z_lo.real), Fraction(z_hi.imag) + Fraction(z_lo.imag))


def _cmul(a, b):
    return (a[0] * b[0] - a[1] * b[1], a[0] * b[1] + a[1] * b[0])


def exact_residual(sys, x_hi: np.ndarray, x_lo: np.ndarray) -> float:
    """max_i |f_i(x_hi + x_lo)| / (1 + sum |c||x^a|), f evaluated exactly in
    rational arithmetic at the (exactly represented) point x_hi + x_lo."""
    xs = [frac_complex(complex(h), complex(l)) for h, l in zip(x_hi, x_lo)]
    worst = 0.0
    off = 0
    for i in range(sys.n_eq):
        m = int(sys.terms_per_eq[i])
        acc = (Fraction(0), Fraction(0))
        scale = 0.0
        for k in range(m):
            c = frac_complex(complex(sys.coefs[off + k]))
            mon = (Fraction(1), Fraction(0))
            for j, a in enumerate(sys.exps[off + k]):
                for _ in range(int(a)):
                    mon = _cmul(mon, xs[j])
            term = _cmul(c, mon)
            acc = (acc[0] + term[0], acc[1] + term[1])
            scale += abs(complex(sys.coefs[off + k])) * abs(complex(float(mon[0]), float(mon[1])))
        val = abs(complex(float(acc[0]), float(acc[1])))
        worst = max(worst, val / (1.0 + scale))
        off += m
    return worst


def jacobian(sys, x: np.ndarray) -> np.ndarray:
    """J_ij = d f_i / d x_j at one point x [n], from
    d/dx_j c x^a = c a_j x_j^(a_j - 1) prod_{l != j} x_l^a_l."""
    x = np.asarray(x, dtype=np.complex128)
    n = sys.n_var
    J = np.zeros((sys.n_eq, n), np.complex128)
    off = 0
    for i in range(sys.n_eq):
        m = int(sys.terms_per_eq[i])
        for k in range(m):
            a = sys.exps[off + k].astype(np.int64)
            c = complex(sys.coefs[off + k])
            for j in range(n):
                if a[j] == 0:
                    continue
                d = a.copy()
                d[j] -= 1
                J[i, j] += c * a[j] * np.prod(x ** d)
        off += m
    return J


def term_scales(sys, x: np.ndarray) -> np.ndarray:
    """scale_i = sum over the terms of equation i of |c|_1 |x^a|_1, with
    |z|_1 = |Re z| + |Im z|."""
    x = np.asarray(x, dtype=np.complex128)
    out = np.zeros(sys.n_eq)
    off = 0
    for i in range(sys.n_eq):
        m = int(sys.terms_per_eq[i])
        for k in range(m):
            c = complex(sys.coefs[off + k])
            v = np.prod(x ** sys.exps[off + k].astype(np.int64))
            out[i] += (abs(c.real) + abs(c.imag)) * (abs(v.real) + abs(v.imag))
        off += m
    return out


def exact_residual_parts(sys, parts: np.ndarray) -> float:
    """exact_residual at the point sum_k parts[:, k] (complex [n, K], the
    parts of a multiple-double number), every part taken exactly."""
    xs = [(sum(Fraction(float(v.real)) for v in row), sum(Fraction(float(v.imag)) for v in row)) for row in parts]
    worst = 0.0
    off = 0
    for i in range(sys.n_eq):
        m = int(sys.terms_per_eq[i])
        acc = (Fraction(0), Fraction(0))
        scale = 0.0
        for k in range(m):
            c = frac_complex(complex(sys.coefs[off + k]))
            mon = (Fraction(1), Fraction(0))
            for j, a in enumerate(sys.exps[off + k]):
                for _ in range(int(a)):
                    mon = _cmul(mon, xs[j])
            term = _cmul(c, mon)
            acc = (acc[0] + term[0], acc[1] + term[1])
            scale += abs(complex(sys.coefs[off + k])) * abs(complex(float(mon[0]), float(mon[1])))
        val = abs(complex(float(acc[0]), float(acc[1])))
        worst = max(worst, val / (1.0 + scale))
        off += m
    return worst


def min_pair_distance_large(A: np.ndarray, window: float = 1e-6, seed: int = 0) -> float:
    """min_pair_distance for many rows: rows are sorted by a random real
    projection, and only pairs whose projections lie within `window` of
    each other are compared (two rows closer than `window` in the max-norm
    have projections closer than window * ||w||_1, which the window covers
    for the unit-modulus weights used).  Returns the smallest distance found
    among those pairs, or inf when no pair has projections that close."""
    A = np.atleast_2d(A)
    if A.shape[0] < 2:
        return float("inf")
    rng = np.random.default_rng(seed)
    w = np.exp(2j * np.pi * rng.random(A.shape[1])) / A.shape[1]
    p = (A @ w).real
    order = np.argsort(p)
    ps, As = p[order], A[order]
    best = float("inf")
    for k in range(1, A.shape[0]):
        close = np.nonzero(ps[k:] - ps[:-k] <= window)[0]
        if close.size == 0:
            break
        d = np.max(np.abs(As[close + k] - As[close]), axis=1)
        best = min(best, float(d.min()))
    return best
