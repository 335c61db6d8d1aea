"""Mixed cells, mixed volume and binomial start solutions of polyhedral
homotopies -- TEST INFRASTRUCTURE ONLY (part of the oracle, under the same
import rule as ``oracle/__init__.py``: tests, the smoke check and the CPU
baseline of the benchmark only).

Section 2.2 of the paper (and the paragraph before it): for coefficients in
general position the polyhedral homotopies let no path diverge; the start
systems come from the mixed cells of a mixed subdivision of the Newton
polytopes, and a cell of volume V starts V paths (Figure 2: one thread makes
the cells, the others solve their start systems and track their paths).  The
paper's cells come from MixedVol and DEMiCs; this module computes them from
the definitions, in the plainest way that finishes on small systems:

  Supports A_i (the exponent vectors of equation i) and an integer lifting w
  (one value per term).  A fine mixed cell picks two points {a_i, b_i} of
  every A_i and has an inner normal v in Q^n with, for every i,
      <a, v> + w(a) = beta_i   for a in {a_i, b_i},
      <c, v> + w(c) > beta_i   for every other c in A_i.
  Its volume is |det D|, D the n x n integer matrix with rows b_i - a_i; the
  mixed volume is the sum of the volumes (Bernstein's count of the isolated
  roots in (C*)^n of a system with general coefficients).

``mixed_cells`` walks the choices depth first, equations ordered by their
number of lower edges (pairs that pass the test on their own), and drops a
partial choice when the linear program "some v meets the conditions of the
equations chosen so far" (``scipy.optimize.linprog``) has no strictly
feasible point, for two of its pairs (each two tested once) or for all of
them together; each complete choice is then checked exactly in rational
arithmetic (``fractions.Fraction``), so the pruning can only cost time.  A
tie (a third point on a cell's lower facet: the lifting is not in general
position) raises ``ValueError``.  ``mixed_cells_brute`` checks every
complete choice exactly, with no linear programming (tiny systems only).

``binomial_starts``: on a cell, equation i keeps c_a y^{a_i} + c_b y^{b_i},
so y^D = beta with beta_i = -c_{a_i} / c_{b_i}; its |det D| solutions are
y = exp(D^{-1} log beta + 2 pi i u) for u over the group D^{-1} Z^n / Z^n
(fractional parts of D^{-1} k, k integer), enumerated by closure from 0
under adding the columns of D^{-1}.

``cell_powers``: the cell's homotopy substitutes x = t^v y and divides
equation i by t^{beta_i}: the term c x^a becomes c y^a t^e with
e = <a, v> + w(a) - beta_i >= 0 (0 exactly on the cell); dividing every power
by the smallest positive one reparametrizes t (t -> t^{1/e_min}, the same
paths), so each positive power is >= 1 and the t-derivative stays bounded at
t = 0.  At t = 1 the homotopy is the system itself, so the V paths of every
cell end at its solutions.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from fractions import Fraction

import numpy as np
from scipy.optimize import linprog

from workloads.systems import PolySystem

from . import polyhedral_homotopy, track


@dataclass(frozen=True)
class Cell:
    pairs: tuple  # ((a, b), ...) per equation: global term indices, a < b
    normal: tuple  # inner normal v (Fractions)
    volume: int


def _supports(sys: PolySystem):
    """[(offset, exponents int64 [m_i, n])] per equation."""
    out, off = [], 0
    for i in range(sys.n_eq):
        m = int(sys.terms_per_eq[i])
        A = np.asarray(sys.exps[off:off + m], dtype=np.int64)
        if len({tuple(r) for r in A}) != m:
            raise ValueError(f"equation {i} lists a monomial twice")
        out.append((off, A))
        off += m
    return out


def _lift_lists(sys: PolySystem, lift):
    w = [int(x) for x in np.asarray(lift).reshape(-1)]
    if len(w) != sys.n_terms:
        raise ValueError("one lifting value per term")
    return w


def _lp_feasible(sup, w, chosen, n) -> bool:
    """Is there v with the conditions of the chosen (i, a, b) (local term
    indices) holding strictly?  max tau s.t. equalities on each pair and
    <c - a, v> + w(c) - w(a) >= tau for the other points, tau <= 1; kept
    unless the optimum is clearly negative or the equalities are
    inconsistent."""
    Aeq, beq, Aub, bub = [], [], [], []
    for (i, a, b) in chosen:
        off, A = sup[i]
        Aeq.append([float(x) for x in (A[a] - A[b])] + [0.0])
        beq.append(float(w[off + b] - w[off + a]))
        for c in range(A.shape[0]):
            if c == a or c == b:
                continue
            Aub.append([float(-x) for x in (A[c] - A[a])] + [1.0])
            bub.append(float(w[off + c] - w[off + a]))
    Aub.append([0.0] * n + [1.0])
    bub.append(1.0)
    res = linprog(c=[0.0] * n + [-1.0], A_ub=Aub, b_ub=bub, A_eq=Aeq, b_eq=beq,
                  bounds=[(None, None)] * (n + 1), method="highs")
    if res.status == 2:
        return False
    if res.status != 0:
        return True
    scale = 1.0 + max(abs(x) for x in w)
    return -res.fun > -1e-9 * scale


def _solve(D, r):
    """Exact solution of D v = r (Fractions), None if D is singular."""
    n = len(D)
    M = [[Fraction(int(x)) for x in D[i]] + [Fraction(int(r[i]))] for i in range(n)]
    for k in range(n):
        p = next((i for i in range(k, n) if M[i][k] != 0), None)
        if p is None:
            return None
        M[k], M[p] = M[p], M[k]
        for i in range(n):
            if i != k and M[i][k] != 0:
                f = M[i][k] / M[k][k]
                for j in range(k, n + 1):
                    M[i][j] -= f * M[k][j]
    return tuple(M[i][n] / M[i][i] for i in range(n))


def _det(D) -> int:
    n = len(D)
    M = [[Fraction(int(x)) for x in row] for row in D]
    d = Fraction(1)
    for k in range(n):
        p = next((i for i in range(k, n) if M[i][k] != 0), None)
        if p is None:
            return 0
        if p != k:
            M[k], M[p] = M[p], M[k]
            d = -d
        d *= M[k][k]
        for i in range(k + 1, n):
            f = M[i][k] / M[k][k]
            for j in range(k, n):
                M[i][j] -= f * M[k][j]
    assert d.denominator == 1
    return int(d)


def _exact_cell(sup, w, chosen):
    """The Cell of a complete choice [(i, a, b)] if it is a fine mixed cell,
    else None; ValueError on a tie."""
    chosen = sorted(chosen)
    D = [sup[i][1][b] - sup[i][1][a] for (i, a, b) in chosen]
    r = [w[sup[i][0] + a] - w[sup[i][0] + b] for (i, a, b) in chosen]
    v = _solve(D, r)
    if v is None:
        return None
    tie = False
    for (i, a, b) in chosen:
        off, A = sup[i]
        base = sum(int(A[a][j]) * v[j] for j in range(len(v))) + w[off + a]
        for c in range(A.shape[0]):
            if c == a or c == b:
                continue
            val = sum(int(A[c][j]) * v[j] for j in range(len(v))) + w[off + c]
            if val < base:
                return None
            tie = tie or val == base
    if tie:  # only a choice that is otherwise a cell is affected
        raise ValueError("lifting not in general position: a third point on a cell's lower facet")
    pairs = tuple((sup[i][0] + a, sup[i][0] + b) for (i, a, b) in chosen)
    return Cell(pairs, v, abs(_det(D)))


def mixed_cells(sys: PolySystem, lift) -> list:
    """Fine mixed cells of the subdivision induced by the integer lifting
    (one value per term), depth first with linear-programming pruning."""
    assert sys.n_eq == sys.n_var
    n = sys.n_var
    sup = _supports(sys)
    w = _lift_lists(sys, lift)
    edges = {}
    for i in range(n):
        m = sup[i][1].shape[0]
        edges[i] = [(a, b) for a in range(m) for b in range(a + 1, m) if _lp_feasible(sup, w, [(i, a, b)], n)]
    order = sorted(range(n), key=lambda i: (len(edges[i]), i))
    # do two edges of two equations pass the test together (memoized)?
    memo = {}

    def compatible(e, f):
        key = (e, f) if e < f else (f, e)
        if key not in memo:
            memo[key] = _lp_feasible(sup, w, [key[0], key[1]], n)
        return memo[key]

    cells = []

    def walk(depth, chosen):
        if depth == n:
            c = _exact_cell(sup, w, chosen)
            if c is not None:
                cells.append(c)
            return
        i = order[depth]
        for (a, b) in edges[i]:
            if not all(compatible((i, a, b), e) for e in chosen):
                continue
            nxt = chosen + [(i, a, b)]
            if depth <= 1 or depth == n - 1 or _lp_feasible(sup, w, nxt, n):
                walk(depth + 1, nxt)

    walk(0, [])
    return sorted(cells, key=lambda c: c.pairs)


def mixed_cells_brute(sys: PolySystem, lift) -> list:
    """Every choice of two points per support, checked exactly (no pruning)."""
    assert sys.n_eq == sys.n_var
    n = sys.n_var
    sup = _supports(sys)
    w = _lift_lists(sys, lift)
    cells = []

    def walk(i, chosen):
        if i == n:
            c = _exact_cell(sup, w, chosen)
            if c is not None:
                cells.append(c)
            return
        m = sup[i][1].shape[0]
        for a in range(m):
            for b in range(a + 1, m):
                walk(i + 1, chosen + [(i, a, b)])

    walk(0, [])
    return sorted(cells, key=lambda c: c.pairs)


def mixed_volume(cells) -> int:
    return int(sum(c.volume for c in cells))


def cell_powers(sys: PolySystem, lift, cell: Cell) -> np.ndarray:
    """Power of t per term in the cell's polyhedral homotopy (0 on the
    cell's terms, the others divided by the smallest positive one)."""
    w = _lift_lists(sys, lift)
    v = cell.normal
    n = sys.n_var
    e = []
    off = 0
    for i in range(sys.n_eq):
        a = cell.pairs[i][0]
        beta = sum(int(sys.exps[a][j]) * v[j] for j in range(n)) + w[a]
        for q in range(off, off + int(sys.terms_per_eq[i])):
            e.append(sum(int(sys.exps[q][j]) * v[j] for j in range(n)) + w[q] - beta)
        off += int(sys.terms_per_eq[i])
    assert all(x >= 0 for x in e)
    pos = [x for x in e if x > 0]
    emin = min(pos) if pos else Fraction(1)
    return np.array([float(x / emin) for x in e], dtype=np.float64)


def _inverse(D):
    n = len(D)
    cols = []
    for j in range(n):
        ej = [1 if i == j else 0 for i in range(n)]
        M = [[Fraction(int(x)) for x in D[i]] + [Fraction(ej[i])] for i in range(n)]
        for k in range(n):
            p = next(i for i in range(k, n) if M[i][k] != 0)
            M[k], M[p] = M[p], M[k]
            for i in range(n):
                if i != k and M[i][k] != 0:
                    f = M[i][k] / M[k][k]
                    for jj in range(k, n + 1):
                        M[i][jj] -= f * M[k][jj]
        cols.append([M[i][n] / M[i][i] for i in range(n)])
    return [[cols[j][i] for j in range(n)] for i in range(n)]  # row i, column j


def binomial_starts(sys: PolySystem, cell: Cell) -> np.ndarray:
    """The |det D| solutions [V, n] of the cell's binomial system
    c_a y^{a_i} + c_b y^{b_i} = 0 (every equation i)."""
    n = sys.n_var
    D = [[int(sys.exps[b][j]) - int(sys.exps[a][j]) for j in range(n)] for (a, b) in cell.pairs]
    beta = np.array([-sys.coefs[a] / sys.coefs[b] for (a, b) in cell.pairs], dtype=np.complex128)
    Dinv = _inverse(D)
    logb = np.log(beta)
    base = np.array([sum(float(Dinv[j][i]) * logb[i] for i in range(n)) for j in range(n)], dtype=np.complex128)
    gens = [tuple(Dinv[j][i] for j in range(n)) for i in range(n)]  # columns of D^{-1}

    def frac(u):
        return tuple(x - math.floor(x) for x in u)

    zero = tuple(Fraction(0) for _ in range(n))
    seen = {zero}
    todo = [zero]
    while todo:
        u = todo.pop()
        for g in gens:
            s = frac(tuple(u[j] + g[j] for j in range(n)))
            if s not in seen:
                seen.add(s)
                todo.append(s)
    if len(seen) != cell.volume:
        raise AssertionError("group order differs from the cell volume")
    out = np.empty((len(seen), n), dtype=np.complex128)
    for k, u in enumerate(sorted(seen)):
        out[k] = np.exp(base + 2j * np.pi * np.array([float(x) for x in u]))
    return out


def track_polyhedral(sys: PolySystem, lift, cells=None, opts=None, threads=None):
    """Solve sys (coefficients in general position) by polyhedral
    homotopies: every cell's binomial solutions tracked to t = 1.  Returns
    (starts [P, n], x [P, n], cls [P], stats [P], cell_of [P]) in cell
    order."""
    if cells is None:
        cells = mixed_cells(sys, lift)
    S, X, C, T, K = [], [], [], [], []
    for k, cell in enumerate(cells):
        st = binomial_starts(sys, cell)
        h = polyhedral_homotopy(sys, cell_powers(sys, lift, cell))
        x, cls, stats = track(h, starts=st, opts=opts, threads=threads)
        S.append(st)
        X.append(x)
        C.append(cls)
        T.append(stats)
        K.append(np.full(st.shape[0], k, dtype=np.int64))
    n = sys.n_var
    if not S:
        return (np.zeros((0, n), np.complex128), np.zeros((0, n), np.complex128), np.zeros(0, np.int8),
                None, np.zeros(0, np.int64))
    return np.concatenate(S), np.concatenate(X), np.concatenate(C), np.concatenate(T), np.concatenate(K)
