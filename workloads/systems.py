"""Seeded synthetic polynomial systems and random constants.

This module is the one source of inputs shared by the CPU oracle and the GPU
library.  It defines polynomial systems as coefficient/exponent lists and
draws the random constants the method consumes (the gamma of the total-degree
homotopy, the hyperplane and slack constants of the embedding).  It contains
none of the method's arithmetic: no evaluation, no tracking, no embedding.

A system is a :class:`PolySystem`: equation ``i`` owns ``terms_per_eq[i]``
consecutive terms; term ``t`` is ``coefs[t] * prod_j x_j ** exps[t, j]``.

Workloads follow the paper's test problems: the cyclic n-roots systems
(Example 2.1, eq. (1) for n = 4; Section 5 for n = 8, 9, 12), the factored
system of Example 3.1 and the membership example of Example 4.1, plus random
dense and sparse systems with standard complex Gaussian coefficients.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np


@dataclass
class PolySystem:
    n_eq: int
    n_var: int
    terms_per_eq: np.ndarray  # int32 [n_eq]
    exps: np.ndarray  # uint8 [T, n_var]
    coefs: np.ndarray  # complex128 [T]
    name: str = ""
    meta: dict = field(default_factory=dict)

    def __post_init__(self):
        self.terms_per_eq = np.ascontiguousarray(self.terms_per_eq, dtype=np.int32)
        self.exps = np.ascontiguousarray(self.exps, dtype=np.uint8).reshape(-1, self.n_var)
        self.coefs = np.ascontiguousarray(self.coefs, dtype=np.complex128)
        assert self.terms_per_eq.shape == (self.n_eq,)
        assert self.exps.shape[0] == self.coefs.shape[0] == int(self.terms_per_eq.sum())

    @property
    def n_terms(self) -> int:
        return int(self.coefs.shape[0])

    def equation_terms(self, i: int):
        """(exps, coefs) of equation i."""
        off = int(self.terms_per_eq[:i].sum())
        m = int(self.terms_per_eq[i])
        return self.exps[off:off + m], self.coefs[off:off + m]

    def degrees(self) -> np.ndarray:
        """Total degree of every equation (max over its terms)."""
        out = np.zeros(self.n_eq, dtype=np.int64)
        for i in range(self.n_eq):
            e, _ = self.equation_terms(i)
            out[i] = int(e.astype(np.int64).sum(axis=1).max())
        return out

    def bezout(self) -> int:
        return int(np.prod(self.degrees(), dtype=object))


def _from_dicts(n_var: int, eqs: list[dict], name: str = "") -> PolySystem:
    """Build a system from one {exponent tuple: coefficient} dict per equation."""
    exps, coefs, tpe = [], [], []
    for d in eqs:
        items = [(k, v) for k, v in d.items() if v != 0]
        tpe.append(len(items))
        for k, v in items:
            exps.append(k)
            coefs.append(v)
    return PolySystem(len(eqs), n_var, np.array(tpe), np.array(exps, dtype=np.uint8).reshape(-1, n_var),
                      np.array(coefs, dtype=np.complex128), name=name)


# ---------------------------------------------------------------- random draws

def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def cn01(rng: np.random.Generator, size) -> np.ndarray:
    """Standard complex Gaussian: real and imaginary parts i.i.d. N(0, 1/2)."""
    s = np.sqrt(0.5)
    return rng.normal(0.0, s, size) + 1j * rng.normal(0.0, s, size)


def unit_gamma(rng: np.random.Generator) -> complex:
    """A random point on the unit circle, angle uniform in [0, 2 pi)."""
    theta = rng.uniform(0.0, 2.0 * np.pi)
    return complex(np.cos(theta), np.sin(theta))


def random_lifting(rng: np.random.Generator, n_terms: int, bits: int = 20) -> np.ndarray:
    """Integer lifting values for the mixed cells of polyhedral homotopies
    (Section 2.2): one uniform integer in [0, 2^bits) per term."""
    return rng.integers(0, 1 << bits, n_terms).astype(np.int32)


def embedding_constants(rng: np.random.Generator, n_eq: int, n_var: int, top_dim: int):
    """Random constants of the embedding E_D (Section 2.1, eq. (2)).

    Returns ``gammas`` [n_eq, D] (the multiplier of slack z_k in equation i)
    and ``hyper`` [D, n_var + 1] (hyperplane k is hyper[k,0] + sum_j
    hyper[k,j+1] x_j + z_k), all standard complex Gaussian.
    """
    gammas = cn01(rng, (n_eq, top_dim))
    hyper = cn01(rng, (top_dim, n_var + 1))
    return gammas, hyper


# ---------------------------------------------------------------- systems

def cyclic(n: int) -> PolySystem:
    """Cyclic n-roots (Example 2.1, eq. (1) for n = 4).

    Equation k < n is the sum over i of x_i x_{i+1} ... x_{i+k-1} (indices mod
    n); equation n is x_1 ... x_n - 1.
    """
    eqs = []
    for k in range(1, n):
        d = {}
        for i in range(n):
            e = [0] * n
            for j in range(k):
                e[(i + j) % n] = 1
            d[tuple(e)] = d.get(tuple(e), 0) + 1.0
        eqs.append(d)
    eqs.append({tuple([1] * n): 1.0, tuple([0] * n): -1.0})
    return _from_dicts(n, eqs, name=f"cyclic{n}")


def with_random_coefficients(sys: PolySystem, rng: np.random.Generator, name: str = "") -> PolySystem:
    """Same supports, standard complex Gaussian coefficients."""
    return PolySystem(sys.n_eq, sys.n_var, sys.terms_per_eq.copy(), sys.exps.copy(),
                      cn01(rng, sys.n_terms), name=name or sys.name + "-rand")


def all_monomials(n: int, deg: int):
    """Exponent vectors of all monomials of total degree <= deg in n variables."""
    out = []
    for e in itertools.product(range(deg + 1), repeat=n):
        if sum(e) <= deg:
            out.append(e)
    out.sort(key=lambda e: (sum(e), e))
    return out


def random_dense(n: int, deg: int, rng: np.random.Generator) -> PolySystem:
    """n equations in n unknowns, every monomial of total degree <= deg present."""
    mons = all_monomials(n, deg)
    exps = np.array(mons * n, dtype=np.uint8).reshape(-1, n)
    return PolySystem(n, n, np.full(n, len(mons)), exps, cn01(rng, exps.shape[0]), name=f"dense{n}d{deg}")


def univariate(coeffs_low_to_high) -> PolySystem:
    """One polynomial in one unknown, sum_k c_k x^k."""
    c = np.asarray(coeffs_low_to_high, dtype=np.complex128)
    keep = [k for k in range(len(c)) if c[k] != 0]
    return PolySystem(1, 1, np.array([len(keep)]), np.array(keep, dtype=np.uint8).reshape(-1, 1), c[keep],
                      name=f"univariate{len(c) - 1}")


def _poly_mul(a: dict, b: dict) -> dict:
    out = {}
    for ea, ca in a.items():
        for eb, cb in b.items():
            e = tuple(x + y for x, y in zip(ea, eb))
            out[e] = out.get(e, 0) + ca * cb
    return {e: c for e, c in out.items() if c != 0}


def _linear(n: int, var: int, root: float) -> dict:
    """x_var - root as an exponent dict."""
    e = [0] * n
    e[var] = 1
    return {tuple(e): 1.0, tuple([0] * n): -float(root)}


def _product_of_factors(n: int, factors) -> dict:
    p = {tuple([0] * n): 1.0}
    for var, root in factors:
        p = _poly_mul(p, _linear(n, var, root))
    return p


def multistep_example() -> PolySystem:
    """The factored system of Example 3.1 (eq. (5)), expanded into terms.

    (x1-1)(x1-2)(x1-3)(x1-4), (x1-1)(x2-1)(x2-2)(x2-3),
    (x1-1)(x1-2)(x3-1)(x3-2), (x1-1)(x2-1)(x3-1)(x4-1).
    """
    n = 4
    eqs = [
        _product_of_factors(n, [(0, 1), (0, 2), (0, 3), (0, 4)]),
        _product_of_factors(n, [(0, 1), (1, 1), (1, 2), (1, 3)]),
        _product_of_factors(n, [(0, 1), (0, 2), (2, 1), (2, 2)]),
        _product_of_factors(n, [(0, 1), (1, 1), (2, 1), (3, 1)]),
    ]
    return _from_dicts(n, eqs, name="multistep")


def membership_example() -> PolySystem:
    """The system of Example 4.1 (eq. (8)): (x1-1)(x1-2), (x1-1) x2^2."""
    n = 2
    x2sq = {(0, 2): 1.0}
    eqs = [_product_of_factors(n, [(0, 1), (0, 2)]), _poly_mul(_linear(n, 0, 1), x2sq)]
    return _from_dicts(n, eqs, name="membership")


def _sparse_exponent_pool(n: int):
    """Exponent vectors with entries 0..3 and total degree 1..4."""
    pool = []

    def rec(prefix, left):
        if len(prefix) == n:
            if sum(prefix) >= 1:
                pool.append(tuple(prefix))
            return
        for a in range(0, min(3, left) + 1):
            rec(prefix + [a], left - a)

    rec([], 4)
    return pool


def random_sparse(rng: np.random.Generator, n: int | None = None, bezout_range=(100, 100_000)) -> PolySystem:
    """One system of the batching workload.

    n uniform in 3..10 unless given; every equation has m uniform in 2..6
    distinct monomials: a constant term plus m-1 monomials drawn uniformly from
    the exponent vectors with entries 0..3 and total degree 1..4.
    Coefficients standard complex Gaussian.  Systems are redrawn when some
    variable appears in no equation or the Bezout number falls outside
    ``bezout_range``.
    """
    while True:
        nn = int(rng.integers(3, 11)) if n is None else n
        pool = _sparse_exponent_pool(nn)
        eqs_e = []
        for _ in range(nn):
            m = int(rng.integers(2, 7))
            idx = rng.choice(len(pool), size=m - 1, replace=False)
            eqs_e.append([tuple([0] * nn)] + [pool[k] for k in sorted(idx)])
        used = np.zeros(nn, dtype=bool)
        degs = []
        for es in eqs_e:
            a = np.array(es)
            used |= a.sum(axis=0) > 0
            degs.append(int(a.sum(axis=1).max()))
        bez = int(np.prod(degs))
        if not used.all() or not (bezout_range[0] <= bez <= bezout_range[1]):
            continue
        exps = np.array([e for es in eqs_e for e in es], dtype=np.uint8)
        tpe = np.array([len(es) for es in eqs_e])
        return PolySystem(nn, nn, tpe, exps, cn01(rng, exps.shape[0]), name=f"sparse{nn}")
