"""The five benchmark workloads, seeded, plus reduced-size variants for tests.

Each builder returns plain data (systems, gammas, embedding constants, arrival
times); nothing here evaluates or tracks anything.

* ``dense4``      random dense n=4, degree 2, all 15 monomials, 16 paths (seed 1)
* ``cyclic7_batch`` cyclic 7 + 8 random-coefficient copies, 9 x 5040 paths (seed 2)
* ``cyclic8_d1``  cyclic 8 embedded for top dimension 1, 40,320 paths + one
                  cascade stage (seed 3)
* ``sparse_batch`` 256 random sparse systems of uneven size (seed 4)
* ``serving``     Poisson arrivals of sparse requests plus one cyclic 9 request
                  embedded for top dimension 2 (seed 5)
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .systems import (PolySystem, cn01, cyclic, embedding_constants, random_dense, random_sparse, rng_for,
                      unit_gamma, with_random_coefficients)


@dataclass
class Workload:
    name: str
    systems: list
    gammas: list  # complex, one per system (total-degree homotopy)
    embed: dict = field(default_factory=dict)  # optional: top_dim, gammas, hyper
    extra: dict = field(default_factory=dict)

    @property
    def n_paths(self) -> int:
        return sum(s.bezout() for s in self.systems)


def dense4(seed: int = 1) -> Workload:
    rng = rng_for(seed)
    s = random_dense(4, 2, rng)
    return Workload("dense4", [s], [unit_gamma(rng)])


def cyclic_batch(n: int = 7, copies: int = 8, seed: int = 2) -> Workload:
    """Cyclic n plus ``copies`` systems with its supports and random coefficients."""
    rng = rng_for(seed)
    base = cyclic(n)
    systems = [base] + [with_random_coefficients(base, rng, name=f"cyclic{n}-rand{k}") for k in range(copies)]
    gammas = [unit_gamma(rng) for _ in systems]
    return Workload(f"cyclic{n}x{copies + 1}", systems, gammas)


def cyclic7_batch(seed: int = 2) -> Workload:
    return cyclic_batch(7, 8, seed)


def embedded_cyclic(n: int, top_dim: int, seed: int) -> Workload:
    """Cyclic n with the constants of its embedding for dimension ``top_dim``.

    The embedding itself is built by the code under test (library or oracle);
    this returns the base system, the gamma of the total-degree homotopy on
    the embedded system and the embedding constants.
    """
    rng = rng_for(seed)
    base = cyclic(n)
    g, h = embedding_constants(rng, base.n_eq, base.n_var, top_dim)
    gamma = unit_gamma(rng)
    return Workload(f"cyclic{n}-d{top_dim}", [base], [gamma], embed={"top_dim": top_dim, "gammas": g, "hyper": h})


def cyclic8_d1(seed: int = 3) -> Workload:
    return embedded_cyclic(8, 1, seed)


def sparse_batch(count: int = 256, seed: int = 4, bezout_range=(100, 100_000)) -> Workload:
    rng = rng_for(seed)
    systems = [random_sparse(rng, bezout_range=bezout_range) for _ in range(count)]
    gammas = [unit_gamma(rng) for _ in systems]
    return Workload(f"sparse{count}", systems, gammas)


def serving(n_requests: int = 2000, rate: float = 200.0, seed: int = 5, bezout_range=(100, 100_000),
            big: tuple | None = (9, 2)) -> Workload:
    """Poisson arrivals (exponential inter-arrival times, mean 1/rate) of sparse
    requests plus one embedded cyclic request arriving with the first one."""
    rng = rng_for(seed)
    gaps = rng.exponential(1.0 / rate, n_requests)
    arrivals = np.cumsum(gaps) - gaps[0]
    systems = [random_sparse(rng, bezout_range=bezout_range) for _ in range(n_requests)]
    gammas = [unit_gamma(rng) for _ in systems]
    extra = {"arrivals": arrivals}
    if big is not None:
        n, d = big
        base = cyclic(n)
        g, h = embedding_constants(rng, base.n_eq, base.n_var, d)
        extra["big"] = {"system": base, "top_dim": d, "gammas": g, "hyper": h, "gamma": unit_gamma(rng),
                        "arrival": 0.0}
    return Workload(f"serving{n_requests}", systems, gammas, extra=extra)


BUILDERS = {
    "dense4": dense4,
    "cyclic7_batch": cyclic7_batch,
    "cyclic8_d1": cyclic8_d1,
    "sparse_batch": sparse_batch,
    "serving": serving,
}
