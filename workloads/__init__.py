"""Seeded synthetic inputs shared by the oracle and the GPU library (no method arithmetic)."""
from .systems import (PolySystem, all_monomials, cn01, cyclic, embedding_constants, membership_example,
                      multistep_example, random_dense, random_lifting, random_sparse, rng_for, univariate,
                      unit_gamma, with_random_coefficients)
from . import configs

__all__ = [
    "PolySystem", "all_monomials", "cn01", "cyclic", "embedding_constants", "membership_example",
    "multistep_example", "random_dense", "random_lifting", "random_sparse", "rng_for", "univariate", "unit_gamma",
    "with_random_coefficients", "configs",
]
