"""GB300 path tracker for polynomial homotopies (total-degree homotopy,
embedding and cascade of a numerical irreducible decomposition).

The compute path is libphc.so (CUDA for sm_103a, C ABI in include/phc.h);
this package only marshals arguments (``_lib``) and allocates the output
tensors for the convenience helpers below.  Nothing here computes on the CPU.

Typical use (a system is any object with n_eq, n_var, terms_per_eq [n_eq],
exps [T, n_var] uint8 and coefs [T] complex)::

    import paper_1804_03807_gb300 as P
    h = P.phc_make_homotopy(system, gamma)          # total-degree homotopy
    r = P.track(h)                                  # every path, on the GPU
    P.refine(h, r)                                  # double double where ill-conditioned
    x, cls = r.x.cpu().numpy().T, r.cls.cpu().numpy()   # endpoints, PHC_REGULAR ...

    E = P.phc_embed(system, 1, gammas, hyper)       # top dimension 1 (eq. (2))
    hE = P.phc_make_homotopy(E, gamma)
    top = P.track(hE)
    stage = P.cascade_from(hE, 1, top)              # dimension 0, from the device outputs
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from ._lib import (PHC_STOP_SKIPPED, phc_cascade_from, PHC_AT_INFINITY, PHC_FAILED, PHC_MAX_VARS, PHC_PREC_FP32_INTERIOR, PHC_PREC_FP64,
                   PHC_REGULAR, PHC_SINGULAR, PHC_STOP_REACHED, STATS_DTYPE, Homotopy, PhcError, SystemLists,
                   load, phc_cascade_stage, phc_default_opts, phc_embed, phc_last_error, phc_make_homotopy,
                   phc_make_homotopy_batch,
                   phc_num_paths, phc_opts, phc_refine_endpoints, phc_track_paths,
                   phc_tail_paths, phc_track_many, phc_track_paths_noalloc, phc_track_pipeline,
                   phc_make_parameter_homotopy, phc_track_from, phc_membership_test, phc_square,
                   phc_many_plan_create, phc_many_plan_run, ManyPlan, phc_track_paths_dd, phc_endgame,
                   phc_mixed_cells, phc_make_polyhedral_homotopy, phc_polyhedral_starts, phc_track_polyhedral,
                   phc_solve_polyhedral, phc_track_paths_qd, phc_fp64_probe)

__all__ = [
    "PHC_AT_INFINITY", "PHC_FAILED", "PHC_MAX_VARS", "PHC_PREC_FP32_INTERIOR", "PHC_PREC_FP64", "PHC_REGULAR",
    "PHC_SINGULAR", "PHC_STOP_REACHED", "STATS_DTYPE", "Homotopy", "PhcError", "SystemLists", "load",
    "phc_cascade_stage", "phc_default_opts", "phc_embed", "phc_last_error", "phc_make_homotopy",
    "phc_make_homotopy_batch", "phc_num_paths",
    "phc_opts", "phc_refine_endpoints", "phc_track_many", "phc_track_paths", "phc_track_paths_noalloc",
    "phc_track_pipeline", "track_many", "phc_cascade_from", "PHC_STOP_SKIPPED", "cascade_from",
    "Tracked", "pipeline", "track", "cascade", "refine",
    "stats_numpy", "phc_tail_paths", "phc_make_parameter_homotopy", "phc_track_from", "phc_membership_test",
    "track_from", "membership", "phc_square", "phc_many_plan_create", "phc_many_plan_run", "ManyPlan",
    "phc_track_paths_dd", "track_dd", "phc_endgame", "endgame",
    "phc_mixed_cells", "phc_make_polyhedral_homotopy", "phc_polyhedral_starts", "phc_track_polyhedral",
    "phc_fp64_probe",
    "phc_solve_polyhedral", "polyhedral_starts", "track_polyhedral", "solve_polyhedral",
    "phc_track_paths_qd", "track_qd",
]


@dataclass
class Tracked:
    """Device outputs of one call: x [n_var, P] complex128 (SoA), cls [P]
    int8, stats [P, 80] uint8 (phc_path_stats records), slack_zero [P] uint8
    for cascade stages."""
    x: object
    cls: object
    stats: object
    slack_zero: object = None


def stats_numpy(stats) -> np.ndarray:
    """Copy a stats tensor to the host as a numpy structured array."""
    return stats.cpu().numpy().view(STATS_DTYPE).reshape(-1)


def _alloc(n_var: int, n: int, device):
    import torch
    x = torch.empty((n_var, n), dtype=torch.complex128, device=device)
    cls = torch.empty(n, dtype=torch.int8, device=device)
    st = torch.empty((n, STATS_DTYPE.itemsize), dtype=torch.uint8, device=device)
    return x, cls, st


def track(h: Homotopy, first: int = 0, n_paths: int | None = None, opts=None, stream=None,
          device="cuda") -> Tracked:
    """Track total-degree paths first..first+n_paths-1 into new tensors."""
    if n_paths is None:
        n_paths = phc_num_paths(h) - first
    x, cls, st = _alloc(h.n, n_paths, device)
    phc_track_paths(h, first, n_paths, opts, x, cls, st, stream)
    return Tracked(x, cls, st)


def track_from(h: Homotopy, starts, starts_per_system: int = 0, opts=None, stream=None) -> Tracked:
    """Track paths of h from the columns of starts [n_var, n] (device)."""
    n = int(starts.shape[1])
    x, cls, st = _alloc(h.n, n, starts.device)
    phc_track_from(h, starts.contiguous(), n, starts_per_system, opts, x, cls, st, stream)
    return Tracked(x, cls, st)


def membership(emb, k: int, witness, points, tol: float = 1e-3, opts=None, stream=None):
    """Homotopy membership test (Section 4.1): for every row of points
    [p, n_var - k] whether it lies on the set whose witness points (device
    [n_var, m], solutions of E_k = emb with zero slacks) are given.  Returns
    (on [p] bool numpy array, Tracked endpoints [n_var, p * m])."""
    import torch
    pts = np.atleast_2d(np.asarray(points, dtype=np.complex128))
    p, m = pts.shape[0], int(witness.shape[1])
    dev = witness.device
    on = torch.empty(p, dtype=torch.uint8, device=dev)
    x = torch.empty((int(emb.n_var), p * m), dtype=torch.complex128, device=dev)
    cls = torch.empty(p * m, dtype=torch.int8, device=dev)
    phc_membership_test(emb, k, witness.contiguous(), pts, tol, opts, on, x, cls, stream)
    return on.cpu().numpy().astype(bool), Tracked(x, cls, None)


def track_dd(h: Homotopy, first: int = 0, n_paths: int | None = None, opts=None, stream=None, device="cuda"):
    """Total-degree paths tracked in complex double double; returns
    (Tracked with the double parts in x, the low parts [n_var, P])."""
    import torch
    if n_paths is None:
        n_paths = phc_num_paths(h) - first
    x, cls, st = _alloc(h.n, n_paths, device)
    xlo = torch.empty_like(x)
    phc_track_paths_dd(h, first, n_paths, opts, x, xlo, cls, st, stream)
    return Tracked(x, cls, st), xlo


def endgame(h: Homotopy, first: int = 0, n_paths: int | None = None, opts=None, stream=None, device="cuda"):
    """Cauchy endgame of total-degree paths; returns (Tracked with the
    estimates in x (cls unused: -1), cycle numbers [P] int32)."""
    import torch
    if n_paths is None:
        n_paths = phc_num_paths(h) - first
    x, cls, st = _alloc(h.n, n_paths, device)
    cls.fill_(-1)
    cyc = torch.empty(n_paths, dtype=torch.int32, device=device)
    phc_endgame(h, first, n_paths, opts, x, cyc, st, stream)
    return Tracked(x, cls, st), cyc


def cascade(h_k: Homotopy, k: int, starts, opts=None, stream=None) -> Tracked:
    """One cascade stage from E_k (handle h_k) on starts [n_var(E_k), n]."""
    import torch
    n = int(starts.shape[1])
    x, cls, st = _alloc(h_k.n - 1, n, starts.device)
    sz = torch.empty(n, dtype=torch.uint8, device=starts.device)
    phc_cascade_stage(h_k, k, starts.contiguous(), n, opts, x, cls, sz, st, stream)
    return Tracked(x, cls, st, sz)


def cascade_from(h_k: Homotopy, k: int, prev: Tracked, opts=None, stream=None) -> Tracked:
    """The cascade stage from E_k fed by the previous stage's outputs (prev.x
    in E_k's unknowns); outputs indexed like prev (cls -1 where no start)."""
    import torch
    n = int(prev.x.shape[1])
    x, cls, st = _alloc(h_k.n - 1, n, prev.x.device)
    sz = torch.empty(n, dtype=torch.uint8, device=prev.x.device)
    phc_cascade_from(h_k, k, prev.x, prev.cls, prev.slack_zero, n, opts, x, cls, sz, st, stream)
    return Tracked(x, cls, st, sz)


def track_many(hs, opts=None, stream=None, device="cuda"):
    """Every path of every handle in hs (different systems), into new tensors."""
    outs = [_alloc(h.n, phc_num_paths(h), device) for h in hs]
    phc_track_many(hs, opts, [o[0] for o in outs], [o[1] for o in outs], [o[2] for o in outs], stream)
    return [Tracked(*o) for o in outs]


def pipeline(h_k: Homotopy, k: int, first: int = 0, n_paths: int | None = None, opts=None, stream=None,
             device="cuda"):
    """Top stage of E_k and the cascade stage below it in one launch; returns
    (top, next) Tracked records indexed by top path (next.cls = -1 where a
    top endpoint was not continued)."""
    import torch
    if n_paths is None:
        n_paths = phc_num_paths(h_k) - first
    xt, ct, st = _alloc(h_k.n, n_paths, device)
    xn, cn, sn = _alloc(h_k.n - 1, n_paths, device)
    sz = torch.empty(n_paths, dtype=torch.uint8, device=device)
    phc_track_pipeline(h_k, k, first, n_paths, opts, xt, ct, st, xn, cn, sz, sn, stream)
    return Tracked(xt, ct, st), Tracked(xn, cn, sn, sz)


def refine(h: Homotopy, r: Tracked, cond_threshold: float = 1e6, cond_max: float = 1e12, max_iters: int = 8,
           stream=None):
    """Double double refinement in place on r.x / r.cls / r.stats; returns x_lo."""
    import torch
    x_lo = torch.empty_like(r.x)
    phc_refine_endpoints(h, r.x, x_lo, int(r.x.shape[1]), cond_threshold, cond_max, max_iters, r.cls, r.stats,
                         stream)
    return x_lo


def polyhedral_starts(h: Homotopy, first: int = 0, n_paths: int | None = None, stream=None, device="cuda"):
    """Start solutions of a polyhedral handle's paths: complex128 [n_var, P]."""
    import torch
    if n_paths is None:
        n_paths = phc_num_paths(h) - first
    x = torch.zeros((h.n, max(n_paths, 1)), dtype=torch.complex128, device=device)
    phc_polyhedral_starts(h, first, n_paths, x, stream)
    return x[:, :n_paths]


def track_polyhedral(h: Homotopy, first: int = 0, n_paths: int | None = None, opts=None, stream=None,
                     device="cuda") -> Tracked:
    """Track the paths of a polyhedral handle (every cell's binomial solutions
    to the roots of its system)."""
    if n_paths is None:
        n_paths = phc_num_paths(h) - first
    x, cls, st = _alloc(h.n, n_paths, device)
    phc_track_polyhedral(h, first, n_paths, opts, x, cls, st, stream)
    return Tracked(x, cls, st)


def solve_polyhedral(sys, lift, max_paths: int, opts=None, stream=None, device="cuda") -> Tracked:
    """The pipelined polyhedral solver (cells made on this thread while the
    GPU tracks): Tracked outputs of the mixed volume's paths, cells in the
    order they were made."""
    x, cls, st = _alloc(sys.n_var, max(max_paths, 1), device)
    mv, _ = phc_solve_polyhedral(sys, lift, opts, max_paths, x, cls, st, stream)
    return Tracked(x[:, :mv], cls[:mv], st[:mv])


def track_qd(h: Homotopy, first: int = 0, n_paths: int | None = None, opts=None, stream=None, device="cuda"):
    """Total-degree paths tracked in complex quad double; returns (Tracked
    with the leading parts in x, the parts complex128 [4, n_var, P])."""
    import torch
    if n_paths is None:
        n_paths = phc_num_paths(h) - first
    parts = torch.empty((4, h.n, n_paths), dtype=torch.complex128, device=device)
    _, cls, st = _alloc(h.n, n_paths, device)
    phc_track_paths_qd(h, first, n_paths, opts, parts, cls, st, stream)
    return Tracked(parts[0], cls, st), parts
