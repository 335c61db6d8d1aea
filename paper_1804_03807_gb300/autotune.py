"""Launch-parameter tuner for the path tracker.

The tracker's results never depend on its launch parameters -- threads per
block, the idle fraction that starts the tail hand-off, threads per path in
the tail kernel -- (tests/test_gpu_tail.py checks the bytes), so the tuner
may choose among them by time alone.  It times each candidate on a sample of
the caller's workload (a prefix of the paths, or a few of the systems) and
keeps the fastest; results are cached per workload signature (kind, number
of unknowns, terms, path count) for the life of the process.

All timing goes through the library calls; nothing here computes paths.
"""
from __future__ import annotations

import itertools
import time

from ._lib import phc_default_opts, phc_num_paths, phc_opts

# Candidate values of each tuned option (0 = the library's own choice).
GRID = {
    "block_threads": (0, 128),
    "tail_threads": (16, 32),
    "tail_drain": (0.7, 0.8, 0.9),
}

_cache: dict = {}


def candidates(n: int, grid: dict = GRID) -> list[dict]:
    """Every combination of the grid's values that the kernels support for n
    unknowns (8 threads per path only for n <= 8)."""
    keys = sorted(grid)
    out = []
    for vals in itertools.product(*(grid[k] for k in keys)):
        c = dict(zip(keys, vals))
        if c.get("tail_threads") == 8 and n > 8:
            continue
        out.append(c)
    return out


def make_opts(base: phc_opts | None, cand: dict) -> phc_opts:
    o = phc_default_opts()
    if base is not None:
        for name, _ in phc_opts._fields_:
            setattr(o, name, getattr(base, name))
    for k, v in cand.items():
        setattr(o, k, v)
    return o


def pick(run, cands: list[dict], timer=None, reps: int = 1):
    """Time run(cand) for every candidate (best of reps after one untimed
    call) and return (fastest candidate, [(seconds, cand), ...]).  Ties keep
    the earlier candidate."""
    timer = timer or _wall
    table = []
    best, best_t = None, float("inf")
    for c in cands:
        run(c)
        t = min(timer(lambda: run(c)) for _ in range(max(1, reps)))
        table.append((t, c))
        if t < best_t:
            best, best_t = c, t
    return best, table


def _wall(fn) -> float:
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    fn()
    torch.cuda.synchronize()
    return time.perf_counter() - t0


def signature(kind: str, hs) -> tuple:
    """Cache key: the call kind and, per handle, (unknowns, terms, paths)."""
    return (kind,) + tuple((h.n, getattr(h, "n_terms", 0), phc_num_paths(h)) for h in hs)


def tune_track(h, base: phc_opts | None = None, sample_paths: int = 20000, timer=None, grid: dict = GRID):
    """Options for phc_track_paths on handle h, tuned on its first
    sample_paths paths.  Returns a phc_opts."""
    from . import track
    key = signature("track", [h])
    if key not in _cache:
        n_paths = min(sample_paths, phc_num_paths(h))
        best, _ = pick(lambda c: track(h, 0, n_paths, opts=make_opts(base, c)), candidates(h.n, grid), timer)
        _cache[key] = best
    return make_opts(base, _cache[key])


def tune_many(hs, base: phc_opts | None = None, sample_systems: int = 32, timer=None, grid: dict = GRID):
    """Options for phc_track_many over handles hs, tuned on every k-th
    handle (about sample_systems of them, so that each size is sampled).
    Returns a phc_opts."""
    from . import track_many
    key = signature("many", hs)
    if key not in _cache:
        step = max(1, len(hs) // max(1, sample_systems))
        sample = list(hs[::step])
        n_max = max(h.n for h in sample)
        best, _ = pick(lambda c: track_many(sample, opts=make_opts(base, c)), candidates(n_max, grid), timer)
        _cache[key] = best
    return make_opts(base, _cache[key])


def clear_cache():
    _cache.clear()
