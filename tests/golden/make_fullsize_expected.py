"""Writes tests/golden/fullsize_expected.npz: what the CPU oracle computes on
the two largest benchmark workloads, for the full-size GPU parity tests.

Calls only the oracle (oracle/) and the seeded input generators
(workloads/).  Un-timed; on 8 cores it takes about an hour:

    python tests/golden/make_fullsize_expected.py

Stored per system (or stage): the class counts (regular, singular, at
infinity, failed) and, for every regular endpoint, its value under a fixed
seeded linear form l(x) = sum_j r_j x_j (complex; r from rng_for(4242)) and
its norm max_j max(|Re x_j|, |Im x_j|).  Two sets of roots agree within a
relative tolerance when their l-values match one to one within that
tolerance times sum_j |r_j| (1 + norm): l is one random projection, so
distinct roots keep distinct values and a root that moved changes its value.

Workloads:
* sparse batch: 256 random sparse systems of uneven size, every
  total-degree path of each (4,322,140 paths), no refinement;
* cyclic 9 embedded for top dimension 2 (the large request of the serving
  workload): the top stage (362,880 paths), then the cascade stage from E_2
  on the regular endpoints with z_2 != 0, then the stage from E_1 on its
  regular endpoints with z_1 != 0 (Section 3.1), no refinement.
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from workloads import configs, rng_for  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "fullsize_expected.npz")


def projection_vector(n_max: int = 12) -> np.ndarray:
    rng = rng_for(4242)
    return rng.normal(size=n_max) + 1j * rng.normal(size=n_max)


def summarize(x: np.ndarray, cls: np.ndarray, r: np.ndarray):
    """(class counts, l-values of the regular endpoints, their norms)."""
    reg = x[cls == 0]
    lv = reg @ r[:x.shape[1]]
    nrm = np.max(np.maximum(np.abs(reg.real), np.abs(reg.imag)), axis=1) if len(reg) else np.zeros(0)
    return np.bincount(cls.astype(np.int64), minlength=4)[:4], lv, nrm


def sparse_batch(r):
    w = configs.sparse_batch()
    counts, lv, nrm, off = [], [], [], [0]
    for i, (s, g) in enumerate(zip(w.systems, w.gammas)):
        x, c, _ = oracle.track(oracle.total_degree(s, g))
        k, l, m = summarize(x, c, r)
        counts.append(k)
        lv.append(l)
        nrm.append(m)
        off.append(off[-1] + len(l))
        print(f"sparse {i}: {len(c)} paths, counts {k.tolist()}", flush=True)
    return np.array(counts), np.concatenate(lv), np.concatenate(nrm), np.array(off)


def cyclic9_d2(r):
    w = configs.serving(n_requests=1, big=(9, 2))
    b = w.extra["big"]
    base, g, hy, gamma = b["system"], b["gammas"], b["hyper"], b["gamma"]
    n = base.n_var
    E2 = oracle.embed(base, 2, g, hy)
    x, c, _ = oracle.track(oracle.total_degree(E2, gamma))
    out = [summarize(x, c, r)]
    print(f"cyclic9 D=2 top: counts {out[0][0].tolist()}", flush=True)
    starts = x[(c == 0) & ~oracle.slack_zero(x, n + 1)]
    Ek = E2
    n_starts = [len(starts)]
    for k in (2, 1):
        E_next, xk, ck, _ = oracle.cascade_stage(Ek, n, n, k, starts)
        out.append(summarize(xk, ck, r))
        print(f"cyclic9 stage {k}->{k - 1}: {len(starts)} starts, counts {out[-1][0].tolist()}", flush=True)
        if k > 1:
            starts = xk[(ck == 0) & ~oracle.slack_zero(xk, n + k - 2)]
            n_starts.append(len(starts))
        Ek = E_next
    counts = np.array([o[0] for o in out])
    off = np.cumsum([0] + [len(o[1]) for o in out])
    return counts, np.concatenate([o[1] for o in out]), np.concatenate([o[2] for o in out]), off, np.array(n_starts)


def main():
    r = projection_vector()
    t0 = time.time()
    c9 = cyclic9_d2(r)
    sp = sparse_batch(r)
    np.savez_compressed(OUT, r=r, sparse_counts=sp[0], sparse_l=sp[1], sparse_norm=sp[2], sparse_off=sp[3],
                        c9_counts=c9[0], c9_l=c9[1], c9_norm=c9[2], c9_off=c9[3], c9_starts=c9[4],
                        threads=oracle.host_threads())
    print(f"wrote {OUT} in {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
