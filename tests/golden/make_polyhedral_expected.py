"""Writes tests/golden/polyhedral_expected.npz: the oracle's polyhedral solves of
the random cyclic 7 and cyclic 8 systems of the polyhedral benchmark (seeds
600 + n, lifting seeds 610 + n), for the full-size GPU parity test of the
polyhedral tracker.

Calls only the oracle (oracle/) and the seeded input generators (workloads/).
Un-timed; the oracle's exact cell search takes a few minutes:

    python tests/golden/make_polyhedral_expected.py

Stored per system (keys suffixed _7 and _8): the cells (pairs of global term
indices, volumes), the mixed volume, the class counts of the polyhedral paths,
and every endpoint (complex [mixed volume, n]).
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from oracle import mixed as M  # noqa: E402
from workloads import cyclic, random_lifting, rng_for, with_random_coefficients  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "polyhedral_expected.npz")


def main():
    t0 = time.time()
    out = {}
    for n in (7, 8):
        g = with_random_coefficients(cyclic(n), rng_for(600 + n))
        lift = random_lifting(rng_for(610 + n), g.n_terms)
        cells = M.mixed_cells(g, lift)
        print(f"cyclic {n}: {len(cells)} cells, mixed volume {M.mixed_volume(cells)} at {time.time() - t0:.0f} s",
              flush=True)
        starts, x, cls, stats, cell_of = M.track_polyhedral(g, lift, cells)
        out[f"pairs_{n}"] = np.array([c.pairs for c in cells], dtype=np.int32)
        out[f"volumes_{n}"] = np.array([c.volume for c in cells], dtype=np.int64)
        out[f"mixed_volume_{n}"] = M.mixed_volume(cells)
        out[f"counts_{n}"] = np.bincount(cls.astype(np.int64), minlength=4)[:4]
        out[f"x_{n}"] = x
    np.savez_compressed(OUT, **out)
    print(f"wrote {OUT} in {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
