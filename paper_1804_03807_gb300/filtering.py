"""The filters of Section 4.2 (Figures 4 and 5) on the GPU.

The cascade of Section 3.1 leaves at every dimension k candidate generic
points: the finite endpoints with z_k = 0 (at dimension 0 every finite
endpoint is a candidate isolated solution).  Regular candidates are kept;
singular ones may lie on a higher-dimensional set, so each is tested, from
the top dimension down, with the homotopy membership test of Section 4.1
(phc_membership_test: one launch tracks every tested point's copy of the
witness points) and dropped when it lies on one.  What is kept at dimension
k is the witness set of dimension k.  Only the selection of candidates (a
few class and slack tests on small arrays) runs on the host; every path is
tracked in libphc.so.
"""
from __future__ import annotations

import numpy as np

from ._lib import PHC_REGULAR, PHC_SINGULAR


def _slack_zero(x: np.ndarray, j: int, tol: float = 1e-8) -> np.ndarray:
    a = np.maximum(np.abs(x.real), np.abs(x.imag))
    return a[:, j] <= tol * (1.0 + a.max(axis=1))


def filter_candidates(levels: dict, n_var_orig: int, tol: float = 1e-3, opts=None):
    """levels[k] = (E_k lists, x [n + k, P] complex128 CUDA tensor, cls [P]
    int8 CUDA tensor): the endpoints of the cascade at dimension k (the top
    dimension D, then D-1, ..., 0; E_0 is the original system).  Returns
    (witness sets {k: points [m, n + k] numpy}, isolated points [.., n]
    numpy, stages [(level, dimension tested against, paths, removed)])."""
    import torch
    from . import membership
    D = max(levels)
    witness, stages = {}, []
    isolated = None
    for k in range(D, -1, -1):
        E, xd, cd = levels[k]
        x = xd.cpu().numpy().T
        cls = cd.cpu().numpy()
        finite = (cls == PHC_REGULAR) | (cls == PHC_SINGULAR)
        cand = finite & (_slack_zero(x, n_var_orig + k - 1) if k >= 1 else np.ones(len(cls), bool))
        keep = x[cand & (cls == PHC_REGULAR)]
        sus = x[cand & (cls == PHC_SINGULAR)]
        for kk in range(D, k, -1):
            if len(sus) == 0:
                break
            Ekk, W = witness[kk]
            if len(W) == 0:
                continue
            Wd = torch.from_numpy(np.ascontiguousarray(W.T)).to(xd.device)
            on, _ = membership(Ekk, kk, Wd, sus[:, :n_var_orig], tol, opts)
            stages.append((k, kk, len(sus) * len(W), int(on.sum())))
            sus = sus[~on]
        kept = np.concatenate([keep, sus]) if len(sus) else keep
        if k >= 1:
            witness[k] = (E, kept)
        else:
            isolated = kept
    return {k: w for k, (E, w) in witness.items()}, isolated, stages
