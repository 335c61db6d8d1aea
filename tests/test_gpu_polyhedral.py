"""Polyhedral homotopies on the GPU (phc_make_polyhedral_homotopy,
phc_polyhedral_starts, phc_track_polyhedral and the pipelined
phc_solve_polyhedral through the C ABI, Section 2.2) against the oracle: the
start solutions of every cell, the tracked endpoints path by path, the
paper's Example 3.1 pipeline (mixed volume 61, then the coefficient-parameter
homotopy of Section 2.3 to the embedded system: 6 paths diverge, 55 start
the cascade), and a random cyclic 7 copy whose 924 roots the total-degree
homotopy does not all reach."""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import mixed as M
import paper_1804_03807_gb300 as P
from workloads import (configs, cyclic, embedding_constants, multistep_example, random_lifting, rng_for,
                       unit_gamma, with_random_coefficients)
from tests._checks import match_sets, min_pair_distance, relative_residual

pytestmark = pytest.mark.gpu
GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_examples.json")))


def _cells_both(g, lift):
    """The library's cells (in its order) and the oracle's own, which must be
    the same set; returns (lib cells array, oracle cells in lib order)."""
    cells, vols, mv = P.phc_mixed_cells(g, lift)
    ref = {c.pairs: c for c in M.mixed_cells(g, lift)}
    keys = [tuple(tuple(int(t) for t in pr) for pr in c) for c in cells]
    assert set(keys) == set(ref)
    return cells, [ref[k] for k in keys]


def _polyhedral_parity(g, lift, tol=1e-10):
    """Starts and endpoints of every cell against the oracle's (the oracle
    tracks from its own binomial solutions); returns the library's outputs
    and the oracle's endpoints in the library's path order."""
    cells, ocells = _cells_both(g, lift)
    h = P.phc_make_polyhedral_homotopy(g, lift, cells)
    n_paths = P.phc_num_paths(h)
    assert n_paths == sum(c.volume for c in ocells)
    starts = P.polyhedral_starts(h).cpu().numpy().T
    r = P.track_polyhedral(h)
    x, cls = r.x.cpu().numpy().T, r.cls.cpu().numpy()
    x_oracle = np.zeros_like(x)
    off = 0
    for cell in ocells:
        V = cell.volume
        So = M.binomial_starts(g, cell)
        ra, rb, d = match_sets(starts[off:off + V], So)
        assert d.max() <= 1e-12, d.max()
        xo, co, _ = oracle.track(oracle.polyhedral_homotopy(g, M.cell_powers(g, lift, cell)), starts=So[rb])
        assert np.array_equal(cls[off:off + V][ra], co)
        e = np.max(np.abs(x[off:off + V][ra] - xo), axis=1) / (1 + np.max(np.abs(xo), axis=1))
        assert e.max() <= tol, e.max()
        x_oracle[off + ra] = xo
        off += V
    return h, cells, x, cls, r, x_oracle


def _distinct(X, tol=1e-6):
    """One row per cluster of rows within tol (1 + norm) of each other."""
    keep = []
    for x in X:
        if not any(np.max(np.abs(x - y)) <= tol * (1 + np.max(np.abs(y))) for y in keep):
            keep.append(x)
    return np.array(keep).reshape(-1, X.shape[1])


@pytest.mark.parametrize("n,seed", [(4, 500), (5, 501)])
def test_polyhedral_starts_and_paths_equal_the_oracles(n, seed):
    g = with_random_coefficients(cyclic(n), rng_for(seed))
    lift = random_lifting(rng_for(seed + 1), g.n_terms)
    h, cells, x, cls, r, _ = _polyhedral_parity(g, lift)
    assert np.all(cls == P.PHC_REGULAR)
    assert np.max(relative_residual(g, x)) < 1e-12
    assert min_pair_distance(x) > 1e-6
    # the pipelined solver makes the same cells in the same order: same bits
    s = P.solve_polyhedral(g, lift, max_paths=x.shape[0] + 3)
    assert np.array_equal(s.x.cpu().numpy().T, x) and np.array_equal(s.cls.cpu().numpy(), cls)


def test_example_3_1_polyhedral_then_parameter_continuation():
    """Section 2.2 then Section 2.3 on the top dimensional system of
    Example 3.1: 61 polyhedral paths solve a random coefficient system with
    its supports, and the coefficient-parameter homotopy carries them to the
    embedded system, where 6 diverge and 55 remain (1 with z_3 = 0, 54 with
    z_3 != 0)."""
    gold = GOLDEN["example_3_1_top_mixed_volume"]
    gold31 = GOLDEN["example_3_1_cascade"]
    D = gold["top_dim"]
    gammas, hyper = embedding_constants(rng_for(510), 4, 4, D)
    E = oracle.embed(multistep_example(), D, gammas, hyper)
    g = with_random_coefficients(E, rng_for(511))
    lift = random_lifting(rng_for(512), g.n_terms)
    h, cells, x, cls, r, x_oracle = _polyhedral_parity(g, lift)
    assert x.shape[0] == gold["mixed_volume"]
    assert np.all(cls == P.PHC_REGULAR)
    gamma = unit_gamma(rng_for(513))
    hp = P.phc_make_parameter_homotopy(E, g.coefs, gamma)
    rp = P.track_from(hp, r.x)
    xe, ce = rp.x.cpu().numpy().T, rp.cls.cpu().numpy()
    finite = (ce == P.PHC_REGULAR) | (ce == P.PHC_SINGULAR)
    fin = _distinct(xe[finite])
    assert fin.shape[0] == gold["cascade_starts"]
    # a regular root ends exactly one path: a path that ends on a root another
    # path reached left its own path near t = 1 while diverging
    jumped = int(finite.sum()) - fin.shape[0]
    assert int((ce == P.PHC_AT_INFINITY).sum()) + jumped == gold["diverged"]
    z = np.abs(fin[:, -1])
    assert int((z < 1e-8).sum()) == gold31["top_slack_zero"]
    assert int((z >= 1e-8).sum()) == gold31["top_slack_nonzero"]
    # the oracle's coefficient-parameter homotopy from its own polyhedral
    # endpoints; which diverging paths end at infinity and which jump near
    # t = 1 is not stable under rounding, the distinct roots and the sum are
    xo, co, _ = oracle.track(oracle.parameter_homotopy(E, g.coefs, gamma), starts=x_oracle)
    fin_o = (co == 0) | (co == 1)
    fo = _distinct(xo[fin_o])
    assert fo.shape[0] == fin.shape[0]
    assert int((co == 2).sum()) + int(fin_o.sum()) - fo.shape[0] == gold["diverged"]
    _, _, d = match_sets(fin, fo)
    assert d.max() <= 1e-10


def test_random_cyclic7_copy_all_924_roots():
    """A copy of the benchmark batch whose total-degree paths miss an orbit
    of 7 roots of large norm: the polyhedral homotopy reaches all 924 roots,
    regular and distinct, and they contain every regular endpoint of the
    oracle's total-degree homotopy."""
    w = configs.cyclic7_batch()
    g, gamma = w.systems[8], w.gammas[8]
    lift = random_lifting(rng_for(520), g.n_terms)
    cells, _, mv = P.phc_mixed_cells(g, lift)
    assert mv == 924
    h = P.phc_make_polyhedral_homotopy(g, lift, cells)
    r = P.track_polyhedral(h)
    x, cls = r.x.cpu().numpy().T, r.cls.cpu().numpy()
    assert np.all(cls == P.PHC_REGULAR)
    assert np.max(relative_residual(g, x)) < 1e-12
    assert min_pair_distance(x) > 1e-6
    xt, ct, _ = oracle.track(oracle.total_degree(g, gamma))
    reg = xt[ct == 0]
    assert reg.shape[0] < 924
    ra, rb, d = match_sets(reg, x)
    assert d.max() <= 1e-9
    missed = np.setdiff1d(np.arange(924), rb)
    assert np.max(np.abs(x[missed])) > 50  # the roots of large norm
    s = P.solve_polyhedral(g, lift, max_paths=924)
    assert np.array_equal(s.x.cpu().numpy().T, x)


@pytest.mark.parametrize("n,seed,G", [(5, 540, 32), (7, 541, 16), (6, 542, 8)])
def test_grouped_and_one_thread_trackers_give_the_same_bits(n, seed, G):
    """A group of G lanes per path (tail_path) and one thread per path run
    the same operations in the same order."""
    g = with_random_coefficients(cyclic(n), rng_for(seed))
    lift = random_lifting(rng_for(seed + 1), g.n_terms)
    cells, _, mv = P.phc_mixed_cells(g, lift)
    h = P.phc_make_polyhedral_homotopy(g, lift, cells)
    one = P.track_polyhedral(h, opts=P.phc_default_opts(group_paths=-1))
    grp = P.track_polyhedral(h, opts=P.phc_default_opts(group_paths=1, tail_threads=G))
    auto = P.track_polyhedral(h)
    for r in (grp, auto):
        assert np.array_equal(r.x.cpu().numpy(), one.x.cpu().numpy())
        assert np.array_equal(r.cls.cpu().numpy(), one.cls.cpu().numpy())
        a, b = P.stats_numpy(r.stats), P.stats_numpy(one.stats)
        for f in ("n_solve", "n_accept", "n_reject", "stop"):
            assert np.array_equal(a[f], b[f]), f
    assert np.all(one.cls.cpu().numpy() == P.PHC_REGULAR)


def test_polyhedral_handle_edges():
    import torch
    g = with_random_coefficients(cyclic(4), rng_for(530))
    lift = random_lifting(rng_for(531), g.n_terms)
    cells, _, mv = P.phc_mixed_cells(g, lift)
    h = P.phc_make_polyhedral_homotopy(g, lift, cells)
    assert P.phc_num_paths(h) == mv == 16
    o = P.phc_default_opts()
    x = torch.zeros((4, 16), dtype=torch.complex128, device="cuda")
    c = torch.zeros(16, dtype=torch.int8, device="cuda")
    with pytest.raises(P.PhcError, match="phc_track_polyhedral"):
        P.phc_track_paths(h, 0, 16, o, x, c)
    with pytest.raises(P.PhcError, match="outside"):
        P.phc_track_polyhedral(h, 10, 7, o, x, c)
    P.phc_track_polyhedral(h, 0, 0, o, x, c)  # empty range
    ht = P.phc_make_homotopy(g, 1.0)
    with pytest.raises(P.PhcError, match="not a polyhedral"):
        P.phc_track_polyhedral(ht, 0, 1, o, x, c)
    # single paths at both ends of the range give the values of the full call
    full = P.track_polyhedral(h)
    for p in (0, 15):
        one = P.track_polyhedral(h, first=p, n_paths=1)
        assert torch.equal(one.x[:, 0], full.x[:, p])
    # the pipelined solver reports a mixed volume above max_paths
    with pytest.raises(P.PhcError, match="exceeds max_paths"):
        P.solve_polyhedral(g, lift, max_paths=15)
    # a choice of pairs that the oracle's exact test rejects is rejected too
    sup = M._supports(g)
    w = [int(v) for v in lift]
    off0, A0 = sup[0]
    rest = [(i, int(cells[0, i, 0]) - sup[i][0], int(cells[0, i, 1]) - sup[i][0]) for i in range(1, 4)]
    for a in range(A0.shape[0]):
        for b in range(a + 1, A0.shape[0]):
            if M._exact_cell(sup, w, [(0, a, b)] + rest) is None:
                bad = cells[:1].copy()
                bad[0, 0] = (off0 + a, off0 + b)
                with pytest.raises(P.PhcError, match="not a fine mixed cell"):
                    P.phc_make_polyhedral_homotopy(g, lift, bad)
                return
    pytest.fail("every pair of equation 0 completes the cell")


@pytest.mark.parametrize("n", [7, 8])
def test_polyhedral_full_size_against_the_stored_oracle(n):
    """The random cyclic 7 and 8 systems of the polyhedral benchmark, whole:
    the library's cells are the oracle's (stored by
    tests/golden/make_polyhedral_expected.py, which calls only the oracle),
    and the pipelined solver's endpoints are the oracle's polyhedral
    endpoints one to one within 1e-10, all regular."""
    from scipy.spatial import cKDTree
    gold = np.load(os.path.join(os.path.dirname(__file__), "golden", "polyhedral_expected.npz"))
    g = with_random_coefficients(cyclic(n), rng_for(600 + n))
    lift = random_lifting(rng_for(610 + n), g.n_terms)
    cells, vols, mv = P.phc_mixed_cells(g, lift)
    assert mv == int(gold[f"mixed_volume_{n}"])
    mine = sorted(tuple(tuple(int(t) for t in pr) for pr in c) for c in cells)
    theirs = sorted(tuple(tuple(int(t) for t in pr) for pr in c) for c in gold[f"pairs_{n}"])
    assert mine == theirs
    r = P.solve_polyhedral(g, lift, mv)
    x, cls = r.x.cpu().numpy().T, r.cls.cpu().numpy()
    assert np.array_equal(np.bincount(cls, minlength=4), gold[f"counts_{n}"])
    xo = gold[f"x_{n}"]
    tree = cKDTree(np.concatenate([xo.real, xo.imag], axis=1))
    d, idx = tree.query(np.concatenate([x.real, x.imag], axis=1), k=1)
    rel = d / (1.0 + np.abs(xo[idx]).max(axis=1))
    assert rel.max() <= 1e-10, rel.max()
    assert len(np.unique(idx)) == mv  # one to one


def test_polyhedral_one_and_two_unknowns():
    """One unknown: the cells are the lower hull's edges of the lifted
    exponents and the paths end at the polynomial's roots (companion matrix
    eigenvalues); two unknowns, sparse: the total-degree homotopy's roots."""
    from workloads import univariate
    rng = rng_for(550)
    c = rng.normal(size=7) + 1j * rng.normal(size=7)
    s = univariate(c)
    lift = random_lifting(rng_for(551), s.n_terms)
    r = P.solve_polyhedral(s, lift, 6)
    x, cls = r.x.cpu().numpy().T, r.cls.cpu().numpy()
    assert x.shape[0] == 6 and np.all(cls == P.PHC_REGULAR)
    _, _, d = match_sets(x, np.roots(c[::-1])[:, None])
    assert d.max() <= 1e-12
    from workloads import PolySystem
    exps = np.array([[0, 0], [2, 1], [1, 3], [0, 2], [0, 0], [3, 0], [1, 1], [0, 1]], dtype=np.uint8)
    s2 = PolySystem(2, 2, np.array([4, 4]), exps, rng.normal(size=8) + 1j * rng.normal(size=8))
    lift2 = random_lifting(rng_for(552), s2.n_terms)
    cells, _, mv = P.phc_mixed_cells(s2, lift2)
    assert mv == M.mixed_volume(M.mixed_cells(s2, lift2))
    r2 = P.solve_polyhedral(s2, lift2, mv)
    x2, c2 = r2.x.cpu().numpy().T, r2.cls.cpu().numpy()
    xt, ct, _ = oracle.track(oracle.total_degree(s2, unit_gamma(rng_for(553))))
    reg = xt[ct == 0]
    assert np.all(c2 == P.PHC_REGULAR) and reg.shape[0] == mv
    _, _, d2 = match_sets(x2, reg)
    assert d2.max() <= 1e-9


def test_random_cyclic11_all_184756_roots():
    """Random-coefficient cyclic 11 by the pipelined polyhedral solve (cells on
    the host threads while the GPU tracks the paths of the cells made so far,
    Section 2.2, Figure 2): the mixed volume is the number of roots of cyclic
    n for prime n, C(2n - 2, n - 1) = C(20, 10) = 184,756 (the roots of cyclic
    7, 924 = C(12, 6), are pinned the same way), where the total-degree
    homotopy would track 11! = 39,916,800 paths.  All but a few paths end at
    regular roots, distinct and with small residuals; the few others fall
    under the at-infinity readings -- on this system 10 end at t = 1 just
    beyond the endpoint bound (norms 1.03e4 to 1.30e4).  11 start solutions
    have norm 7.9e6, beyond diverge_norm: the polyhedral divergence bound is
    relative to the start, and they reach regular roots."""
    from math import comb
    from tests._checks import min_pair_distance_large
    g = with_random_coefficients(cyclic(11), rng_for(911))
    lift = random_lifting(rng_for(961), g.n_terms)
    r = P.solve_polyhedral(g, lift, comb(20, 10))
    x, c = r.x.cpu().numpy().T, r.cls.cpu().numpy()
    st = P.stats_numpy(r.stats)
    assert x.shape[0] == comb(20, 10) == 184756
    reg = c == P.PHC_REGULAR
    assert reg.sum() >= 184756 - 64, np.bincount(c, minlength=4)
    o = P.phc_default_opts()
    # diverged (stop code 1), beyond the endpoint bound, or growing at the end: the
    # at-infinity readings
    far = (st["stop"] == 1) | (st["norm_x"] > o.endpoint_inf_norm) | (st["grew"] != 0)
    assert np.all(c[~reg] == P.PHC_AT_INFINITY) and np.all(far[~reg])
    xr = x[reg]
    res = np.concatenate([relative_residual(g, xr[k:k + 8192]) for k in range(0, xr.shape[0], 8192)])
    assert res.max() <= 1e-12, res.max()
    assert min_pair_distance_large(xr, 1e-6) > 1e-6
