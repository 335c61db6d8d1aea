"""Edge cases through the C ABI on the GPU: the largest number of unknowns
(12) in every tracker (double, double double, quad double, forced tail
hand-off and compaction off and on, polyhedral), single paths at the ends of
the range, and empty calls of every entry point."""
import numpy as np
import pytest
import torch

import oracle
import paper_1804_03807_gb300 as P
from workloads import PolySystem, cn01, configs, cyclic, rng_for, unit_gamma
from workloads.systems import all_monomials
from tests._checks import exact_residual_parts, match_sets, relative_residual, same_set

pytestmark = pytest.mark.gpu


def _system12(seed=95):
    """11 random linear equations and one random quadratic in 12 unknowns
    (every monomial present): Bezout number 2."""
    rng = rng_for(seed)
    n = 12
    lin, quad = all_monomials(n, 1), all_monomials(n, 2)
    exps = np.array(lin * 11 + quad, dtype=np.uint8).reshape(-1, n)
    tpe = np.array([len(lin)] * 11 + [len(quad)])
    return PolySystem(n, n, tpe, exps, cn01(rng, exps.shape[0]), name="mixed12")


def test_twelve_unknowns_every_tracker():
    s = _system12()
    g = unit_gamma(rng_for(96))
    h = P.phc_make_homotopy(s, g)
    assert P.phc_num_paths(h) == 2
    xo, co, _ = oracle.track(oracle.total_degree(s, g), threads=1)
    assert np.bincount(co, minlength=4)[0] == 2
    outs = []
    for o in (P.phc_default_opts(tail_drain=0.0, compact=0), P.phc_default_opts(),
              P.phc_default_opts(tail_drain=1e-9, block_threads=32, max_blocks=1)):
        r = P.track(h, opts=o)
        outs.append((r.x.cpu().numpy(), r.cls.cpu().numpy(), r.stats.cpu().numpy()))
    for a in outs[1:]:
        for u, v in zip(outs[0], a):
            assert u.tobytes() == v.tobytes()
    x, c = outs[0][0].T, outs[0][1]
    ok, err = same_set(x[c == 0], xo[co == 0], 1e-10)
    assert ok and relative_residual(s, x[c == 0]).max() <= 1e-12, err
    rd, xlo = P.track_dd(h)
    xd = rd.x.cpu().numpy().T
    assert np.array_equal(rd.cls.cpu().numpy(), c)
    ok, err = same_set(xd[c == 0], xo[co == 0], 1e-10)
    assert ok, err


def test_twelve_unknowns_quad_double_and_polyhedral():
    """The same system in quad double (both endpoints equal to the oracle's
    quad double endpoints within 1e-55 and roots of f to 1e-58 in exact
    arithmetic) and by polyhedral homotopies: the mixed volume of a dense
    system is its Bezout number (2), and the two paths end at the oracle's
    total-degree roots."""
    from fractions import Fraction
    from workloads import random_lifting
    s = _system12()
    g = unit_gamma(rng_for(96))
    h = P.phc_make_homotopy(s, g)
    r, parts = P.track_qd(h)
    pg = np.transpose(parts.cpu().numpy(), (2, 1, 0))
    po, co, _ = oracle.track_qd(oracle.total_degree(s, g))
    assert np.all(r.cls.cpu().numpy() == 0) and np.all(co == 0)
    ra, rb, rel = match_sets(pg[:, :, 0], po[:, :, 0])
    assert len(ra) == 2 and rel.max() <= 1e-10
    for a, b in zip(ra, rb):
        for j in range(12):
            for part in (np.real, np.imag):
                d = sum(Fraction(float(part(v))) - Fraction(float(part(w))) for v, w in zip(pg[a, j], po[b, j]))
                assert abs(float(d)) <= 1e-55 * (1 + np.abs(po[b, :, 0]).max())
        assert exact_residual_parts(s, pg[a]) <= 1e-58
    lift = random_lifting(rng_for(97), s.n_terms)
    _, vols, mv = P.phc_mixed_cells(s, lift)
    assert mv == 2
    rp = P.solve_polyhedral(s, lift, mv)
    xp, cp = rp.x.cpu().numpy().T, rp.cls.cpu().numpy()
    assert np.all(cp == P.PHC_REGULAR)
    ok, err = same_set(xp, po[:, :, 0], 1e-10)
    assert ok and relative_residual(s, xp).max() <= 1e-12, err


def test_single_paths_at_the_ends_and_empty_calls():
    w = configs.cyclic7_batch()
    hb = P.phc_make_homotopy_batch(w.systems[:2], w.gammas[:2])
    total = P.phc_num_paths(hb)
    whole = P.track(hb)
    for first in (0, total - 1):
        r = P.track(hb, first=first, n_paths=1)
        assert np.array_equal(r.x.cpu().numpy()[:, 0], whole.x.cpu().numpy()[:, first])
        assert r.cls.cpu().numpy()[0] == whole.cls.cpu().numpy()[first]
    # empty calls return without work
    e = torch.empty((7, 0), dtype=torch.complex128, device="cuda")
    c = torch.empty(0, dtype=torch.int8, device="cuda")
    P.phc_track_paths(hb, total, 0, None, e, c)
    P.phc_track_paths_dd(hb, 0, 0, None, e, e, c)
    P.phc_track_many([], None, [], [])
    h5 = P.phc_make_homotopy(cyclic(5), 0.6 + 0.8j)
    P.phc_track_from(h5, e[:5], 0, 0, None, e[:5], c)
    P.phc_cascade_stage(h5, 1, e[:5], 0, None, e[:4], c, c)
    on = torch.empty(0, dtype=torch.uint8, device="cuda")
    E = P.phc_embed(cyclic(4), 1)
    P.phc_membership_test(E, 1, torch.zeros((5, 1), dtype=torch.complex128, device="cuda"), np.zeros((0, 4)),
                          1e-3, None, on)
    with pytest.raises(P.PhcError):
        P.phc_track_paths(hb, total, 1, None, e, c)  # beyond the last path
    torch.cuda.synchronize()


def test_fp64_probe_measures_the_derived_peak():
    """The measured FP64 rate lies near the peak derived from the units and
    the clock (152 SMs x 2 FMA per clock x 2 flops x 2.07 GHz = 1.259
    TFLOP/s); bad counts are rejected."""
    v = P.phc_fp64_probe(16, 200_000)
    assert 0.6 * 1.259 <= v <= 1.2 * 1.259, v
    with pytest.raises(P.PhcError):
        P.phc_fp64_probe(0, 10)
    with pytest.raises(P.PhcError):
        P.phc_fp64_probe(4, 0)


@pytest.mark.parametrize("rules,accepted", [((0.01, 0.1, 3), 18), ((0.05, 0.2, 2), 8)])
def test_step_counts_on_a_linear_path_gpu(rules, accepted):
    """The hand-counted steps of the path from x - 1 to x - a (every step
    accepted; the step sizes follow from the expansion rule alone: 18 with
    the default rules, 8 with h_init 0.05, h_max 0.2 and expansion after 2
    accepts), in the one-thread tracker and with the tail hand-off forced."""
    h_init, h_max, after = rules
    for k, a in enumerate((0.5 + 0.25j, -2 + 1j, 3j)):
        s = PolySystem(1, 1, np.array([2]), np.array([[1], [0]], dtype=np.uint8), np.array([1, -a]))
        h = P.phc_make_homotopy(s, unit_gamma(rng_for(720 + k)))
        for drain in (0.0, 1e-9):
            o = P.phc_default_opts(tail_drain=drain)
            o.h_init, o.h_max, o.expand_after = h_init, h_max, after
            r = P.track(h, opts=o)
            st = P.stats_numpy(r.stats)
            assert r.cls.cpu().numpy()[0] == P.PHC_REGULAR
            assert abs(r.x.cpu().numpy()[0, 0] - a) <= 1e-14 * abs(a)
            assert st["n_accept"][0] == accepted and st["n_reject"][0] == 0 and st["t"][0] == 1.0
            assert st["n_solve"][0] == 4 * accepted + st["n_newton"][0]
