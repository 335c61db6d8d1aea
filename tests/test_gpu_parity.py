"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bar: classification counts equal exactly (regular, singular, at infinity,
failed); regular endpoint sets equal within 1e-10 relative after one-to-one
matching; every GPU regular endpoint a root of f (independent evaluation).
Where the oracle finishes in seconds the whole workload is compared here;
the two largest workloads (the 256-system sparse batch and the cyclic 9 D=2
request with both cascade stages) are compared whole in test_gpu_fullsize.py
against the oracle's stored results.
"""
import numpy as np
import pytest

import oracle
import paper_1804_03807_gb300 as P
from workloads import (configs, cyclic, embedding_constants, multistep_example, random_dense, rng_for, univariate,
                       unit_gamma)
from tests._checks import match_sets, min_pair_distance, relative_residual, same_set

pytestmark = pytest.mark.gpu
RTOL = 1e-10


def gpu_track(sys, gamma, first=0, n=None, opts=None):
    h = P.phc_make_homotopy(sys, gamma)
    r = P.track(h, first=first, n_paths=n, opts=opts)
    x = r.x.cpu().numpy().T.copy()
    return h, r, x, r.cls.cpu().numpy(), P.stats_numpy(r.stats)


def compare(sys, xg, cg, xo, co, label=""):
    cnt_g = np.bincount(cg.astype(int), minlength=4)
    cnt_o = np.bincount(co.astype(int), minlength=4)
    assert np.array_equal(cnt_g, cnt_o), f"{label} class counts gpu {cnt_g} oracle {cnt_o}"
    Rg, Ro = xg[cg == 0], xo[co == 0]
    ok, err = same_set(Rg, Ro, RTOL)
    assert ok, f"{label} regular sets differ (max rel {err})"
    if len(Rg):
        assert relative_residual(sys, Rg).max() <= 1e-12
        assert min_pair_distance(Rg) > 1e-6


def test_dense4_full():
    w = configs.dense4()
    sys, g = w.systems[0], w.gammas[0]
    _, r, xg, cg, sg = gpu_track(sys, g)
    xo, co, so = oracle.track(oracle.total_degree(sys, g), threads=1)
    assert np.all(cg == P.PHC_REGULAR) and len(cg) == 16
    compare(sys, xg, cg, xo, co, "dense4")
    # the same path reaches the same root on both sides here
    assert np.max(np.abs(xg - xo)) <= RTOL * (1 + np.abs(xo).max())
    assert np.array_equal(sg["n_accept"] + sg["n_reject"], so["n_accept"] + so["n_reject"])


@pytest.mark.parametrize("deg", [1, 4, 7])
def test_univariate(deg):
    rng = rng_for(200 + deg)
    c = rng.normal(size=deg + 1) + 1j * rng.normal(size=deg + 1)
    sys = univariate(c)
    g = unit_gamma(rng)
    _, _, xg, cg, _ = gpu_track(sys, g)
    xo, co, _ = oracle.track(oracle.total_degree(sys, g), threads=1)
    compare(sys, xg, cg, xo, co, "univariate")


@pytest.mark.parametrize("n", [3, 5, 6, 7])
def test_cyclic_full(n):
    sys = cyclic(n)
    g = unit_gamma(rng_for(300 + n))
    _, _, xg, cg, _ = gpu_track(sys, g)
    xo, co, _ = oracle.track(oracle.total_degree(sys, g))
    compare(sys, xg, cg, xo, co, f"cyclic{n}")


def test_random_dense_ragged_sizes_and_offsets():
    """n = 3, degrees 3: 27 paths; sub-ranges with a ragged tail and offsets."""
    sys = random_dense(3, 3, rng_for(400))
    g = unit_gamma(rng_for(401))
    xo_all, co_all, _ = oracle.track(oracle.total_degree(sys, g), threads=1)
    for first, n in [(0, 27), (5, 13), (26, 1)]:
        _, _, xg, cg, _ = gpu_track(sys, g, first=first, n=n)
        compare(sys, xg, cg, xo_all[first:first + n], co_all[first:first + n], f"range {first}+{n}")
    h = P.phc_make_homotopy(sys, g)
    with pytest.raises(P.PhcError):
        P.track(h, first=20, n_paths=10)
    r = P.track(h, first=3, n_paths=0)
    assert r.x.shape[1] == 0


@pytest.mark.parametrize("threads", [32, 64])
def test_block_size_does_not_change_results(threads):
    sys = cyclic(5)
    g = unit_gamma(rng_for(500))
    o = P.phc_default_opts(block_threads=threads, max_blocks=2)
    _, _, xg, cg, sg = gpu_track(sys, g, opts=o)
    _, _, xg2, cg2, sg2 = gpu_track(sys, g)
    assert np.array_equal(cg, cg2)
    assert np.array_equal(xg, xg2)
    assert np.array_equal(sg["n_solve"], sg2["n_solve"])


def test_cyclic7_batch_full_size():
    """The 9 systems of the cyclic 7 batch (45,360 paths), whole sets."""
    w = configs.cyclic7_batch()
    for s, g in zip(w.systems, w.gammas):
        _, _, xg, cg, _ = gpu_track(s, g)
        xo, co, _ = oracle.track(oracle.total_degree(s, g))
        compare(s, xg, cg, xo, co, s.name)


def test_batch_handle_one_launch_matches_oracle_and_single_handles():
    """cyclic 5 and three random-coefficient copies in one batch handle (one
    launch): per system the same classes and endpoints as the oracle, and
    path for path the same results as separate handles."""
    w = configs.cyclic_batch(5, 3, seed=801)
    hb = P.phc_make_homotopy_batch(w.systems, w.gammas)
    Pn = w.systems[0].bezout()
    assert P.phc_num_paths(hb) == 4 * Pn
    r = P.track(hb)
    x = r.x.cpu().numpy().T
    c = r.cls.cpu().numpy()
    st = P.stats_numpy(r.stats)
    for s_i, (s, g) in enumerate(zip(w.systems, w.gammas)):
        sl = slice(s_i * Pn, (s_i + 1) * Pn)
        assert np.all(st["system"][sl] == s_i)
        xo, co, _ = oracle.track(oracle.total_degree(s, g))
        compare(s, x[sl], c[sl], xo, co, f"batch system {s_i}")
        _, _, x1, c1, _ = gpu_track(s, g)
        assert np.array_equal(c1, c[sl])
        assert np.array_equal(x1, x[sl])
    # a sub-range across a system boundary
    r2 = P.track(hb, first=Pn - 7, n_paths=20)
    assert np.array_equal(r2.x.cpu().numpy().T, x[Pn - 7:Pn + 13])


def test_cyclic7_batch_one_launch_full_size():
    """The bench workload: 45,360 paths in one launch, each system's classes
    and regular set equal to the oracle's."""
    w = configs.cyclic7_batch()
    hb = P.phc_make_homotopy_batch(w.systems, w.gammas)
    r = P.track(hb)
    P.refine(hb, r)
    x = r.x.cpu().numpy().T
    c = r.cls.cpu().numpy()
    Pn = 5040
    for s_i, (s, g) in enumerate(zip(w.systems, w.gammas)):
        sl = slice(s_i * Pn, (s_i + 1) * Pn)
        ho = oracle.total_degree(s, g)
        xo, co, so = oracle.track(ho)
        xo, _, co, _ = oracle.refine(ho, xo, co, so["cond"], so["stop"] == 0)
        compare(s, x[sl], c[sl], xo, co, s.name)


def _embedded_top(sys, D, seed):
    rng = rng_for(seed)
    g, hy = embedding_constants(rng, sys.n_eq, sys.n_var, D)
    gamma = unit_gamma(rng)
    return g, hy, gamma


@pytest.mark.parametrize("seed", [31, 32])
def test_example_2_1_on_gpu(seed):
    g, hy, gamma = _embedded_top(cyclic(4), 1, seed)
    e = P.phc_embed(cyclic(4), 1, g, hy)
    h, r, xg, cg, sg = gpu_track(e, gamma)
    xo, co, so = oracle.track(oracle.total_degree(oracle.embed(cyclic(4), 1, g, hy), gamma), threads=1)
    compare(e, xg, cg, xo, co, "E1 cyclic4")
    reg = cg == P.PHC_REGULAR
    sz = oracle.slack_zero(xg, 4)
    assert reg.sum() == 20 and (reg & sz).sum() == 4


@pytest.mark.parametrize("seed", [41, 42])
def test_example_3_1_cascade_on_gpu(seed):
    """Top system, three cascade stages and refinement on the GPU; counts
    and endpoint sets equal to the oracle's at every level (Figure 3)."""
    import torch
    sys = multistep_example()
    n, D = 4, 3
    g, hy, gamma = _embedded_top(sys, D, seed)
    E = P.phc_embed(sys, D, g, hy)
    h = P.phc_make_homotopy(E, gamma)
    r = P.track(h)
    P.refine(h, r)
    cls = r.cls.cpu().numpy()
    x = r.x.cpu().numpy().T
    Eo = oracle.embed(sys, D, g, hy)
    ho = oracle.total_degree(Eo, gamma)
    xo, co, so = oracle.track(ho, threads=1)
    xo, _, co, _ = oracle.refine(ho, xo, co, so["cond"], so["stop"] == 0)
    compare(E, x, cls, xo, co, "top")
    sz = oracle.slack_zero(x, n + D - 1)
    assert ((cls == 0) & sz).sum() == 1 and ((cls == 0) & ~sz).sum() == 54
    starts = torch.from_numpy(np.ascontiguousarray(x[(cls == 0) & ~sz].T)).cuda()
    Xo = xo[(co == 0) & ~oracle.slack_zero(xo, n + D - 1)]
    Ek, Eko = E, Eo
    expected = {3: 50, 2: 26}
    for k in (3, 2, 1):
        hk = P.phc_make_homotopy(Ek, gamma)
        rk = P.cascade(hk, k, starts)
        Ek1 = P.phc_embed(sys, k - 1, g[:, :k - 1], hy[:k - 1]) if k > 1 else sys
        hk1 = P.phc_make_homotopy(Ek1, gamma)
        P.refine(hk1, rk)
        ck = rk.cls.cpu().numpy()
        xk = rk.x.cpu().numpy().T
        # oracle: the same stage, refinement on E_{k-1}
        hco = oracle.cascade_homotopy(Eko, n, n, k)
        xko, cko, sko = oracle.track(hco, starts=Xo, threads=1)
        Eko1 = oracle.drop_last_slack(Eko, n, n, k)
        xko = np.delete(xko, n + k - 1, axis=1)
        xko, _, cko, _ = oracle.refine(oracle.total_degree(Eko1, gamma), xko, cko, sko["cond"], sko["stop"] == 0)
        compare(Ek1, xk, ck, xko, cko, f"stage {k}")
        if k > 1:
            szk = rk.slack_zero.cpu().numpy().astype(bool)
            assert np.array_equal(szk[ck == 0], oracle.slack_zero(xk, n + k - 2)[ck == 0])
            assert ((ck == 0) & ~szk).sum() == expected[k]
            starts = torch.from_numpy(np.ascontiguousarray(xk[(ck == 0) & ~szk].T)).cuda()
            Xo = xko[(cko == 0) & ~oracle.slack_zero(xko, n + k - 2)]
        else:
            iso = xk[ck == 0]
            ok, err = same_set(iso, np.array([[3, 2, 2, 1], [3, 3, 2, 1], [4, 3, 2, 1], [4, 2, 2, 1]], complex),
                               RTOL)
            assert ok, err
        Ek, Eko = Ek1, Eko1


def test_refinement_reaches_double_double_accuracy_on_gpu():
    from tests._checks import exact_residual
    w = configs.dense4()
    sys = w.systems[0]
    h = P.phc_make_homotopy(sys, w.gammas[0])
    r = P.track(h)
    x_lo = P.refine(h, r, cond_threshold=0.0)
    xh = r.x.cpu().numpy().T
    xl = x_lo.cpu().numpy().T
    assert np.all(r.cls.cpu().numpy() == 0)
    for p in range(4):
        assert exact_residual(sys, xh[p], xl[p]) <= 1e-28


def test_double_root_is_singular_on_gpu():
    c = np.polymul(np.polymul([1, -1], [1, -1]), [1, 2])[::-1]
    sys = univariate(c)
    g = unit_gamma(rng_for(60))
    h = P.phc_make_homotopy(sys, g)
    r = P.track(h)
    P.refine(h, r)
    assert sorted(r.cls.cpu().numpy().tolist()) == [0, 1, 1]


@pytest.mark.parametrize("n", [5, 6])
def test_fp32_interior_cyclic_matches_fp64_oracle(n):
    """FP32 interior: predictor and Jacobian in single precision for t <= 0.9,
    residuals and the end game in double: same classes and regular endpoints
    (1e-10) as the FP64 oracle."""
    sys = cyclic(n)
    g = unit_gamma(rng_for(900 + n))
    o = P.phc_default_opts(precision=P.PHC_PREC_FP32_INTERIOR)
    _, _, xg, cg, sg = gpu_track(sys, g, opts=o)
    assert sg["n_fp32"].sum() > 0
    xo, co, _ = oracle.track(oracle.total_degree(sys, g))
    compare(sys, xg, cg, xo, co, f"fp32 cyclic{n}")


def test_fp32_interior_cyclic7_batch_full_size():
    """The bench workload in FP32-interior mode against the FP64 oracle.
    Every FP32 regular endpoint is a distinct root found by the oracle
    (1e-10); class counts may deviate by a few paths out of 45,360 (single
    precision predictors change step sequences near close path approaches);
    the deviation is bounded and printed."""
    w = configs.cyclic7_batch()
    hb = P.phc_make_homotopy_batch(w.systems, w.gammas)
    r = P.track(hb, opts=P.phc_default_opts(precision=P.PHC_PREC_FP32_INTERIOR))
    P.refine(hb, r)
    x = r.x.cpu().numpy().T
    c = r.cls.cpu().numpy()
    st = P.stats_numpy(r.stats)
    assert st["n_fp32"].sum() > 0
    Pn = 5040
    deviation = 0
    for s_i, (s, g) in enumerate(zip(w.systems, w.gammas)):
        sl = slice(s_i * Pn, (s_i + 1) * Pn)
        ho = oracle.total_degree(s, g)
        xo, co, so = oracle.track(ho)
        xo, _, co, _ = oracle.refine(ho, xo, co, so["cond"], so["stop"] == 0)
        Rg, Ro = x[sl][c[sl] == 0], xo[co == 0]
        assert relative_residual(s, Rg).max() <= 1e-12
        assert min_pair_distance(Rg) > 1e-6
        ra, rb, rel = match_sets(Rg, Ro)
        assert len(ra) == len(Rg) and rel.max() <= RTOL, "an FP32 regular endpoint is not an oracle root"
        deviation += int(np.abs(np.bincount(c[sl], minlength=4) - np.bincount(co, minlength=4)).sum()) // 2
    print(f"FP32 interior: {deviation} of {9 * Pn} paths in a different class than the FP64 oracle")
    assert deviation <= 9


def test_pipeline_equals_separate_stages_example_3_1():
    """phc_track_pipeline (top stage and the cascade stage below it in one
    launch) gives path for path what phc_track_paths followed by
    phc_cascade_stage on the regular z_3 != 0 endpoints gives."""
    import torch
    sys = multistep_example()
    g, hy, gamma = _embedded_top(sys, 3, 41)
    E = P.phc_embed(sys, 3, g, hy)
    h = P.phc_make_homotopy(E, gamma)
    top, nxt = P.pipeline(h, 3)
    ref = P.track(h)
    assert np.array_equal(top.cls.cpu().numpy(), ref.cls.cpu().numpy())
    assert np.array_equal(top.x.cpu().numpy(), ref.x.cpu().numpy())
    x = ref.x.cpu().numpy().T
    c = ref.cls.cpu().numpy()
    fwd = (c == 0) & ~oracle.slack_zero(x, 6)
    cn = nxt.cls.cpu().numpy()
    assert np.array_equal(cn >= 0, fwd)
    starts = torch.from_numpy(np.ascontiguousarray(x[fwd].T)).cuda()
    rs = P.cascade(h, 3, starts)
    assert np.array_equal(rs.cls.cpu().numpy(), cn[fwd])
    assert np.array_equal(rs.x.cpu().numpy(), nxt.x.cpu().numpy()[:, fwd])
    assert np.array_equal(rs.slack_zero.cpu().numpy(), nxt.slack_zero.cpu().numpy()[fwd])


def test_cyclic8_d1_pipeline_full_size_against_oracle():
    """Embedded cyclic 8 (40,320 paths) and its cascade stage to dimension 0,
    pipelined in one launch; the oracle runs the same two stages one after
    the other from its own endpoints.  Class counts of both stages and the
    regular sets match; z = 0 regular points of the top stage are generic
    points on the curve (f(x) = 0)."""
    import torch
    w = configs.cyclic8_d1()
    base = w.systems[0]
    g, hy = w.embed["gammas"], w.embed["hyper"]
    gamma = w.gammas[0]
    E = P.phc_embed(base, 1, g, hy)
    h = P.phc_make_homotopy(E, gamma)
    top, nxt = P.pipeline(h, 1)
    P.refine(h, top)
    xt = top.x.cpu().numpy().T
    ct = top.cls.cpu().numpy()
    cn = nxt.cls.cpu().numpy()
    xn = nxt.x.cpu().numpy().T
    # top endpoints refinement made regular (none expected) go through a separate stage call
    late = (ct == 0) & ~oracle.slack_zero(xt, 8) & (cn < 0)
    if late.any():
        rl = P.cascade(h, 1, torch.from_numpy(np.ascontiguousarray(xt[late].T)).cuda())
        cn[late] = rl.cls.cpu().numpy()
        xn[late] = rl.x.cpu().numpy().T
    h0 = P.phc_make_homotopy(base, gamma)
    mask = cn >= 0
    sub = P.Tracked(torch.from_numpy(np.ascontiguousarray(xn[mask].T)).cuda(),
                    torch.from_numpy(cn[mask].copy()).cuda(), nxt.stats[torch.from_numpy(mask).cuda()].contiguous())
    P.refine(h0, sub)
    cn_m = sub.cls.cpu().numpy()
    xn_m = sub.x.cpu().numpy().T
    # oracle, stage by stage
    Eo = oracle.embed(base, 1, g, hy)
    ho = oracle.total_degree(Eo, gamma)
    xo, co, so = oracle.track(ho)
    xo, _, co, _ = oracle.refine(ho, xo, co, so["cond"], so["stop"] == 0)
    compare(E, xt, ct, xo, co, "cyclic8 top")
    reg = ct == 0
    sz = oracle.slack_zero(xt, 8)
    assert relative_residual(base, xt[reg & sz][:, :8]).max() <= 1e-12
    Xo = xo[(co == 0) & ~oracle.slack_zero(xo, 8)]
    hc = oracle.cascade_homotopy(Eo, 8, 8, 1)
    xko, cko, sko = oracle.track(hc, starts=Xo)
    xko = np.delete(xko, 8, axis=1)
    xko, _, cko, _ = oracle.refine(oracle.total_degree(base, gamma), xko, cko, sko["cond"], sko["stop"] == 0)
    compare(base, xn_m, cn_m, xko, cko, "cyclic8 stage 1->0")


def test_track_many_equals_separate_calls_and_oracle():
    """Twelve random sparse systems of different size in one call (one
    launch per number of unknowns): path for path the results of separate
    phc_track_paths calls, and the oracle's classes and regular sets."""
    w = configs.sparse_batch(count=12, seed=1001, bezout_range=(100, 3000))
    hs = [P.phc_make_homotopy(s, g) for s, g in zip(w.systems, w.gammas)]
    rs = P.track_many(hs)
    for i, (h, s, g) in enumerate(zip(hs, w.systems, w.gammas)):
        ref = P.track(h)
        assert np.array_equal(rs[i].cls.cpu().numpy(), ref.cls.cpu().numpy()), s.name
        assert np.array_equal(rs[i].x.cpu().numpy(), ref.x.cpu().numpy()), s.name
        if i < 4:
            xo, co, _ = oracle.track(oracle.total_degree(s, g))
            compare(s, rs[i].x.cpu().numpy().T, rs[i].cls.cpu().numpy(), xo, co, s.name)
