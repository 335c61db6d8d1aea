"""The tail kernels and the compaction change nothing but where a path is
finished.

When most threads of a tracking launch have run out of paths, the paths
that are still running move, at the start of their next step, to a kernel
that gives every path a group of threads (opts.tail_drain, opts.tail_threads).
That kernel performs the same floating point operations in the same order, so
endpoints, classes and every per-path statistic must be identical, bit for
bit, to a run without the hand-off.  The same holds for the compaction of
the single-homotopy tracker (opts.compact: running paths move to the lowest
threads of their block once the queue is empty).  Each case runs with both
off; with the compaction alone; with the default; and, for every group size
of the tail kernel, on a one-block grid with a drain fraction so small that
nearly every path is handed off after its first step.
"""
import numpy as np
import pytest

import paper_1804_03807_gb300 as P
from workloads import configs, cyclic, embedding_constants, multistep_example, random_dense, rng_for, unit_gamma

pytestmark = pytest.mark.gpu


def _opts(drain, tiny_grid=False, group=0, compact=1):
    o = P.phc_default_opts()
    o.tail_drain = drain
    o.tail_threads = group
    o.compact = compact
    if tiny_grid:
        o.block_threads = 32
        o.max_blocks = 1
    return o


def _host(r):
    out = [r.x.cpu().numpy(), r.cls.cpu().numpy(), r.stats.cpu().numpy()]
    if r.slack_zero is not None:
        out.append(r.slack_zero.cpu().numpy())
    return out


def _same(a, b, label):
    for u, v in zip(a, b):
        assert u.shape == v.shape
        assert u.tobytes() == v.tobytes(), f"{label}: results differ"


def _three_ways(run, h):
    """Hand-off off, default, and forced with each group size the kernel has
    for this number of unknowns; returns the results and the fewest paths moved."""
    base = _host(run(_opts(0.0, compact=0)))
    assert P.phc_tail_paths(h) == 0
    _same(base, _host(run(_opts(0.0))), "compaction of running paths")
    dflt = _host(run(_opts(0.8)))
    _same(base, dflt, "default drain")
    moved = []
    for group in ([8] if h.n <= 8 else []) + [16, 32]:
        forced = _host(run(_opts(1e-9, tiny_grid=True, group=group)))
        moved.append(P.phc_tail_paths(h))
        _same(base, forced, f"forced hand-off, {group} threads per path")
    return base, min(moved)


@pytest.mark.parametrize("case", ["dense4", "cyclic5", "ragged27", "dense9", "dense10"])
def test_tail_handoff_bit_identical_total_degree(case):
    if case == "dense4":
        w = configs.dense4()
        sys, g = w.systems[0], w.gammas[0]
    elif case == "cyclic5":
        sys, g = cyclic(5), unit_gamma(rng_for(305))
    elif case == "ragged27":
        sys, g = random_dense(3, 3, rng_for(400)), unit_gamma(rng_for(401))
    else:
        # n = 9 and 10 (16 threads per path): all monomials of degree <= 2
        n = int(case[5:])
        rng = rng_for(900 + n)
        sys, g = random_dense(n, 2, rng), unit_gamma(rng)
    h = P.phc_make_homotopy(sys, g)
    (_, cls, _), moved = _three_ways(lambda o: P.track(h, opts=o), h)
    n_paths = P.phc_num_paths(h)
    # a 32-thread grid holds at most 32 paths at once: every path tracked
    # after the queue ran dry and still running moves (most of the last 32)
    assert moved >= min(n_paths, 32) // 2, moved
    assert np.isin(cls, [0, 1, 2, 3]).all()


def test_tail_handoff_bit_identical_batch_handle():
    w = configs.cyclic_batch(n=5, copies=3)
    h = P.phc_make_homotopy_batch(w.systems, w.gammas)
    _, moved = _three_ways(lambda o: P.track(h, opts=o), h)
    assert moved > 0


def test_tail_handoff_bit_identical_cascade_stages():
    """Cascade stages (explicit starts, and starts selected from the previous
    stage's outputs) of Example 3.1 with the top dimension D = 3."""
    import torch
    sys = multistep_example()
    D = 3
    rng = rng_for(41)
    g, hy = embedding_constants(rng, sys.n_eq, sys.n_var, D)
    gamma = unit_gamma(rng)
    E = P.phc_embed(sys, D, g, hy)
    h = P.phc_make_homotopy(E, gamma)
    top = P.track(h, opts=_opts(0.0))
    x = top.x.cpu().numpy().T
    cls = top.cls.cpu().numpy()
    keep = (cls == 0) & (np.abs(x[:, -1]) > 1e-8 * (1 + np.abs(x).max(axis=1)))
    starts = torch.from_numpy(np.ascontiguousarray(x[keep].T)).cuda()
    (xs, cs, _, _), moved = _three_ways(lambda o: P.cascade(h, D, starts, opts=o), h)
    assert moved > 0
    _, moved = _three_ways(lambda o: P.cascade_from(h, D, top, opts=o), h)
    assert moved > 0


def test_tail_handoff_bit_identical_many_systems():
    """phc_track_many (one launch per number of unknowns, a warp per system):
    the multi-system tail kernel leaves results byte-identical too."""
    w = configs.sparse_batch(count=12, seed=1001, bezout_range=(100, 3000))
    hs = [P.phc_make_homotopy(s, g) for s, g in zip(w.systems, w.gammas)]

    def run(o):
        return [_host(r) for r in P.track_many(hs, opts=o)]

    base = run(_opts(0.0))
    for o in (_opts(0.85), _opts(1e-9, tiny_grid=True)):
        for a, b in zip(base, run(o)):
            _same(a, b, "track_many with the tail hand-off")


def _stage_outputs(top, nxt):
    """Host copies of a pipelined launch: the top stage whole, the cascade
    stage on the entries it tracked (cls >= 0; the others are not written)."""
    c2 = nxt.cls.cpu().numpy()
    ok = c2 >= 0
    return [top.x.cpu().numpy(), top.cls.cpu().numpy(), top.stats.cpu().numpy(), c2,
            nxt.x.cpu().numpy()[:, ok], nxt.stats.cpu().numpy()[ok], nxt.slack_zero.cpu().numpy()[ok]]


@pytest.mark.parametrize("D", [1, 3])
def test_tail_handoff_bit_identical_pipeline(D):
    """phc_track_pipeline (top stage and cascade stage in one launch): paths
    handed off in either stage finish in the pipelined tail kernel with the
    same bits, including those that move on to the cascade stage there."""
    sys = multistep_example() if D == 3 else cyclic(5)
    rng = rng_for(50 + D)
    g, hy = embedding_constants(rng, sys.n_eq, sys.n_var, D)
    gamma = unit_gamma(rng)
    h = P.phc_make_homotopy(P.phc_embed(sys, D, g, hy), gamma)
    base = _stage_outputs(*P.pipeline(h, D, opts=_opts(0.0)))
    assert P.phc_tail_paths(h) == 0
    for o in (_opts(0.85), _opts(1e-9, tiny_grid=True)):
        _same(base, _stage_outputs(*P.pipeline(h, D, opts=o)), "pipeline with the tail hand-off")
    assert P.phc_tail_paths(h) > 0


def test_track_paths_replays_in_a_cuda_graph():
    """After one call with the same sizes (which allocates the handle's
    scratch), phc_track_paths issues no allocation and no host
    synchronisation: its launches (counters, tracker, tail, classification)
    capture into a CUDA graph, and each replay gives the same bytes."""
    import torch
    w = configs.cyclic_batch(n=5, copies=3)
    h = P.phc_make_homotopy_batch(w.systems, w.gammas)
    n = P.phc_num_paths(h)
    x = torch.empty((h.n, n), dtype=torch.complex128, device="cuda")
    cls = torch.empty(n, dtype=torch.int8, device="cuda")
    st = torch.empty((n, P.STATS_DTYPE.itemsize), dtype=torch.uint8, device="cuda")
    P.phc_track_paths(h, 0, n, None, x, cls, st)
    torch.cuda.synchronize()
    ref = [x.cpu().numpy(), cls.cpu().numpy(), st.cpu().numpy()]
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        P.phc_track_paths(h, 0, n, None, x, cls, st)
    for _ in range(2):
        x.zero_()
        cls.fill_(-7)
        st.zero_()
        g.replay()
        torch.cuda.synchronize()
        _same(ref, [x.cpu().numpy(), cls.cpu().numpy(), st.cpu().numpy()], "graph replay")
    assert P.phc_tail_paths(h) > 0


def test_tail_handoff_bit_identical_fp32_interior():
    """FP32 interior: only paths whose remaining steps are all double move to
    the tail kernel; the results stay byte-identical."""
    w = configs.cyclic_batch(n=5, copies=3)
    h = P.phc_make_homotopy_batch(w.systems, w.gammas)

    def run(o):
        o.precision = P.PHC_PREC_FP32_INTERIOR
        return P.track(h, opts=o)

    base = _host(run(_opts(0.0, compact=0)))
    assert P.stats_numpy(run(_opts(0.0)).stats)["n_fp32"].sum() > 0
    for o in (_opts(0.0), _opts(0.85), _opts(1e-9, tiny_grid=True)):
        _same(base, _host(run(o)), "FP32 interior with the tail hand-off and the compaction")
    assert P.phc_tail_paths(h) > 0


def test_compaction_bit_identical_on_a_full_cyclic7_system():
    """5040 paths of a random cyclic 7 copy on the full grid: compaction and
    hand-off off, compaction alone, both (the default): the same bytes, and
    with the compaction fewer paths reach the tail kernel."""
    w = configs.cyclic7_batch()
    h = P.phc_make_homotopy(w.systems[1], w.gammas[1])
    base = _host(P.track(h, opts=_opts(0.0, compact=0)))
    _same(base, _host(P.track(h, opts=_opts(0.0))), "compaction")
    _same(base, _host(P.track(h, opts=_opts(0.8, compact=0))), "hand-off")
    moved_plain = P.phc_tail_paths(h)
    _same(base, _host(P.track(h, opts=_opts(0.8))), "compaction and hand-off")
    print(f"paths moved to the tail kernel: {moved_plain} without, {P.phc_tail_paths(h)} with the compaction")
