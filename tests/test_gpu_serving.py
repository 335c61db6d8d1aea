"""Continuous batching: requests admitted while others run overlap on the
device, and every request's result equals its result alone (and the
oracle's)."""
import numpy as np
import pytest

import oracle
import paper_1804_03807_gb300 as P
from paper_1804_03807_gb300 import serving
from workloads import configs, cyclic, embedding_constants, rng_for, unit_gamma
from tests._checks import same_set

pytestmark = pytest.mark.gpu


def _mix():
    w = configs.serving(n_requests=16, rate=200.0, seed=1200, bezout_range=(100, 800), big=None)
    reqs = [serving.Request(i, s, g, float(a)) for i, (s, g, a) in
            enumerate(zip(w.systems, w.gammas, w.extra["arrivals"]))]
    rng = rng_for(1201)
    g, hy = embedding_constants(rng, 5, 5, 1)
    reqs.append(serving.Request(len(reqs), cyclic(5), unit_gamma(rng), 0.0, 1, g, hy))
    return reqs


def test_each_result_is_the_same_alone_and_in_the_mix():
    reqs = _mix()
    # the embedded request in chunks of 37 paths (alone: one chunk)
    srv = serving.Server(slots=2, max_inflight=2, big_chunk=37)
    mixed = srv.run(reqs)
    # work overlapped: some request was admitted before an earlier one finished
    assert any(mixed[j].admitted < mixed[i].finished for i in range(len(mixed)) for j in range(len(mixed))
               if j != i and mixed[j].arrival >= mixed[i].arrival)
    for req, r in zip(reqs, mixed):
        alone = serving.solve_alone(req)
        assert len(alone.stages) == len(r.stages) == 1 + req.top_dim
        for (xa, ca), (xm, cm) in zip(alone.stages, r.stages):
            assert np.array_equal(ca, cm), req.rid
            ok = ca >= 0
            assert np.allclose(xa[:, ok], xm[:, ok], rtol=1e-10, atol=0), req.rid
    s = serving.latency_summary(mixed)
    assert s["count"] == len(reqs) and s["p99_s"] >= s["p50_s"] > 0


def test_served_results_match_the_oracle():
    reqs = _mix()
    res = serving.Server(slots=2).run(reqs[:3] + reqs[-1:], realtime=False)
    for req, r in zip(reqs[:3], res[:3]):
        xo, co, _ = oracle.track(oracle.total_degree(req.system, req.gamma))
        x, c = r.stages[0]
        assert np.array_equal(np.bincount(c, minlength=4), np.bincount(co, minlength=4))
        ok, err = same_set(x.T[c == 0], xo[co == 0], 1e-10)
        assert ok, err
    # the embedded request: top stage and the stage to dimension 0
    big = reqs[-1]
    E = oracle.embed(big.system, 1, big.gammas, big.hyper)
    ho = oracle.total_degree(E, big.gamma)
    xo, co, so = oracle.track(ho)
    x, c = res[-1].stages[0]
    assert np.array_equal(np.bincount(c, minlength=4), np.bincount(co, minlength=4))
    starts = xo[(co == 0) & ~oracle.slack_zero(xo, 5)]
    hc = oracle.cascade_homotopy(E, 5, 5, 1)
    xk, ck, _ = oracle.track(hc, starts=starts)
    x1, c1 = res[-1].stages[1]
    sel = c1 >= 0
    assert sel.sum() == len(starts)
    assert np.array_equal(np.bincount(c1[sel], minlength=4), np.bincount(ck, minlength=4))
    ok, err = same_set(x1.T[sel][c1[sel] == 0], np.delete(xk, 5, axis=1)[ck == 0], 1e-10)
    assert ok, err


def test_small_requests_keep_their_latency_beside_the_large_request():
    """600 Poisson small requests (200/s) served alone and then beside the
    cyclic 9 D=2 request (362,880 top-stage paths and two cascade stages)
    arriving first: the small requests' p99 latency stays within 3x of its
    value without the large request, every small result is the same in both
    runs, and the large request's results (computed in chunks on the
    low-priority streams) equal one unchunked launch per stage."""
    import torch
    w = configs.serving(n_requests=600, rate=200.0, seed=5, bezout_range=(100, 1000), big=(9, 2))
    small = [serving.Request(i, s, g, float(a)) for i, (s, g, a) in
             enumerate(zip(w.systems, w.gammas, w.extra["arrivals"]))]
    b = w.extra["big"]
    big = serving.Request(len(small), b["system"], b["gamma"], 0.0, b["top_dim"], b["gammas"], b["hyper"])
    srv = serving.Server(slots=2, max_inflight=4)
    srv.run(small[:8], realtime=False)  # warm-up
    alone = srv.run(small)
    mixed = srv.run(small + [big])
    p99_alone = serving.latency_summary(alone)["p99_s"]
    p99_mixed = serving.latency_summary(mixed[:-1])["p99_s"]
    print(f"small p99 alone {p99_alone:.3f} s, beside cyclic 9 D=2 {p99_mixed:.3f} s; "
          f"cyclic 9 D=2 latency {mixed[-1].latency:.2f} s")
    assert p99_mixed <= 3 * p99_alone
    for ra, rm in zip(alone, mixed[:-1]):
        (xa, ca), (xm, cm) = ra.stages[0], rm.stages[0]
        assert np.array_equal(ca, cm) and np.array_equal(xa, xm)
    # the large request, one launch per stage
    E2 = P.phc_embed(b["system"], 2, b["gammas"], b["hyper"])
    E1 = P.phc_embed(b["system"], 1, b["gammas"][:, :1], b["hyper"][:1])
    h2, h1 = P.phc_make_homotopy(E2, b["gamma"]), P.phc_make_homotopy(E1, b["gamma"])
    top = P.track(h2)
    s2 = P.cascade_from(h2, 2, top)
    s1 = P.cascade_from(h1, 1, s2)
    torch.cuda.synchronize()
    for (xm, cm), ref in zip(mixed[-1].stages, (top, s2, s1)):
        assert np.array_equal(cm, ref.cls.cpu().numpy())
        assert np.array_equal(xm[:, cm >= 0], ref.x.cpu().numpy()[:, cm >= 0])
