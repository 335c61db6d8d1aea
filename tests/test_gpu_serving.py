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
    srv = serving.Server(slots=2, max_inflight=2)
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
