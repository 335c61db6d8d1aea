"""The multi-system batching launch as a prepared plan (phc_many_plan_*):
byte for byte the results of phc_track_many, and capturable in a CUDA graph
(a run allocates nothing and does not synchronise with the host)."""
import numpy as np
import pytest
import torch

import paper_1804_03807_gb300 as P
from workloads import configs

pytestmark = pytest.mark.gpu


def _outs(hs):
    out = []
    for h in hs:
        n = P.phc_num_paths(h)
        out.append((torch.empty((h.n, n), dtype=torch.complex128, device="cuda"),
                    torch.empty(n, dtype=torch.int8, device="cuda"),
                    torch.empty((n, P.STATS_DTYPE.itemsize), dtype=torch.uint8, device="cuda")))
    return out


def _host(outs):
    return [(x.cpu().numpy(), c.cpu().numpy(), s.cpu().numpy()) for x, c, s in outs]


def test_plan_equals_track_many_and_replays_in_a_cuda_graph():
    w = configs.sparse_batch(count=12, seed=1001, bezout_range=(100, 3000))
    hs = [P.phc_make_homotopy(s, g) for s, g in zip(w.systems, w.gammas)]
    ref = _host([(r.x, r.cls, r.stats) for r in P.track_many(hs)])
    outs = _outs(hs)
    plan = P.phc_many_plan_create(hs, None, [o[0] for o in outs], [o[1] for o in outs], [o[2] for o in outs])
    P.phc_many_plan_run(plan)
    torch.cuda.synchronize()
    for (a, b) in zip(ref, _host(outs)):
        for u, v in zip(a, b):
            assert np.array_equal(u, v)
    # a plan without stats arrays keeps records of its own
    outs2 = _outs(hs)
    plan2 = P.phc_many_plan_create(hs, None, [o[0] for o in outs2], [o[1] for o in outs2], None)
    P.phc_many_plan_run(plan2)
    torch.cuda.synchronize()
    for (a, b) in zip(ref, _host(outs2)):
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    # captured once, replayed twice
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        P.phc_many_plan_run(plan)
    for _ in range(2):
        for x, c, s in outs:
            x.zero_()
            c.fill_(-7)
            s.zero_()
        g.replay()
        torch.cuda.synchronize()
        for (a, b) in zip(ref, _host(outs)):
            for u, v in zip(a, b):
                assert np.array_equal(u, v)
