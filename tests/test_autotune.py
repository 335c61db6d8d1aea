"""The launch-parameter tuner: candidate generation, choice by time, cache.

Its choices cannot change results (tests/test_gpu_tail.py checks that the
launch parameters leave every byte alone), so these tests check the tuner's
own logic on the CPU with a fake workload and clock, and on the GPU that a
tuned call runs and matches the default call.
"""
import pytest

from paper_1804_03807_gb300 import autotune


def test_candidates_respect_the_kernels_group_sizes():
    grid = {"tail_threads": (8, 16, 32), "tail_drain": (0.7, 0.9)}
    small = autotune.candidates(7, grid)
    large = autotune.candidates(11, grid)
    assert len(small) == 6 and len(large) == 4
    assert all(c["tail_threads"] != 8 for c in large)
    assert {(c["tail_threads"], c["tail_drain"]) for c in small} == {(g, d) for g in (8, 16, 32) for d in (0.7, 0.9)}


def test_pick_takes_the_fastest_and_keeps_the_first_on_ties():
    cost = {0.7: 3.0, 0.85: 1.0, 0.95: 1.0}
    calls = []
    cands = [{"tail_drain": d} for d in (0.7, 0.85, 0.95)]
    clock = {"t": 0.0}

    def run(c):
        calls.append(c["tail_drain"])
        clock["t"] = cost[c["tail_drain"]]

    def timer(fn):
        fn()
        return clock["t"]

    best, table = autotune.pick(run, cands, timer=timer, reps=2)
    assert best == {"tail_drain": 0.85}
    assert [t for t, _ in table] == [3.0, 1.0, 1.0]
    assert calls.count(0.7) == 3  # one untimed call and two timed


def test_make_opts_copies_the_base_and_applies_the_candidate():
    import paper_1804_03807_gb300 as P
    base = P.phc_default_opts()
    base.max_steps = 1234
    o = autotune.make_opts(base, {"tail_threads": 16, "block_threads": 128})
    assert o.max_steps == 1234 and o.tail_threads == 16 and o.block_threads == 128
    assert base.tail_threads == 0


@pytest.mark.gpu
def test_tuned_many_call_matches_the_default_call():
    import paper_1804_03807_gb300 as P
    from workloads import configs
    w = configs.sparse_batch(count=10, seed=1001, bezout_range=(100, 2000))
    hs = [P.phc_make_homotopy(s, g) for s, g in zip(w.systems, w.gammas)]
    autotune.clear_cache()
    grid = {"tail_threads": (16, 32), "tail_drain": (0.85, 0.95)}
    o = autotune.tune_many(hs, sample_systems=5, grid=grid)
    assert (o.tail_threads, o.tail_drain) in {(g, d) for g in (16, 32) for d in (0.85, 0.95)}
    assert autotune.tune_many(hs, grid=grid).tail_threads == o.tail_threads  # cached
    tuned = P.track_many(hs, opts=o)
    plain = P.track_many(hs)
    for a, b in zip(tuned, plain):
        assert a.x.cpu().numpy().tobytes() == b.x.cpu().numpy().tobytes()
        assert a.cls.cpu().numpy().tobytes() == b.cls.cpu().numpy().tobytes()
