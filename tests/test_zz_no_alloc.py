"""phc_track_paths_noalloc against phc_track_paths, through the C ABI.

The no-allocation entry point is for callers that cannot allocate device
memory while they run: a process whose GPU memory is held by another
allocator (a framework's caching allocator that reserved the free memory at
start-up), or a serving loop that allocates everything up front and must not
stall in cudaMalloc afterwards.  It keeps its scratch (the path-queue counter
and, without a stats array, the per-path records) in one static device array
shared by all calls.  Two calls in a row must give the endpoints and classes
of phc_track_paths, within the tolerance of the parity tests.
"""
import numpy as np
import pytest
import torch

import paper_1804_03807_gb300 as P
from workloads import configs, cyclic, rng_for, unit_gamma

pytestmark = pytest.mark.gpu
RTOL = 1e-10


def _outputs(h, n):
    x = torch.empty((h.n, n), dtype=torch.complex128, device="cuda")
    cls = torch.empty(n, dtype=torch.int8, device="cuda")
    return x, cls


def _same(ref, x, cls, st=None):
    xr, cr = ref.x.cpu().numpy(), ref.cls.cpu().numpy()
    xn, cn = x.cpu().numpy(), cls.cpu().numpy()
    assert np.array_equal(cr, cn)
    err = np.max(np.abs(xr - xn) / (1.0 + np.abs(xr)))
    assert err <= RTOL, err
    if st is not None:
        a, b = P.stats_numpy(ref.stats), P.stats_numpy(st)
        for f in ("n_solve", "n_fp32", "n_newton", "stop"):
            assert np.array_equal(a[f], b[f]), f


def test_noalloc_matches_track_paths_on_two_calls_in_a_row():
    sys = cyclic(5)
    h = P.phc_make_homotopy(sys, unit_gamma(rng_for(700)))
    n = P.phc_num_paths(h)
    ref = P.track(h)  # the existing entry point
    torch.cuda.synchronize()
    for call in range(2):
        x, cls = _outputs(h, n)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        P.phc_track_paths_noalloc(h, 0, n, None, x, cls, None)
        torch.cuda.synchronize()
        if call == 1:  # after the per-device set-up of the first call
            assert torch.cuda.mem_get_info()[0] == free_before
        _same(ref, x, cls)


def test_noalloc_scratch_is_reset_between_different_problems():
    """A smaller problem, then the first one again: the shared counter and
    records from the previous call do not leak into the next."""
    w = configs.dense4()
    hs = P.phc_make_homotopy(w.systems[0], w.gammas[0])
    hb = P.phc_make_homotopy(cyclic(5), unit_gamma(rng_for(701)))
    refs = {id(hs): P.track(hs), id(hb): P.track(hb)}
    for h in (hs, hb, hs):
        n = P.phc_num_paths(h)
        x, cls = _outputs(h, n)
        P.phc_track_paths_noalloc(h, 0, n, None, x, cls, None)
        torch.cuda.synchronize()
        _same(refs[id(h)], x, cls)
    # with a caller-owned stats array the records go there
    n = P.phc_num_paths(hb)
    x, cls = _outputs(hb, n)
    st = torch.empty((n, P.STATS_DTYPE.itemsize), dtype=torch.uint8, device="cuda")
    P.phc_track_paths_noalloc(hb, 0, n, None, x, cls, st)
    torch.cuda.synchronize()
    _same(refs[id(hb)], x, cls)
    assert np.array_equal(P.stats_numpy(st)["n_solve"], P.stats_numpy(refs[id(hb)].stats)["n_solve"])


def test_noalloc_rejects_ranges_beyond_its_scratch():
    h = P.phc_make_homotopy(cyclic(9), 1.0)
    n = P._lib.PHC_NOALLOC_MAX_PATHS + 1
    x, cls = _outputs(h, 1)
    with pytest.raises(P.PhcError) as ei:
        P.phc_track_paths_noalloc(h, 0, n, None, x, cls, None)
    assert ei.value.code == P._lib.PHC_EUNSUPPORTED
    assert "PHC_NOALLOC_MAX_PATHS" in str(ei.value)


def _noalloc(h, first, n, opts):
    x, cls = _outputs(h, n)
    st = torch.empty((n, P.STATS_DTYPE.itemsize), dtype=torch.uint8, device="cuda")
    P.phc_track_paths_noalloc(h, first, n, opts, x, cls, st)
    torch.cuda.synchronize()
    return x, cls, st


@pytest.mark.parametrize("precision", [P.PHC_PREC_FP64, P.PHC_PREC_FP32_INTERIOR])
def test_noalloc_sub_range_batch_handle_and_precision(precision):
    """A batch handle (cyclic 5 and two random-coefficient copies), a
    sub-range that starts inside the first system and ends inside the last,
    in double and in FP32-interior arithmetic: classes, endpoints and the
    per-path counters (units, single precision units, Newton steps, stop
    reason) equal those of phc_track_paths; the handle's hand-off counters
    read 0 afterwards."""
    w = configs.cyclic_batch(5, 2, seed=702)
    hb = P.phc_make_homotopy_batch(w.systems, w.gammas)
    o = P.phc_default_opts(precision=precision)
    first, n = 37, P.phc_num_paths(hb) - 37 - 11
    ref = P.track(hb, first=first, n_paths=n, opts=o)
    torch.cuda.synchronize()
    x, cls, st = _noalloc(hb, first, n, o)
    _same(ref, x, cls, st)
    if precision == P.PHC_PREC_FP32_INTERIOR:
        assert P.stats_numpy(st)["n_fp32"].sum() > 0
    assert P.phc_tail_paths(hb) == 0


def test_noalloc_hand_off_beyond_its_record_cap():
    """An early hand-off (tail_drain 0.1) on 5040 paths of a random cyclic 7
    copy would move more paths than the static scratch holds; the call starts
    the hand-off later instead, with the results of phc_track_paths."""
    w = configs.cyclic7_batch()
    h = P.phc_make_homotopy(w.systems[1], w.gammas[1])
    o = P.phc_default_opts(tail_drain=0.1)
    n = P.phc_num_paths(h)
    ref = P.track(h, opts=o)
    torch.cuda.synchronize()
    assert P.phc_tail_paths(h) > P._lib.PHC_NOALLOC_MAX_HANDOFF  # what phc_track_paths handed off
    x, cls, st = _noalloc(h, 0, n, o)
    _same(ref, x, cls, st)
