"""The library's mixed-cell enumeration (host code behind phc_mixed_cells,
Section 2.2) against the oracle's, and its mixed volumes against counts that
other methods fix.  CPU only: the enumeration does no device work."""
import ctypes
import json
import os

import numpy as np
import pytest

import oracle
from oracle import mixed as M
from workloads import (PolySystem, cyclic, embedding_constants, multistep_example, random_dense, random_lifting,
                       random_sparse, rng_for, unit_gamma, with_random_coefficients)

P = pytest.importorskip("paper_1804_03807_gb300")

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_examples.json")))


def _lib_cells(sys, lift):
    cells, vols, mv = P.phc_mixed_cells(sys, lift)
    return sorted(tuple(tuple(int(t) for t in pr) for pr in c) for c in cells), vols, mv


@pytest.mark.parametrize("which,seed", [("cyclic4", 400), ("cyclic5", 401), ("dense3", 402), ("sparse3", 403),
                                        ("cyclic5", 404)])
def test_cells_equal_the_oracles(which, seed):
    rng = rng_for(seed)
    if which.startswith("cyclic"):
        sys = with_random_coefficients(cyclic(int(which[-1])), rng)
    elif which == "dense3":
        sys = random_dense(3, 2, rng)
    else:
        sys = random_sparse(rng, n=3, bezout_range=(8, 64))
    lift = random_lifting(rng, sys.n_terms)
    cells, vols, mv = _lib_cells(sys, lift)
    ref = M.mixed_cells(sys, lift)
    assert cells == sorted(c.pairs for c in ref)
    assert sorted(vols.tolist()) == sorted(c.volume for c in ref)
    assert mv == M.mixed_volume(ref) == int(vols.sum())


def test_example_3_1_top_system_has_the_papers_mixed_volume():
    g = GOLDEN["example_3_1_top_mixed_volume"]
    gammas, hyper = embedding_constants(rng_for(410), 4, 4, g["top_dim"])
    E = oracle.embed(multistep_example(), g["top_dim"], gammas, hyper)
    for seed in (411, 412):
        assert _lib_cells(E, random_lifting(rng_for(seed), E.n_terms))[2] == g["mixed_volume"]


@pytest.mark.parametrize("n,random", [(6, True), (7, False)])
def test_mixed_volume_counts_the_total_degree_roots(n, random):
    """Bernstein: at most mixed-volume many isolated roots in (C*)^n, as many
    for coefficients in general position.  The oracle's total-degree homotopy
    finds 156 regular roots of a random-coefficient cyclic 6 and 924 of
    cyclic 7 itself (whose roots are all regular); random-coefficient copies
    of cyclic 7 can lose roots of large norm to the total-degree homotopy."""
    g = cyclic(n)
    if random:
        g = with_random_coefficients(g, rng_for(420 + n))
    h = oracle.total_degree(g, unit_gamma(rng_for(421)))
    _, cls, _ = oracle.track(h)
    assert _lib_cells(g, random_lifting(rng_for(422), g.n_terms))[2] == int(np.sum(cls == 0)) == {6: 156, 7: 924}[n]


def test_dense_mixed_volume_is_bezout_for_larger_systems():
    for n, d in ((4, 2), (2, 7), (5, 1)):
        sys = random_dense(n, d, rng_for(430 + n))
        assert _lib_cells(sys, random_lifting(rng_for(431), sys.n_terms))[2] == d ** n


def test_counting_call_and_partial_output():
    g = with_random_coefficients(cyclic(5), rng_for(440))
    lift = np.ascontiguousarray(random_lifting(rng_for(441), g.n_terms))
    L = P.load()
    tpe = np.ascontiguousarray(g.terms_per_eq, dtype=np.int32)
    exps = np.ascontiguousarray(g.exps, dtype=np.uint8)
    cnt, mv = ctypes.c_int64(), ctypes.c_int64()
    assert L.phc_mixed_cells(5, tpe.ctypes.data, exps.ctypes.data, lift.ctypes.data, 0, None, None,
                             ctypes.byref(cnt), ctypes.byref(mv)) == 0
    full, _, mv_full = P.phc_mixed_cells(g, lift)
    assert cnt.value == full.shape[0] and mv.value == mv_full == 70
    part = np.zeros((3, 5, 2), dtype=np.int32)
    assert L.phc_mixed_cells(5, tpe.ctypes.data, exps.ctypes.data, lift.ctypes.data, 3, part.ctypes.data, None,
                             ctypes.byref(cnt), None) == 0
    assert np.array_equal(part, full[:3])


def test_bad_inputs_are_rejected():
    g = with_random_coefficients(cyclic(4), rng_for(450))
    with pytest.raises(P.PhcError, match="general position"):
        P.phc_mixed_cells(g, np.zeros(g.n_terms, dtype=np.int32))
    with pytest.raises(P.PhcError, match="0..2"):
        P.phc_mixed_cells(g, np.full(g.n_terms, -1, dtype=np.int32))
    dup = with_random_coefficients(cyclic(4), rng_for(451))
    dup.exps[1] = dup.exps[0]
    with pytest.raises(P.PhcError, match="twice"):
        P.phc_mixed_cells(dup, random_lifting(rng_for(452), dup.n_terms))


def test_a_support_of_one_point_has_no_cells():
    s = PolySystem(2, 2, np.array([1, 2]), np.array([[1, 1], [1, 0], [0, 0]], dtype=np.uint8),
                   np.array([1.0, 2.0, 3.0]))
    cells, vols, mv = P.phc_mixed_cells(s, np.array([5, 7, 9], dtype=np.int32))
    assert cells.shape[0] == 0 and mv == 0


def test_host_allocation_failure_is_an_error_code():
    """Two equations of 4096 terms each (every exponent pair below 64) ask for
    16.8 M candidate edges; under an address-space limit the search runs out
    of host memory, and the call returns PHC_ENOMEM instead of aborting the
    process (run in a child process, whose limit does not outlive it)."""
    import subprocess
    import sys as _sys
    if not os.path.exists("/proc/self/status"):
        pytest.skip("needs /proc/self/status")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = r'''
import resource, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
import paper_1804_03807_gb300 as P
from workloads import PolySystem, random_lifting, rng_for
grid = np.array([(a, b) for a in range(64) for b in range(64)], dtype=np.uint8)
s = PolySystem(2, 2, np.array([4096, 4096]), np.vstack([grid, grid]), np.ones(8192, dtype=np.complex128))
lift = random_lifting(rng_for(560), s.n_terms)
P.load()
vm = int(open("/proc/self/status").read().split("VmSize:")[1].split()[0]) * 1024
resource.setrlimit(resource.RLIMIT_AS, (vm + (96 << 20), resource.RLIM_INFINITY))
try:
    P.phc_mixed_cells(s, lift)
    print("no error")
except P.PhcError as e:
    print("code", e.code, str(e))
'''
    r = subprocess.run([_sys.executable, "-c", code, root], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert "code -2" in r.stdout and "allocation" in r.stdout, r.stdout + r.stderr[-2000:]


def test_cells_do_not_depend_on_the_host_threads():
    """The search's subtrees run on the host threads and their cells are
    emitted in task order, so the cells, their order and the volumes are the
    same for any number of threads (PHC_HOST_THREADS, read at each call)."""
    g = with_random_coefficients(cyclic(7), rng_for(470))
    lift = random_lifting(rng_for(471), g.n_terms)
    old = os.environ.get("PHC_HOST_THREADS")
    runs = []
    try:
        for t in ("1", "3", "8"):
            os.environ["PHC_HOST_THREADS"] = t
            cells, vols, mv = P.phc_mixed_cells(g, lift)
            runs.append((np.asarray(cells).tobytes(), np.asarray(vols).tobytes(), mv))
    finally:
        if old is None:
            os.environ.pop("PHC_HOST_THREADS", None)
        else:
            os.environ["PHC_HOST_THREADS"] = old
    assert runs[0][2] == 924
    assert all(r == runs[0] for r in runs[1:])
