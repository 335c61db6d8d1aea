"""CPU oracle for the path tracker -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the GPU library
(``paper_1804_03807_gb300``) and never imports it.

The arithmetic lives in ``phc_oracle.c`` (complex double, naive per-monomial
evaluation, sequential tracker, double double refinement, a pthreads work
crew).  This module builds it with gcc, binds it with ctypes and writes the
embedding of Section 2.1 (eq. (2)) and the cascade of Section 3.1 out as plain
list manipulation.

Parity pins (tests/test_oracle_*.py): Bezout counts, roots-of-unity starts,
residuals, companion-matrix roots (n = 1), resultant roots (n = 2), gamma
invariance, cyclic symmetry, Example 2.1 and Example 3.1 counts, double double
against exact rationals, step counts of a linear path counted by hand.
Parity unpinned: per-path step counts where floating point decides them, and
the map from start solutions to endpoints (reported only).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from workloads.systems import PolySystem

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "phc_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libphc_oracle.so")
_lock = threading.Lock()
_lib = None

REGULAR, SINGULAR, AT_INFINITY, FAILED = 0, 1, 2, 3
CLASS_NAMES = {REGULAR: "regular", SINGULAR: "singular", AT_INFINITY: "at_infinity", FAILED: "failed"}

STATS_DTYPE = np.dtype([
    ("t", "f8"), ("h", "f8"), ("cond", "f8"), ("relres", "f8"), ("norm_x", "f8"),
    ("n_accept", "i4"), ("n_reject", "i4"), ("n_newton", "i4"), ("n_solve", "i4"),
    ("cls", "i4"), ("stop", "i4"), ("growth", "f8"),
])


class Opts(ctypes.Structure):
    _fields_ = [
        ("h_init", ctypes.c_double), ("h_max", ctypes.c_double), ("h_min", ctypes.c_double),
        ("expand_after", ctypes.c_int32), ("expand", ctypes.c_double), ("shrink", ctypes.c_double),
        ("max_corr_iters", ctypes.c_int32), ("corr_tol", ctypes.c_double), ("corr_contract", ctypes.c_double),
        ("max_steps", ctypes.c_int32), ("max_steps_decade", ctypes.c_int32), ("diverge_norm", ctypes.c_double), ("endpoint_inf_norm", ctypes.c_double),
        ("end_zone", ctypes.c_double), ("growth_inf", ctypes.c_double), ("end_iters", ctypes.c_int32), ("end_tol", ctypes.c_double),
        ("cond_regular", ctypes.c_double), ("res_regular", ctypes.c_double), ("slack_tol", ctypes.c_double),
    ]


class _Hom(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32), ("n", ctypes.c_int32), ("n_terms", ctypes.c_int32),
        ("terms_per_eq", ctypes.c_void_p), ("exps", ctypes.c_void_p), ("coefs", ctypes.c_void_p),
        ("gamma_re", ctypes.c_double), ("gamma_im", ctypes.c_double),
        ("row", ctypes.c_int32), ("slack", ctypes.c_int32), ("coefs0", ctypes.c_void_p),
        ("powers", ctypes.c_void_p),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, no contraction of a*b+c)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            L.orc_track.restype = ctypes.c_int
            L.orc_track_qd.restype = ctypes.c_int
            L.orc_num_paths.restype = ctypes.c_int64
            L.orc_refine.restype = ctypes.c_int
            assert L.orc_stats_size() == STATS_DTYPE.itemsize
            assert L.orc_opts_size() == ctypes.sizeof(Opts)
            assert L.orc_homotopy_size() == ctypes.sizeof(_Hom)
            _lib = L
    return _lib


def default_opts() -> Opts:
    o = Opts()
    lib().orc_default_opts(ctypes.byref(o))
    return o


def host_threads() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


class Homotopy:
    """Keeps the numpy buffers alive behind the C struct."""

    def __init__(self, sys: PolySystem, kind: int, gamma: complex = 1.0, row: int = -1, slack: int = -1,
                 coefs0=None, powers=None):
        assert sys.n_eq == sys.n_var, "the tracker needs a square system"
        self.sys = sys
        self.n = sys.n_var
        self._tpe = np.ascontiguousarray(sys.terms_per_eq, dtype=np.int32)
        self._exps = np.ascontiguousarray(sys.exps, dtype=np.uint8)
        self._coefs = np.ascontiguousarray(np.stack([sys.coefs.real, sys.coefs.imag], axis=1), dtype=np.float64)
        self._coefs0 = None
        if coefs0 is not None:
            c0 = np.asarray(coefs0, dtype=np.complex128).reshape(-1)
            assert c0.shape[0] == sys.n_terms, "start coefficients must match the target's terms"
            self._coefs0 = np.ascontiguousarray(np.stack([c0.real, c0.imag], axis=1), dtype=np.float64)
        self._powers = None
        if powers is not None:
            self._powers = np.ascontiguousarray(powers, dtype=np.float64).reshape(-1)
            assert self._powers.shape[0] == sys.n_terms, "one power of t per term"
        self.c = _Hom(kind, self.n, sys.n_terms, self._tpe.ctypes.data, self._exps.ctypes.data,
                      self._coefs.ctypes.data, float(np.real(gamma)), float(np.imag(gamma)), row, slack,
                      None if self._coefs0 is None else self._coefs0.ctypes.data,
                      None if self._powers is None else self._powers.ctypes.data)

    def ref(self):
        return ctypes.byref(self.c)


def total_degree(sys: PolySystem, gamma: complex) -> Homotopy:
    """H(x,t) = (1-t) gamma g(x) + t f(x), g_i = x_i^{d_i} - 1."""
    return Homotopy(sys, 0, gamma)


def parameter_homotopy(target: PolySystem, start_coefs, gamma: complex) -> Homotopy:
    """H(x,t) = (1-t) gamma g(x) + t f(x), f = target, g = the target's
    supports with the coefficients start_coefs (Section 2.3: the solutions
    of a random coefficient system start the paths to the target).  Paths
    start from explicit solutions of g (track(..., starts=...))."""
    return Homotopy(target, 2, gamma, coefs0=start_coefs)


def polyhedral_homotopy(sys: PolySystem, powers) -> Homotopy:
    """The polyhedral homotopy of one mixed cell (Section 2.2): term q of
    sys carries the factor t^{powers[q]} (0 on the cell's terms); paths start
    from the cell's binomial solutions (oracle.mixed.binomial_starts) and end
    at solutions of sys."""
    return Homotopy(sys, 3, 1.0, powers=powers)


def end_measures(h: Homotopy, x: np.ndarray):
    """(cond, relres) of the endpoint x as a root of H(., 1)."""
    xb = np.ascontiguousarray(x, dtype=np.complex128)
    c = ctypes.c_double()
    r = ctypes.c_double()
    lib().orc_end_measures(h.ref(), xb.view(np.float64).ctypes.data_as(ctypes.c_void_p), ctypes.byref(c),
                           ctypes.byref(r))
    return c.value, r.value


def cascade_homotopy(emb: PolySystem, n_eq_orig: int, n_var_orig: int, k: int) -> Homotopy:
    """Cascade stage k -> k-1 on E_k (Section 3.1): hyperplane k (equation
    n_eq_orig + k - 1) keeps its slack z_k (variable n_var_orig + k - 1) and
    has its other terms scaled by (1 - t)."""
    return Homotopy(emb, 1, 1.0, row=n_eq_orig + k - 1, slack=n_var_orig + k - 1)


def num_paths(h: Homotopy) -> int:
    return int(lib().orc_num_paths(h.ref()))


def start_solution(h: Homotopy, p: int) -> np.ndarray:
    out = np.zeros(2 * h.n)
    lib().orc_start_solution(h.ref(), ctypes.c_int64(p), out.ctypes.data_as(ctypes.c_void_p))
    return out[0::2] + 1j * out[1::2]


def track(h: Homotopy, starts: np.ndarray | None = None, first: int = 0, n_paths: int | None = None,
          opts: Opts | None = None, threads: int | None = None):
    """Track paths; returns (x [P, n] complex128, cls [P] int8, stats [P])."""
    L = lib()
    if starts is not None:
        starts = np.ascontiguousarray(starts, dtype=np.complex128).reshape(-1, h.n)
        n_paths = starts.shape[0]
        sbuf = starts.view(np.float64).ctypes.data_as(ctypes.c_void_p)
    else:
        if n_paths is None:
            n_paths = num_paths(h) - first
        sbuf = None
    x = np.zeros((n_paths, h.n), dtype=np.complex128)
    cls = np.zeros(n_paths, dtype=np.int8)
    stats = np.zeros(n_paths, dtype=STATS_DTYPE)
    o = opts if opts is not None else default_opts()
    rc = L.orc_track(h.ref(), sbuf, ctypes.c_int64(first), ctypes.c_int64(n_paths), ctypes.byref(o),
                     int(threads or host_threads()), x.view(np.float64).ctypes.data_as(ctypes.c_void_p),
                     cls.ctypes.data_as(ctypes.c_void_p), stats.ctypes.data_as(ctypes.c_void_p))
    if rc != 0:
        raise ValueError(f"orc_track failed: {rc}")
    return x, cls, stats


def track_dd(h: Homotopy, starts: np.ndarray | None = None, first: int = 0, n_paths: int | None = None,
             opts: Opts | None = None, threads: int | None = None):
    """Track paths in complex double double (Section 5, Table 2: the solver in
    double double arithmetic); returns (x_hi, x_lo [P, n] complex128, cls,
    stats)."""
    L = lib()
    if starts is not None:
        starts = np.ascontiguousarray(starts, dtype=np.complex128).reshape(-1, h.n)
        n_paths = starts.shape[0]
        sbuf = starts.view(np.float64).ctypes.data_as(ctypes.c_void_p)
    else:
        if n_paths is None:
            n_paths = num_paths(h) - first
        sbuf = None
    xh = np.zeros((n_paths, h.n), dtype=np.complex128)
    xl = np.zeros((n_paths, h.n), dtype=np.complex128)
    cls = np.zeros(n_paths, dtype=np.int8)
    stats = np.zeros(n_paths, dtype=STATS_DTYPE)
    o = opts if opts is not None else default_opts()
    rc = L.orc_track_dd(h.ref(), sbuf, ctypes.c_int64(first), ctypes.c_int64(n_paths), ctypes.byref(o),
                        int(threads or host_threads()), xh.view(np.float64).ctypes.data_as(ctypes.c_void_p),
                        xl.view(np.float64).ctypes.data_as(ctypes.c_void_p), cls.ctypes.data_as(ctypes.c_void_p),
                        stats.ctypes.data_as(ctypes.c_void_p))
    if rc != 0:
        raise ValueError(f"orc_track_dd failed: {rc}")
    return xh, xl, cls, stats


def track_qd(h: Homotopy, starts: np.ndarray | None = None, first: int = 0, n_paths: int | None = None,
             opts: Opts | None = None, threads: int | None = None):
    """Track paths in complex quad double (Section 5, Table 2: the solver in
    quad double arithmetic); returns (x [P, n, 4] complex128: the four parts
    of every coordinate, cls, stats)."""
    L = lib()
    if starts is not None:
        starts = np.ascontiguousarray(starts, dtype=np.complex128).reshape(-1, h.n)
        n_paths = starts.shape[0]
        sbuf = starts.view(np.float64).ctypes.data_as(ctypes.c_void_p)
    else:
        if n_paths is None:
            n_paths = num_paths(h) - first
        sbuf = None
    x = np.zeros((n_paths, h.n, 4), dtype=np.complex128)
    cls = np.zeros(n_paths, dtype=np.int8)
    stats = np.zeros(n_paths, dtype=STATS_DTYPE)
    o = opts if opts is not None else default_opts()
    rc = L.orc_track_qd(h.ref(), sbuf, ctypes.c_int64(first), ctypes.c_int64(n_paths), ctypes.byref(o),
                        int(threads or host_threads()), x.view(np.float64).ctypes.data_as(ctypes.c_void_p),
                        cls.ctypes.data_as(ctypes.c_void_p), stats.ctypes.data_as(ctypes.c_void_p))
    if rc != 0:
        raise ValueError(f"orc_track_qd failed: {rc}")
    return x, cls, stats


def qd_op(name: str, a, b):
    """Quad double primitives for the exact-rational tests: name in qd_add,
    qd_mul, qd_div; a, b and the result are four doubles."""
    L = lib()
    out = np.zeros(4)
    ab = np.ascontiguousarray(a, dtype=np.float64)
    bb = np.ascontiguousarray(b, dtype=np.float64)
    getattr(L, "orc_" + name)(ab.ctypes.data_as(ctypes.c_void_p), bb.ctypes.data_as(ctypes.c_void_p),
                              out.ctypes.data_as(ctypes.c_void_p))
    return out


def endgame(h: Homotopy, first: int = 0, n_paths: int | None = None, opts: Opts | None = None):
    """Cauchy endgame (reading in phc_oracle.c): per total-degree path the
    cycle number c (0: no estimate) and the mean of the samples of x over c
    loops around t = 1 (the estimate of the endpoint).  Returns (x [P, n],
    cycle [P], stats)."""
    if n_paths is None:
        n_paths = num_paths(h) - first
    x = np.zeros((n_paths, h.n), dtype=np.complex128)
    cyc = np.zeros(n_paths, dtype=np.int32)
    stats = np.zeros(n_paths, dtype=STATS_DTYPE)
    o = opts if opts is not None else default_opts()
    rc = lib().orc_endgame(h.ref(), ctypes.c_int64(first), ctypes.c_int64(n_paths), ctypes.byref(o),
                           x.view(np.float64).ctypes.data_as(ctypes.c_void_p), cyc.ctypes.data_as(ctypes.c_void_p),
                           stats.ctypes.data_as(ctypes.c_void_p))
    if rc != 0:
        raise ValueError(f"orc_endgame failed: {rc}")
    return x, cyc, stats


def refine(h: Homotopy, x: np.ndarray, cls: np.ndarray, cond: np.ndarray, reached: np.ndarray,
           cond_threshold: float = 1e6, cond_max: float = 1e12, max_iters: int = 8):
    """Double double Newton refinement at t = 1 of the ill-conditioned
    endpoints of paths that reached t = 1.  Returns (x_hi, x_lo, cls, cond)."""
    xh = np.ascontiguousarray(x, dtype=np.complex128).copy()
    xl = np.zeros_like(xh)
    c = np.ascontiguousarray(cls, dtype=np.int8).copy()
    cd = np.ascontiguousarray(cond, dtype=np.float64).copy()
    lib().orc_refine(h.ref(), xh.view(np.float64).ctypes.data_as(ctypes.c_void_p),
                     xl.view(np.float64).ctypes.data_as(ctypes.c_void_p), ctypes.c_int64(xh.shape[0]),
                     ctypes.c_double(cond_threshold), ctypes.c_double(cond_max), int(max_iters),
                     c.ctypes.data_as(ctypes.c_void_p), cd.ctypes.data_as(ctypes.c_void_p),
                     np.ascontiguousarray(reached, dtype=np.int32).ctypes.data_as(ctypes.c_void_p))
    return xh, xl, c, cd


def evaluate(h: Homotopy, x: np.ndarray, t: float):
    """(H, H_x, H_t) at (x, t)."""
    n = h.n
    xb = np.ascontiguousarray(x, dtype=np.complex128)
    H = np.zeros(n, np.complex128)
    Hx = np.zeros((n, n), np.complex128)
    Ht = np.zeros(n, np.complex128)
    lib().orc_eval(h.ref(), xb.view(np.float64).ctypes.data_as(ctypes.c_void_p), ctypes.c_double(t),
                   H.view(np.float64).ctypes.data_as(ctypes.c_void_p),
                   Hx.view(np.float64).ctypes.data_as(ctypes.c_void_p),
                   Ht.view(np.float64).ctypes.data_as(ctypes.c_void_p))
    return H, Hx, Ht


def lu_solve(A: np.ndarray, b: np.ndarray) -> np.ndarray:
    n = A.shape[0]
    Ab = np.ascontiguousarray(A, dtype=np.complex128)
    bb = np.ascontiguousarray(b, dtype=np.complex128)
    x = np.zeros(n, np.complex128)
    rc = lib().orc_lu_solve(n, Ab.view(np.float64).ctypes.data_as(ctypes.c_void_p),
                            bb.view(np.float64).ctypes.data_as(ctypes.c_void_p),
                            x.view(np.float64).ctypes.data_as(ctypes.c_void_p))
    if rc:
        raise np.linalg.LinAlgError("singular")
    return x


def dd_op(name: str, a, b):
    """Double double primitives for the exact-rational tests: name in
    two_sum, two_prod (double inputs) or dd_add, dd_mul, dd_div (pairs)."""
    L = lib()
    out = np.zeros(2)
    op = out.ctypes.data_as(ctypes.c_void_p)
    if name in ("two_sum", "two_prod"):
        getattr(L, "orc_" + name)(ctypes.c_double(a), ctypes.c_double(b), op)
    else:
        ab = np.array(a, dtype=np.float64)
        bb = np.array(b, dtype=np.float64)
        getattr(L, "orc_" + name)(ab.ctypes.data_as(ctypes.c_void_p), bb.ctypes.data_as(ctypes.c_void_p), op)
    return float(out[0]), float(out[1])


# ------------------------------------------------------------------ embedding

def embed(sys: PolySystem, top_dim: int, gammas: np.ndarray, hyper: np.ndarray) -> PolySystem:
    """The embedded system E_D of Section 2.1 (eq. (2) for D = 1).

    Unknowns: x_1..x_n, z_1..z_D.  Equation i (i <= n_eq) is
    f_i(x) + sum_k gammas[i,k] z_k; equation n_eq + k is
    hyper[k,0] + sum_j hyper[k,j+1] x_j + z_k.  Only square systems.
    """
    assert sys.n_eq == sys.n_var, "square systems only"
    n, D = sys.n_var, top_dim
    N = n + D
    exps, coefs, tpe = [], [], []
    off = 0
    for i in range(sys.n_eq):
        m = int(sys.terms_per_eq[i])
        for k in range(m):
            exps.append(list(sys.exps[off + k]) + [0] * D)
            coefs.append(sys.coefs[off + k])
        for k in range(D):
            e = [0] * N
            e[n + k] = 1
            exps.append(e)
            coefs.append(gammas[i, k])
        tpe.append(m + D)
        off += m
    for k in range(D):
        exps.append([0] * N)
        coefs.append(hyper[k, 0])
        for j in range(n):
            e = [0] * N
            e[j] = 1
            exps.append(e)
            coefs.append(hyper[k, j + 1])
        e = [0] * N
        e[n + k] = 1
        exps.append(e)
        coefs.append(1.0)
        tpe.append(n + 2)
    return PolySystem(sys.n_eq + D, N, np.array(tpe), np.array(exps, dtype=np.uint8), np.array(coefs),
                      name=f"{sys.name}-E{D}")


def square(sys: PolySystem, consts: np.ndarray) -> PolySystem:
    """A square system from a non-square one (Section 2.1).  Underdetermined
    (n_eq < n_var): add the n_var - n_eq hyperplanes
    consts[k, 0] + sum_j consts[k, j+1] x_j.  Overdetermined (n_eq > n_var):
    add n_eq - n_var unknowns s_k after x and the term consts[i, k] s_k to
    every equation i.  Square: unchanged."""
    n_eq, n = sys.n_eq, sys.n_var
    N = max(n_eq, n)
    exps, coefs, tpe = [], [], []
    off = 0
    for i in range(n_eq):
        m = int(sys.terms_per_eq[i])
        for q in range(m):
            exps.append(list(sys.exps[off + q]) + [0] * (N - n))
            coefs.append(sys.coefs[off + q])
        if n_eq > n:
            for k in range(N - n):
                e = [0] * N
                e[n + k] = 1
                exps.append(e)
                coefs.append(consts[i, k])
            m += N - n
        tpe.append(m)
        off += int(sys.terms_per_eq[i])
    if n_eq < n:
        for k in range(N - n_eq):
            exps.append([0] * N)
            coefs.append(consts[k, 0])
            for j in range(n):
                e = [0] * N
                e[j] = 1
                exps.append(e)
                coefs.append(consts[k, j + 1])
            tpe.append(n + 1)
    return PolySystem(N, N, np.array(tpe), np.array(exps, dtype=np.uint8).reshape(-1, N), np.array(coefs),
                      name=f"{sys.name}-sq")


def drop_last_slack(emb: PolySystem, n_eq_orig: int, n_var_orig: int, k: int) -> PolySystem:
    """E_k with z_k = 0 and hyperplane k removed, i.e. E_{k-1}."""
    N = emb.n_var
    s = n_var_orig + k - 1
    row = n_eq_orig + k - 1
    exps, coefs, tpe = [], [], []
    off = 0
    for i in range(emb.n_eq):
        m = int(emb.terms_per_eq[i])
        if i == row:
            off += m
            continue
        cnt = 0
        for q in range(m):
            e = emb.exps[off + q]
            if e[s] != 0:
                continue
            exps.append([int(v) for j, v in enumerate(e) if j != s])
            coefs.append(emb.coefs[off + q])
            cnt += 1
        tpe.append(cnt)
        off += m
    return PolySystem(emb.n_eq - 1, N - 1, np.array(tpe), np.array(exps, dtype=np.uint8).reshape(-1, N - 1),
                      np.array(coefs), name=f"{emb.name}-drop{k}")


def slack_zero(x: np.ndarray, slack_index: int, tol: float = 1e-8) -> np.ndarray:
    """|z| <= tol (1 + ||x||), norms max over max(|Re|, |Im|)."""
    a = np.maximum(np.abs(x.real), np.abs(x.imag))
    return a[:, slack_index] <= tol * (1.0 + a.max(axis=1))


def cascade_stage(emb: PolySystem, n_eq_orig: int, n_var_orig: int, k: int, starts: np.ndarray,
                  opts: Opts | None = None, threads: int | None = None):
    """Track the cascade homotopy E_k -> E_{k-1} from ``starts`` (solutions of
    E_k with z_k != 0).  Returns (E_{k-1}, x without z_k, cls, stats)."""
    h = cascade_homotopy(emb, n_eq_orig, n_var_orig, k)
    x, cls, st = track(h, starts=starts, opts=opts, threads=threads)
    s = n_var_orig + k - 1
    x_next = np.delete(x, s, axis=1)
    return drop_last_slack(emb, n_eq_orig, n_var_orig, k), x_next, cls, st


# ------------------------------------------------------------------ membership test and filtering (Section 4)

def membership_target(emb: PolySystem, n_var_orig: int, k: int, z: np.ndarray) -> PolySystem:
    """E_k with the constant c_j0 of every hyperplane j (the last k equations)
    replaced by c_j3 = -sum_i c_ji z_i, so that (z, 0) satisfies every
    hyperplane (Section 4.1, Example 4.1: c_3 = -2 c_1 for the point (2, 0))."""
    coefs = np.array(emb.coefs, dtype=np.complex128).copy()
    bounds = np.concatenate([[0], np.cumsum(emb.terms_per_eq)])
    z = np.asarray(z, dtype=np.complex128)
    for j in range(k):
        row = emb.n_eq - k + j
        const, acc = None, 0.0 + 0.0j
        for q in range(int(bounds[row]), int(bounds[row + 1])):
            e = np.asarray(emb.exps[q], dtype=np.int64)
            if e.sum() == 0:
                const = q
            elif e[:n_var_orig].sum() == 1 and e.sum() == 1:
                acc += coefs[q] * z[int(np.argmax(e[:n_var_orig]))]
        assert const is not None, "a hyperplane without constant term"
        coefs[const] = -acc
    return PolySystem(emb.n_eq, emb.n_var, np.array(emb.terms_per_eq), np.array(emb.exps), coefs,
                      name=f"{emb.name}-moved")


def membership(emb: PolySystem, n_var_orig: int, k: int, witness: np.ndarray, points: np.ndarray,
               tol: float = 1e-3, threads: int | None = None):
    """Homotopy membership test (Section 4.1, Example 4.1).  witness [m, N]:
    the generic points of a k-dimensional set, solutions of E_k = emb with
    zero slacks.  For every test point z (rows of points, the first
    n_var_orig unknowns) the hyperplane constants move from c_0 to c_3
    along (1-t) E_k(c_0) + t E_k(c_3); z lies on the set when one endpoint
    (regular or singular) equals (z, 0) within tol (1 + ||z||) in every
    unknown.  The tolerance is loose because the points tested are singular
    endpoints of the cascade (on a higher-dimensional set the Jacobian loses
    rank and the end Newton steps converge slowly: in Example 3.1 they are
    accurate to about 1e-4, while the other endpoints are at distance >= 1).
    Returns (on [p] bool, per point the endpoints and classes)."""
    witness = np.atleast_2d(np.asarray(witness, dtype=np.complex128))
    on, ends = [], []
    for z in np.atleast_2d(np.asarray(points, dtype=np.complex128)):
        target = membership_target(emb, n_var_orig, k, z)
        h = parameter_homotopy(target, emb.coefs, 1.0)
        x, c, st = track(h, starts=witness, threads=threads)
        zz = np.concatenate([z, np.zeros(emb.n_var - n_var_orig)])
        nz = np.max(np.maximum(np.abs(z.real), np.abs(z.imag)))
        d = np.max(np.maximum(np.abs((x - zz).real), np.abs((x - zz).imag)), axis=1)
        on.append(bool(np.any(((c == REGULAR) | (c == SINGULAR)) & (d <= tol * (1.0 + nz)))))
        ends.append((x, c))
    return np.array(on, dtype=bool), ends


def filter_candidates(levels: dict, n_var_orig: int, tol: float = 1e-3, threads: int | None = None):
    """The filters of Section 4.2 (Figures 4 and 5).  levels[k] = (E_k,
    x [P, n + k], cls [P]) are the endpoints of the cascade at dimension k
    (top level D first, then D-1, ..., 0; E_0 is the original system), each
    point's last unknown being z_k for k >= 1.  At every level the finite
    candidates with z_k = 0 (all endpoints at level 0) that are regular are
    kept; the singular ones are tested against the witness sets of the
    higher dimensions, from the top down, and dropped when on one.  The
    witness set of dimension k is what is kept at level k.

    Returns (witness sets {k: points [m, n + k]}, isolated points at level 0
    (the kept and the remaining singular candidates), and the filter stages
    as (level, dimension tested against, paths tracked, points removed))."""
    D = max(levels)
    witness, stages = {}, []
    isolated = None
    for k in range(D, -1, -1):
        E, x, cls = levels[k]
        finite = (cls == REGULAR) | (cls == SINGULAR)
        cand = finite & (slack_zero(x, n_var_orig + k - 1) if k >= 1 else np.ones(len(cls), bool))
        keep = x[cand & (cls == REGULAR)]
        sus = x[cand & (cls == SINGULAR)]
        for kk in range(D, k, -1):
            if len(sus) == 0:
                break
            Ekk, W = witness[kk]
            if len(W) == 0:
                continue
            on, _ = membership(Ekk, n_var_orig, kk, W, sus[:, :n_var_orig], tol, threads)
            stages.append((k, kk, len(sus) * len(W), int(on.sum())))
            sus = sus[~on]
        kept = np.concatenate([keep, sus]) if len(sus) else keep
        if k >= 1:
            witness[k] = (E, kept)
        else:
            isolated = kept
    return {k: w for k, (E, w) in witness.items()}, isolated, stages
