"""ctypes binding of libphc.so (include/phc.h): argument marshalling only.

Every function here has the name of the C entry point it calls.  Device
arrays are torch CUDA tensors (their ``data_ptr()`` is passed); the stream is
torch's current CUDA stream unless one is given.  There is no fallback: if
the shared library is missing, loading raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libphc.so")

PHC_OK, PHC_EINVAL, PHC_ENOMEM, PHC_ECUDA, PHC_ETIMEOUT, PHC_EUNSUPPORTED = 0, -1, -2, -3, -4, -5
PHC_REGULAR, PHC_SINGULAR, PHC_AT_INFINITY, PHC_FAILED = 0, 1, 2, 3
PHC_STOP_REACHED, PHC_STOP_DIVERGED, PHC_STOP_STEP_MIN, PHC_STOP_BUDGET, PHC_STOP_NONFINITE = 0, 1, 2, 3, 4
PHC_STOP_SKIPPED = 5
PHC_PREC_FP64, PHC_PREC_FP32_INTERIOR = 0, 1
PHC_MAX_VARS = 12
PHC_NOALLOC_MAX_PATHS = 52428
PHC_NOALLOC_MAX_HANDOFF = 4096

EXPORTED = [
    "phc_default_opts", "phc_make_homotopy", "phc_num_paths", "phc_track_paths", "phc_embed", "phc_cascade_stage",
    "phc_refine_endpoints", "phc_last_error", "phc_destroy_homotopy", "phc_free_lists", "phc_sizeof_opts",
    "phc_sizeof_stats", "phc_track_paths_noalloc", "phc_make_homotopy_batch", "phc_track_pipeline",
    "phc_track_many", "phc_cascade_from", "phc_tail_paths", "phc_make_parameter_homotopy", "phc_track_from",
    "phc_membership_test", "phc_square", "phc_many_plan_create", "phc_many_plan_run", "phc_many_plan_destroy",
]


class PhcError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"phc error {code}: {msg}")
        self.code = code


class phc_cd(ctypes.Structure):
    _fields_ = [("re", ctypes.c_double), ("im", ctypes.c_double)]


class phc_opts(ctypes.Structure):
    _fields_ = [
        ("h_init", ctypes.c_double), ("h_max", ctypes.c_double), ("h_min", ctypes.c_double),
        ("expand_after", ctypes.c_int32), ("expand", ctypes.c_double), ("shrink", ctypes.c_double),
        ("max_corr_iters", ctypes.c_int32), ("corr_tol", ctypes.c_double), ("corr_contract", ctypes.c_double),
        ("max_steps", ctypes.c_int32), ("max_steps_decade", ctypes.c_int32),
        ("diverge_norm", ctypes.c_double), ("endpoint_inf_norm", ctypes.c_double), ("end_zone", ctypes.c_double),
        ("growth_inf", ctypes.c_double),
        ("end_iters", ctypes.c_int32), ("end_tol", ctypes.c_double),
        ("cond_regular", ctypes.c_double), ("res_regular", ctypes.c_double), ("slack_tol", ctypes.c_double),
        ("precision", ctypes.c_int32), ("fp32_t_max", ctypes.c_double), ("fp32_pivot_ratio", ctypes.c_double),
        ("block_threads", ctypes.c_int32), ("max_blocks", ctypes.c_int32), ("tail_drain", ctypes.c_double),
        ("tail_threads", ctypes.c_int32), ("compact", ctypes.c_int32), ("group_paths", ctypes.c_int32),
    ]


STATS_DTYPE = np.dtype([
    ("t", "f8"), ("h", "f8"), ("cond", "f8"), ("relres", "f8"), ("norm_x", "f8"), ("growth", "f8"),
    ("n_accept", "i4"), ("n_reject", "i4"), ("n_newton", "i4"), ("n_solve", "i4"), ("stop", "i4"),
    ("n_fp32", "i4"), ("grew", "i4"), ("system", "i4"),
])


class phc_system_lists(ctypes.Structure):
    _fields_ = [
        ("n_eq", ctypes.c_int32), ("n_var", ctypes.c_int32), ("n_terms", ctypes.c_int32),
        ("terms_per_eq", ctypes.POINTER(ctypes.c_int32)), ("exps", ctypes.POINTER(ctypes.c_uint8)),
        ("coefs", ctypes.POINTER(phc_cd)),
    ]


_lib = None


def load() -> ctypes.CDLL:
    """Load libphc.so (built in-tree by paper_1804_03807_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libphc.so is not built ({LIB_PATH}); run paper_1804_03807_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    L.phc_default_opts.argtypes = [ctypes.POINTER(phc_opts)]
    L.phc_make_homotopy.argtypes = [i32, i32, vp, vp, vp, phc_cd, ctypes.POINTER(vp)]
    L.phc_make_homotopy_batch.argtypes = [i32, i32, vp, vp, i32, vp, vp, ctypes.POINTER(vp)]
    L.phc_num_paths.argtypes = [vp, ctypes.POINTER(i64)]
    L.phc_track_paths.argtypes = [vp, i64, i64, ctypes.POINTER(phc_opts), vp, vp, vp, vp]
    L.phc_track_paths_noalloc.argtypes = [vp, i64, i64, ctypes.POINTER(phc_opts), vp, vp, vp, vp]
    L.phc_embed.argtypes = [i32, i32, vp, vp, vp, i32, vp, vp, ctypes.c_uint64,
                            ctypes.POINTER(ctypes.POINTER(phc_system_lists))]
    L.phc_track_paths_dd.argtypes = [vp, i64, i64, ctypes.POINTER(phc_opts), vp, vp, vp, vp, vp]
    L.phc_endgame.argtypes = [vp, i64, i64, ctypes.POINTER(phc_opts), vp, vp, vp, vp]
    L.phc_track_paths_qd.argtypes = [vp, i64, i64, ctypes.POINTER(phc_opts), vp, vp, vp, vp]
    L.phc_many_plan_create.argtypes = [vp, i32, ctypes.POINTER(phc_opts), vp, vp, vp, vp, ctypes.POINTER(vp)]
    L.phc_many_plan_run.argtypes = [vp, vp]
    L.phc_many_plan_destroy.argtypes = [vp]
    L.phc_many_plan_destroy.restype = None
    L.phc_square.argtypes = [i32, i32, vp, vp, vp, vp, ctypes.c_uint64,
                             ctypes.POINTER(ctypes.POINTER(phc_system_lists))]
    L.phc_cascade_stage.argtypes = [vp, i32, vp, i64, ctypes.POINTER(phc_opts), vp, vp, vp, vp, vp]
    L.phc_cascade_from.argtypes = [vp, i32, vp, vp, vp, i64, ctypes.POINTER(phc_opts), vp, vp, vp, vp, vp]
    L.phc_track_many.argtypes = [vp, i32, ctypes.POINTER(phc_opts), vp, vp, vp, vp]
    L.phc_track_pipeline.argtypes = [vp, i32, i64, i64, ctypes.POINTER(phc_opts), vp, vp, vp, vp, vp, vp, vp, vp]
    L.phc_refine_endpoints.argtypes = [vp, vp, vp, i64, ctypes.c_double, ctypes.c_double, i32, vp, vp, vp]
    L.phc_tail_paths.argtypes = [vp, vp, ctypes.POINTER(i64), ctypes.POINTER(i64)]
    L.phc_make_parameter_homotopy.argtypes = [i32, i32, vp, vp, i32, vp, vp, phc_cd, ctypes.POINTER(vp)]
    L.phc_track_from.argtypes = [vp, vp, i64, i64, ctypes.POINTER(phc_opts), vp, vp, vp, vp]
    L.phc_membership_test.argtypes = [i32, i32, vp, vp, vp, i32, vp, i64, vp, i64, ctypes.c_double,
                                      ctypes.POINTER(phc_opts), vp, vp, vp, vp]
    L.phc_mixed_cells.argtypes = [i32, vp, vp, vp, i64, vp, vp, ctypes.POINTER(i64), ctypes.POINTER(i64)]
    L.phc_make_polyhedral_homotopy.argtypes = [i32, vp, vp, vp, vp, vp, i64, ctypes.POINTER(vp)]
    L.phc_polyhedral_starts.argtypes = [vp, i64, i64, vp, vp]
    L.phc_track_polyhedral.argtypes = [vp, i64, i64, ctypes.POINTER(phc_opts), vp, vp, vp, vp]
    L.phc_solve_polyhedral.argtypes = [i32, vp, vp, vp, vp, ctypes.POINTER(phc_opts), i64, vp, vp, vp,
                                       ctypes.POINTER(i64), ctypes.POINTER(i64), vp]
    L.phc_fp64_probe.argtypes = [i32, i64, ctypes.POINTER(ctypes.c_double), vp]
    L.phc_last_error.restype = ctypes.c_char_p
    L.phc_destroy_homotopy.argtypes = [vp]
    L.phc_destroy_homotopy.restype = None
    L.phc_free_lists.argtypes = [ctypes.POINTER(phc_system_lists)]
    L.phc_free_lists.restype = None
    for name in ("phc_default_opts", "phc_make_homotopy", "phc_make_homotopy_batch", "phc_num_paths",
                 "phc_track_paths",
                 "phc_track_paths_noalloc", "phc_track_pipeline", "phc_track_many", "phc_cascade_from",
                 "phc_embed",
                 "phc_cascade_stage", "phc_refine_endpoints", "phc_sizeof_opts", "phc_sizeof_stats",
                 "phc_tail_paths", "phc_make_parameter_homotopy", "phc_track_from", "phc_membership_test",
                 "phc_square", "phc_many_plan_create", "phc_many_plan_run", "phc_track_paths_dd", "phc_endgame",
                 "phc_mixed_cells", "phc_make_polyhedral_homotopy", "phc_polyhedral_starts",
                 "phc_track_polyhedral", "phc_solve_polyhedral", "phc_track_paths_qd", "phc_fp64_probe"):
        getattr(L, name).restype = ctypes.c_int
    if L.phc_sizeof_opts() != ctypes.sizeof(phc_opts):
        raise ImportError("phc_opts layout mismatch between phc.h and the binding")
    if L.phc_sizeof_stats() != STATS_DTYPE.itemsize:
        raise ImportError("phc_path_stats layout mismatch between phc.h and the binding")
    _lib = L
    return L


def _check(rc: int):
    if rc != PHC_OK:
        raise PhcError(rc, load().phc_last_error().decode())


def _stream_ptr(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(getattr(stream, "cuda_stream", stream) or 0)


def _ptr(t) -> int | None:
    return None if t is None else int(t.data_ptr())


def _lists(sys):
    tpe = np.ascontiguousarray(sys.terms_per_eq, dtype=np.int32)
    exps = np.ascontiguousarray(sys.exps, dtype=np.uint8)
    coefs = np.ascontiguousarray(sys.coefs, dtype=np.complex128)
    return tpe, exps, coefs


class Homotopy:
    """Owning wrapper of a phc_homotopy* (destroyed with the object)."""

    def __init__(self, ptr: int, n: int):
        self.ptr = ptr
        self.n = n

    def __del__(self):
        if getattr(self, "ptr", None) and _lib is not None:
            _lib.phc_destroy_homotopy(ctypes.c_void_p(self.ptr))
            self.ptr = None


def phc_default_opts(**overrides) -> phc_opts:
    o = phc_opts()
    _check(load().phc_default_opts(ctypes.byref(o)))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def phc_make_homotopy(sys, gamma: complex) -> Homotopy:
    """Total-degree homotopy of the square system ``sys`` (an object with
    n_eq, n_var, terms_per_eq, exps, coefs)."""
    L = load()
    tpe, exps, coefs = _lists(sys)
    out = ctypes.c_void_p()
    _check(L.phc_make_homotopy(int(sys.n_eq), int(sys.n_var), tpe.ctypes.data, exps.ctypes.data, coefs.ctypes.data,
                               phc_cd(float(np.real(gamma)), float(np.imag(gamma))), ctypes.byref(out)))
    return Homotopy(out.value, int(sys.n_var))


def phc_make_homotopy_batch(systems, gammas) -> Homotopy:
    """One handle for systems that share supports (terms_per_eq, exps) and
    differ in coefficients and gamma; path p of system s is s * P + p."""
    L = load()
    tpe, exps, _ = _lists(systems[0])
    for s in systems[1:]:
        if not (np.array_equal(np.asarray(s.terms_per_eq), tpe) and np.array_equal(np.asarray(s.exps), exps)):
            raise ValueError("systems of a batch must share terms_per_eq and exps")
    coefs = np.ascontiguousarray(np.stack([np.asarray(s.coefs, dtype=np.complex128) for s in systems]))
    gam = np.ascontiguousarray(np.asarray(gammas, dtype=np.complex128))
    out = ctypes.c_void_p()
    _check(L.phc_make_homotopy_batch(int(systems[0].n_eq), int(systems[0].n_var), tpe.ctypes.data, exps.ctypes.data,
                                     len(systems), coefs.ctypes.data, gam.ctypes.data, ctypes.byref(out)))
    return Homotopy(out.value, int(systems[0].n_var))


def phc_make_parameter_homotopy(target, start_coefs, gamma: complex = 1.0) -> Homotopy:
    """(1-t) gamma g + t f: f = ``target`` (one system, or a list of systems
    sharing supports: one per target), g = the supports with the
    coefficients ``start_coefs``."""
    L = load()
    systems = target if isinstance(target, (list, tuple)) else [target]
    tpe, exps, _ = _lists(systems[0])
    for t in systems[1:]:
        if not (np.array_equal(np.asarray(t.terms_per_eq), tpe) and np.array_equal(np.asarray(t.exps), exps)):
            raise ValueError("targets must share terms_per_eq and exps")
    ct = np.ascontiguousarray(np.stack([np.asarray(t.coefs, dtype=np.complex128) for t in systems]))
    cs = np.ascontiguousarray(np.asarray(start_coefs, dtype=np.complex128).reshape(-1))
    out = ctypes.c_void_p()
    _check(L.phc_make_parameter_homotopy(int(systems[0].n_eq), int(systems[0].n_var), tpe.ctypes.data,
                                         exps.ctypes.data, len(systems), cs.ctypes.data, ct.ctypes.data,
                                         phc_cd(float(np.real(gamma)), float(np.imag(gamma))), ctypes.byref(out)))
    return Homotopy(out.value, int(systems[0].n_var))


def phc_mixed_cells(sys, lift):
    """Fine mixed cells of the supports of ``sys`` under the integer lifting
    ``lift`` [T] (host call): (cells int32 [n_cells, n, 2] of global term
    indices, volumes int64 [n_cells], mixed volume)."""
    L = load()
    tpe, exps, _ = _lists(sys)
    w = np.ascontiguousarray(np.asarray(lift).reshape(-1), dtype=np.int32)
    n = int(sys.n_var)
    count, mv = ctypes.c_int64(), ctypes.c_int64()
    cap = 1 << 16
    while True:  # a second enumeration only when the first buffer was too small
        cells = np.zeros((cap, n, 2), dtype=np.int32)
        vols = np.zeros(cap, dtype=np.int64)
        _check(L.phc_mixed_cells(n, tpe.ctypes.data, exps.ctypes.data, w.ctypes.data, cap, cells.ctypes.data,
                                 vols.ctypes.data, ctypes.byref(count), ctypes.byref(mv)))
        if count.value <= cap:
            return cells[:count.value].copy(), vols[:count.value].copy(), int(mv.value)
        cap = int(count.value)


def phc_make_polyhedral_homotopy(sys, lift, cells) -> Homotopy:
    """Polyhedral homotopies of ``sys`` (coefficients in general position)
    over ``cells`` (int32 [n_cells, n, 2] from phc_mixed_cells, same lift)."""
    L = load()
    tpe, exps, coefs = _lists(sys)
    w = np.ascontiguousarray(np.asarray(lift).reshape(-1), dtype=np.int32)
    c = np.ascontiguousarray(np.asarray(cells, dtype=np.int32))
    out = ctypes.c_void_p()
    _check(L.phc_make_polyhedral_homotopy(int(sys.n_var), tpe.ctypes.data, exps.ctypes.data, coefs.ctypes.data,
                                          w.ctypes.data, c.ctypes.data, int(c.shape[0]), ctypes.byref(out)))
    return Homotopy(out.value, int(sys.n_var))


def phc_polyhedral_starts(h: Homotopy, first_path: int, n_paths: int, x_out, stream=None):
    _check(load().phc_polyhedral_starts(ctypes.c_void_p(h.ptr), int(first_path), int(n_paths), _ptr(x_out),
                                        _stream_ptr(stream)))


def phc_track_polyhedral(h: Homotopy, first_path: int, n_paths: int, opts, x_out, cls_out, stats_out=None,
                         stream=None):
    _check(load().phc_track_polyhedral(ctypes.c_void_p(h.ptr), int(first_path), int(n_paths),
                                       ctypes.byref(opts) if opts is not None else None, _ptr(x_out), _ptr(cls_out),
                                       _ptr(stats_out), _stream_ptr(stream)))


def phc_solve_polyhedral(sys, lift, opts, max_paths: int, x_out, cls_out, stats_out=None, stream=None):
    """Cells on this thread, paths on the GPU as the cells come (Figure 2);
    returns (mixed volume, number of cells)."""
    L = load()
    tpe, exps, coefs = _lists(sys)
    w = np.ascontiguousarray(np.asarray(lift).reshape(-1), dtype=np.int32)
    npaths, ncells = ctypes.c_int64(), ctypes.c_int64()
    _check(L.phc_solve_polyhedral(int(sys.n_var), tpe.ctypes.data, exps.ctypes.data, coefs.ctypes.data,
                                  w.ctypes.data, ctypes.byref(opts) if opts is not None else None, int(max_paths),
                                  _ptr(x_out), _ptr(cls_out), _ptr(stats_out), ctypes.byref(npaths),
                                  ctypes.byref(ncells), _stream_ptr(stream)))
    return int(npaths.value), int(ncells.value)


def phc_track_from(h: Homotopy, starts, n_starts: int, starts_per_system: int, opts, x_out, cls_out,
                   stats_out=None, stream=None):
    """starts: complex128 CUDA tensor [n_var, n_starts] (SoA)."""
    _check(load().phc_track_from(ctypes.c_void_p(h.ptr), _ptr(starts), int(n_starts), int(starts_per_system),
                                 ctypes.byref(opts) if opts is not None else None, _ptr(x_out), _ptr(cls_out),
                                 _ptr(stats_out), _stream_ptr(stream)))


def phc_membership_test(emb, k: int, witness, points, tol: float, opts, on_out, x_out=None, cls_out=None,
                        stream=None):
    """emb: the embedded system E_k (lists); witness: complex128 CUDA tensor
    [n_var, m]; points: host array [p, n_var - k]; on_out: uint8 CUDA tensor [p]."""
    L = load()
    tpe, exps, coefs = _lists(emb)
    pts = np.ascontiguousarray(np.atleast_2d(np.asarray(points, dtype=np.complex128)))
    if 1 <= int(k) < int(emb.n_var) and pts.shape[1] != int(emb.n_var) - int(k):
        raise ValueError(f"test points need {int(emb.n_var) - int(k)} coordinates, got {pts.shape[1]}")
    m = int(witness.shape[1])
    _check(L.phc_membership_test(int(emb.n_eq), int(emb.n_var), tpe.ctypes.data, exps.ctypes.data,
                                 coefs.ctypes.data, int(k), _ptr(witness), m, pts.ctypes.data, pts.shape[0],
                                 ctypes.c_double(tol), ctypes.byref(opts) if opts is not None else None,
                                 _ptr(on_out), _ptr(x_out), _ptr(cls_out), _stream_ptr(stream)))


def phc_num_paths(h: Homotopy) -> int:
    v = ctypes.c_int64()
    _check(load().phc_num_paths(ctypes.c_void_p(h.ptr), ctypes.byref(v)))
    return int(v.value)


def phc_tail_paths(h: Homotopy, stream=None, units: bool = False):
    """Paths the last tracking call on h handed to a tail
    kernel (with units=True: (paths, units run in the tail kernel))."""
    v = ctypes.c_int64()
    u = ctypes.c_int64()
    _check(load().phc_tail_paths(ctypes.c_void_p(h.ptr), ctypes.c_void_p(_stream_ptr(stream)), ctypes.byref(v),
                                 ctypes.byref(u)))
    return (int(v.value), int(u.value)) if units else int(v.value)


def phc_track_paths(h: Homotopy, first_path: int, n_paths: int, opts, x_out, cls_out, stats_out=None, stream=None):
    """x_out: complex128 CUDA tensor [n_var, n_paths]; cls_out: int8 [n_paths];
    stats_out: uint8 [n_paths, 80] or None."""
    _check(load().phc_track_paths(ctypes.c_void_p(h.ptr), int(first_path), int(n_paths),
                                  ctypes.byref(opts) if opts is not None else None, _ptr(x_out), _ptr(cls_out),
                                  _ptr(stats_out), _stream_ptr(stream)))


def phc_track_paths_dd(h: Homotopy, first_path: int, n_paths: int, opts, x_hi, x_lo, cls_out, stats_out=None,
                       stream=None):
    """Tracking in complex double double: x_hi, x_lo complex128 [n_var, n_paths]."""
    _check(load().phc_track_paths_dd(ctypes.c_void_p(h.ptr), int(first_path), int(n_paths),
                                     ctypes.byref(opts) if opts is not None else None, _ptr(x_hi), _ptr(x_lo),
                                     _ptr(cls_out), _ptr(stats_out), _stream_ptr(stream)))


def phc_track_paths_qd(h: Homotopy, first_path: int, n_paths: int, opts, x_out, cls_out, stats_out=None,
                       stream=None):
    """x_out: complex128 CUDA tensor [4, n_var, n_paths] (the four parts)."""
    _check(load().phc_track_paths_qd(ctypes.c_void_p(h.ptr), int(first_path), int(n_paths),
                                     ctypes.byref(opts) if opts is not None else None, _ptr(x_out), _ptr(cls_out),
                                     _ptr(stats_out), _stream_ptr(stream)))


def phc_endgame(h: Homotopy, first_path: int, n_paths: int, opts, x_out, cycle_out, stats_out=None, stream=None):
    """Cauchy endgame: x_out complex128 [n_var, n_paths], cycle_out int32 [n_paths]."""
    _check(load().phc_endgame(ctypes.c_void_p(h.ptr), int(first_path), int(n_paths),
                              ctypes.byref(opts) if opts is not None else None, _ptr(x_out), _ptr(cycle_out),
                              _ptr(stats_out), _stream_ptr(stream)))


def phc_fp64_probe(warps_per_block: int = 16, iters: int = 200_000, stream=None) -> float:
    """Measured FP64 rate of the current device in TFLOP/s (synchronizes)."""
    out = ctypes.c_double(0.0)
    _check(load().phc_fp64_probe(int(warps_per_block), int(iters), ctypes.byref(out), _stream_ptr(stream)))
    return out.value


def phc_track_paths_noalloc(h: Homotopy, first_path: int, n_paths: int, opts, x_out, cls_out, stats_out=None,
                            stream=None):
    """phc_track_paths without device allocation during the call (static scratch)."""
    _check(load().phc_track_paths_noalloc(ctypes.c_void_p(h.ptr), int(first_path), int(n_paths),
                                          ctypes.byref(opts) if opts is not None else None, _ptr(x_out),
                                          _ptr(cls_out), _ptr(stats_out), _stream_ptr(stream)))


class SystemLists:
    """Host copy of a phc_system_lists (the output of phc_embed)."""

    def __init__(self, n_eq, n_var, terms_per_eq, exps, coefs):
        self.n_eq, self.n_var = int(n_eq), int(n_var)
        self.terms_per_eq, self.exps, self.coefs = terms_per_eq, exps, coefs


def phc_embed(sys, top_dim: int, gammas=None, hyper=None, seed: int = 0) -> SystemLists:
    L = load()
    tpe, exps, coefs = _lists(sys)
    g = None if gammas is None else np.ascontiguousarray(gammas, dtype=np.complex128)
    hy = None if hyper is None else np.ascontiguousarray(hyper, dtype=np.complex128)
    out = ctypes.POINTER(phc_system_lists)()
    _check(L.phc_embed(int(sys.n_eq), int(sys.n_var), tpe.ctypes.data, exps.ctypes.data, coefs.ctypes.data,
                       int(top_dim), None if g is None else g.ctypes.data, None if hy is None else hy.ctypes.data,
                       ctypes.c_uint64(seed), ctypes.byref(out)))
    s = out.contents
    T, N = s.n_terms, s.n_var
    res = SystemLists(
        s.n_eq, N,
        np.ctypeslib.as_array(s.terms_per_eq, shape=(s.n_eq,)).copy(),
        np.ctypeslib.as_array(s.exps, shape=(T * N,)).copy().reshape(T, N),
        np.ctypeslib.as_array(ctypes.cast(s.coefs, ctypes.POINTER(ctypes.c_double)), shape=(2 * T,)).copy()
        .view(np.complex128),
    )
    L.phc_free_lists(out)
    return res


def _copy_lists(L, out) -> SystemLists:
    s = out.contents
    T, N = s.n_terms, s.n_var
    res = SystemLists(
        s.n_eq, N,
        np.ctypeslib.as_array(s.terms_per_eq, shape=(s.n_eq,)).copy(),
        np.ctypeslib.as_array(s.exps, shape=(T * N,)).copy().reshape(T, N),
        np.ctypeslib.as_array(ctypes.cast(s.coefs, ctypes.POINTER(ctypes.c_double)), shape=(2 * T,)).copy()
        .view(np.complex128),
    )
    L.phc_free_lists(out)
    return res


def phc_square(sys, consts=None, seed: int = 0) -> SystemLists:
    """The square system of Section 2.1 (random hyperplanes for an
    underdetermined, new unknowns with random multipliers for an
    overdetermined system)."""
    L = load()
    tpe, exps, coefs = _lists(sys)
    c = None if consts is None else np.ascontiguousarray(consts, dtype=np.complex128)
    out = ctypes.POINTER(phc_system_lists)()
    _check(L.phc_square(int(sys.n_eq), int(sys.n_var), tpe.ctypes.data, exps.ctypes.data, coefs.ctypes.data,
                        None if c is None else c.ctypes.data, ctypes.c_uint64(seed), ctypes.byref(out)))
    return _copy_lists(L, out)


def phc_cascade_stage(h: Homotopy, k: int, starts, n_starts: int, opts, x_out, cls_out, slack_zero_out,
                      stats_out=None, stream=None):
    _check(load().phc_cascade_stage(ctypes.c_void_p(h.ptr), int(k), _ptr(starts), int(n_starts),
                                    ctypes.byref(opts) if opts is not None else None, _ptr(x_out), _ptr(cls_out),
                                    _ptr(slack_zero_out), _ptr(stats_out), _stream_ptr(stream)))


def phc_cascade_from(h: Homotopy, k: int, x_prev, cls_prev, slack_zero_prev, n: int, opts, x_out, cls_out,
                     slack_zero_out, stats_out=None, stream=None):
    _check(load().phc_cascade_from(ctypes.c_void_p(h.ptr), int(k), _ptr(x_prev), _ptr(cls_prev),
                                   _ptr(slack_zero_prev), int(n), ctypes.byref(opts) if opts is not None else None,
                                   _ptr(x_out), _ptr(cls_out), _ptr(slack_zero_out), _ptr(stats_out),
                                   _stream_ptr(stream)))


def phc_track_many(hs, opts, x_outs, cls_outs, stats_outs=None, stream=None):
    """Track every path of the handles hs in one launch per number of unknowns."""
    n = len(hs)
    H = (ctypes.c_void_p * n)(*[h.ptr for h in hs])
    X = (ctypes.c_void_p * n)(*[_ptr(x) for x in x_outs])
    C = (ctypes.c_void_p * n)(*[_ptr(c) for c in cls_outs])
    S = None if stats_outs is None else (ctypes.c_void_p * n)(*[_ptr(t) for t in stats_outs])
    _check(load().phc_track_many(H, n, ctypes.byref(opts) if opts is not None else None, X, C, S,
                                 _stream_ptr(stream)))


class ManyPlan:
    """Owning wrapper of a phc_many_plan* (destroyed with the object); keeps
    the handles and output tensors it refers to alive."""

    def __init__(self, ptr: int, keep):
        self.ptr = ptr
        self._keep = keep

    def __del__(self):
        if getattr(self, "ptr", None) and _lib is not None:
            _lib.phc_many_plan_destroy(ctypes.c_void_p(self.ptr))
            self.ptr = None


def phc_many_plan_create(hs, opts, x_outs, cls_outs, stats_outs=None, stream=None) -> ManyPlan:
    n = len(hs)
    H = (ctypes.c_void_p * n)(*[h.ptr for h in hs])
    X = (ctypes.c_void_p * n)(*[_ptr(x) for x in x_outs])
    C = (ctypes.c_void_p * n)(*[_ptr(c) for c in cls_outs])
    S = None if stats_outs is None else (ctypes.c_void_p * n)(*[_ptr(t) for t in stats_outs])
    out = ctypes.c_void_p()
    _check(load().phc_many_plan_create(H, n, ctypes.byref(opts) if opts is not None else None, X, C, S,
                                       _stream_ptr(stream), ctypes.byref(out)))
    return ManyPlan(out.value, (list(hs), list(x_outs), list(cls_outs), stats_outs))


def phc_many_plan_run(plan: ManyPlan, stream=None):
    _check(load().phc_many_plan_run(ctypes.c_void_p(plan.ptr), _stream_ptr(stream)))


def phc_track_pipeline(h: Homotopy, k: int, first_path: int, n_paths: int, opts, x_top, cls_top, stats_top, x_next,
                       cls_next, slack_zero_next, stats_next, stream=None):
    _check(load().phc_track_pipeline(ctypes.c_void_p(h.ptr), int(k), int(first_path), int(n_paths),
                                     ctypes.byref(opts) if opts is not None else None, _ptr(x_top), _ptr(cls_top),
                                     _ptr(stats_top), _ptr(x_next), _ptr(cls_next), _ptr(slack_zero_next),
                                     _ptr(stats_next), _stream_ptr(stream)))


def phc_refine_endpoints(h: Homotopy, x_hi, x_lo, n: int, cond_threshold: float, cond_max: float, max_iters: int,
                         cls, stats, stream=None):
    _check(load().phc_refine_endpoints(ctypes.c_void_p(h.ptr), _ptr(x_hi), _ptr(x_lo), int(n),
                                       ctypes.c_double(cond_threshold), ctypes.c_double(cond_max), int(max_iters),
                                       _ptr(cls), _ptr(stats), _stream_ptr(stream)))


def phc_last_error() -> str:
    return load().phc_last_error().decode()
