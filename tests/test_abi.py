"""C-ABI boundary on CPU: the library loads, exports every symbol the header
declares, mirrors its structs, and rejects bad input before touching a GPU.
Host-side logic (the embedding) is compared with the oracle's."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import paper_1804_03807_gb300 as P
from paper_1804_03807_gb300 import _lib
from workloads import PolySystem, configs, cyclic, embedding_constants, multistep_example, rng_for

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "phc.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(phc_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = P.load()
    names = declared_functions()
    assert "phc_track_paths" in names and "phc_cascade_stage" in names
    for name in names:
        assert hasattr(L, name), name
    assert set(_lib.EXPORTED) <= set(names)


def test_struct_mirrors():
    L = P.load()
    assert L.phc_sizeof_opts() == ctypes.sizeof(_lib.phc_opts)
    assert L.phc_sizeof_stats() == P.STATS_DTYPE.itemsize == 80


def test_default_opts_match_the_oracle_readings():
    g = P.phc_default_opts()
    o = oracle.default_opts()
    for name, _ in oracle.Opts._fields_:
        assert getattr(g, name) == getattr(o, name), name


def test_default_launch_options():
    """Options with no counterpart in the oracle (they never change a
    result): the tail hand-off on by default at 0.8 idle with 32 threads per
    path, double precision, library-chosen grid."""
    g = P.phc_default_opts()
    assert g.tail_drain == 0.8 and g.tail_threads == 0 and g.compact == 1
    assert g.precision == P.PHC_PREC_FP64 and g.block_threads == 0 and g.max_blocks == 0
    assert g.fp32_t_max == 0.9 and g.fp32_pivot_ratio == 1e4


def _bad(sys_kwargs):
    base = dict(n_eq=2, n_var=2, terms_per_eq=np.array([2, 2]),
                exps=np.array([[1, 0], [0, 0], [0, 1], [0, 0]], dtype=np.uint8),
                coefs=np.array([1, -1, 1, -1], dtype=complex))
    base.update(sys_kwargs)

    class S:
        pass

    s = S()
    for k, v in base.items():
        setattr(s, k, v)
    return s


@pytest.mark.parametrize("kw,needle", [
    (dict(n_eq=1, terms_per_eq=np.array([4])), "square"),
    (dict(coefs=np.array([1, np.nan, 1, -1], dtype=complex)), "not finite"),
    (dict(exps=np.zeros((4, 2), dtype=np.uint8)), "degree 0"),
    (dict(terms_per_eq=np.array([4, 0])), "no terms"),
])
def test_make_homotopy_rejects_bad_systems(kw, needle):
    with pytest.raises(P.PhcError) as ei:
        P.phc_make_homotopy(_bad(kw), 1.0)
    assert ei.value.code == _lib.PHC_EINVAL
    assert needle in str(ei.value)


def test_make_homotopy_rejects_zero_gamma_and_too_many_unknowns():
    with pytest.raises(P.PhcError):
        P.phc_make_homotopy(cyclic(3), 0.0)
    with pytest.raises(P.PhcError) as ei:
        P.phc_make_homotopy(cyclic(13), 1.0)
    assert "outside" in str(ei.value)


@pytest.mark.parametrize("sys,D,seed", [(cyclic(4), 1, 1), (cyclic(5), 2, 2), (multistep_example(), 3, 3)])
def test_embedding_matches_the_oracle(sys, D, seed):
    g, hy = embedding_constants(rng_for(seed), sys.n_eq, sys.n_var, D)
    a = P.phc_embed(sys, D, g, hy)
    b = oracle.embed(sys, D, g, hy)
    assert (a.n_eq, a.n_var) == (b.n_eq, b.n_var)
    assert np.array_equal(a.terms_per_eq, b.terms_per_eq)
    assert np.array_equal(a.exps, b.exps)
    assert np.array_equal(a.coefs, b.coefs)


def test_embedding_lower_dimension_is_the_dropped_slack():
    """E_{k-1} from the first k-1 constants equals E_k with z_k = 0 and
    hyperplane k removed (what each cascade stage lands on)."""
    sys = multistep_example()
    g, hy = embedding_constants(rng_for(4), 4, 4, 3)
    e3 = oracle.embed(sys, 3, g, hy)
    e2 = P.phc_embed(sys, 2, g[:, :2], hy[:2])
    d = oracle.drop_last_slack(e3, 4, 4, 3)
    assert np.array_equal(e2.terms_per_eq, d.terms_per_eq)
    assert np.array_equal(e2.exps, d.exps)
    assert np.array_equal(e2.coefs, d.coefs)


def test_embed_errors_and_seeded_constants():
    with pytest.raises(P.PhcError):
        P.phc_embed(cyclic(4), -1)
    with pytest.raises(P.PhcError):
        P.phc_embed(cyclic(8), 5)  # 13 unknowns
    a = P.phc_embed(cyclic(4), 1, seed=7)
    b = P.phc_embed(cyclic(4), 1, seed=7)
    c = P.phc_embed(cyclic(4), 1, seed=8)
    assert np.array_equal(a.coefs, b.coefs) and not np.array_equal(a.coefs, c.coefs)


def test_parameter_homotopy_and_membership_reject_bad_input():
    """Checked on the host before any device work."""
    s = cyclic(3)
    with pytest.raises(P.PhcError) as e:
        P.phc_make_parameter_homotopy(s, s.coefs, 0.0)
    assert e.value.code == P._lib.PHC_EINVAL and "gamma" in str(e.value)
    bad = np.array(s.coefs, dtype=complex)
    bad[1] = np.nan
    with pytest.raises(P.PhcError) as e:
        P.phc_make_parameter_homotopy(s, bad, 1.0)
    assert "start coefficient" in str(e.value)
    E = P.phc_embed(multistep_example(), 1, *embedding_constants(rng_for(5), 4, 4, 1))

    class Fake:  # stands for device tensors: never dereferenced on these paths
        def __init__(self, shape):
            self.shape = shape

        def data_ptr(self):
            return 16

        def contiguous(self):
            return self

    on = Fake((1,))
    for k, tol, needle in [(0, 1e-3, "k = 0"), (5, 1e-3, "k = 5"), (1, 0.0, "tol")]:
        with pytest.raises(P.PhcError) as e:
            P.phc_membership_test(E, k, Fake((5, 1)), np.zeros((1, 4)), tol, None, on, stream=0)
        assert needle in str(e.value)
    # the last equation of the original system is not a hyperplane
    with pytest.raises(P.PhcError) as e:
        P.phc_membership_test(multistep_example(), 1, Fake((4, 1)), np.zeros((1, 3)), 1e-3, None, on, stream=0)
    assert "not a hyperplane" in str(e.value)
    pts = np.zeros((1, 4), complex)
    pts[0, 2] = np.inf
    with pytest.raises(P.PhcError) as e:
        P.phc_membership_test(E, 1, Fake((5, 1)), pts, 1e-3, None, on, stream=0)
    assert "not finite" in str(e.value)


def test_square_matches_the_oracle():
    """phc_square (host code of the library) against the oracle's list
    manipulation, with the same constants: an underdetermined, an
    overdetermined and a square system."""
    rng = rng_for(81)
    sphere = PolySystem(1, 3, np.array([4]), np.array([[2, 0, 0], [0, 2, 0], [0, 0, 2], [0, 0, 0]], np.uint8),
                        np.array([1, 1, 1, -1], complex), name="sphere")
    over = PolySystem(3, 2, np.array([2, 2, 2]), np.array([[1, 0], [0, 0], [0, 1], [0, 0], [1, 1], [0, 0]], np.uint8),
                      np.array([1, -1, 1, -2, 1, -2], complex), name="over")
    for sys, shape in [(sphere, (2, 4)), (over, (3, 1)), (cyclic(4), (0, 0))]:
        c = rng.normal(size=shape) + 1j * rng.normal(size=shape)
        a = P.phc_square(sys, c if c.size else None)
        b = oracle.square(sys, c)
        assert (a.n_eq, a.n_var) == (b.n_eq, b.n_var) == (max(sys.n_eq, sys.n_var),) * 2
        assert np.array_equal(a.terms_per_eq, b.terms_per_eq)
        assert np.array_equal(a.exps, b.exps)
        assert np.array_equal(a.coefs, b.coefs)
    with pytest.raises(P.PhcError):
        P.phc_embed(sphere, 1)  # embedding needs a square system
