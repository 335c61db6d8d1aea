"""The coefficient-parameter homotopy (Section 2.3), the homotopy membership
test (Section 4.1) and the filters of Section 4.2 on the GPU, through the C
ABI, against the oracle."""
import numpy as np
import pytest
import torch

import oracle
import paper_1804_03807_gb300 as P
from paper_1804_03807_gb300 import filtering
from workloads import configs, embedding_constants, membership_example, multistep_example, rng_for, unit_gamma
from tests._checks import relative_residual, same_set

pytestmark = pytest.mark.gpu
RTOL = 1e-10


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x).T)).cuda()


def _counts(c):
    return np.bincount(np.asarray(c).astype(int), minlength=4)


def test_parameter_homotopy_against_oracle():
    """From the 924 roots of one random cyclic 7 copy to the next copy:
    class counts and regular endpoints equal to the oracle's, every regular
    endpoint a root of the target."""
    w = configs.cyclic7_batch()
    s1, s2 = w.systems[1], w.systems[2]
    xo1, co1, _ = oracle.track(oracle.total_degree(s1, w.gammas[1]))
    R1 = xo1[co1 == 0]
    g = unit_gamma(rng_for(23))
    h = P.phc_make_parameter_homotopy(s2, s1.coefs, g)
    assert P.phc_num_paths(h) == 0
    r = P.track_from(h, _dev(R1))
    xg, cg = r.x.cpu().numpy().T, r.cls.cpu().numpy()
    xo, co, _ = oracle.track(oracle.parameter_homotopy(s2, s1.coefs, g), starts=R1)
    assert np.array_equal(_counts(cg), _counts(co)) and _counts(cg)[0] == 924
    ok, err = same_set(xg[cg == 0], xo[co == 0], RTOL)
    assert ok, err
    assert relative_residual(s2, xg[cg == 0]).max() <= 1e-12
    with pytest.raises(P.PhcError):
        P.track(h, n_paths=1)  # no total-degree start system


def test_parameter_homotopy_several_targets_in_one_launch():
    """Three targets sharing the start: entry q belongs to target q / m; each
    block of results equals the one-target call's, bit for bit."""
    w = configs.cyclic_batch(5, 4, seed=803)
    src = w.systems[1]
    xo, co, _ = oracle.track(oracle.total_degree(src, w.gammas[1]))
    R = xo[co == 0]
    m = len(R)
    targets = w.systems[2:5]
    hb = P.phc_make_parameter_homotopy(targets, src.coefs, 1j)
    starts = _dev(np.concatenate([R] * 3))
    rb = P.track_from(hb, starts, starts_per_system=m)
    for i, t in enumerate(targets):
        h1 = P.phc_make_parameter_homotopy(t, src.coefs, 1j)
        r1 = P.track_from(h1, _dev(R))
        assert np.array_equal(rb.cls.cpu().numpy()[i * m:(i + 1) * m], r1.cls.cpu().numpy())
        assert np.array_equal(rb.x.cpu().numpy()[:, i * m:(i + 1) * m], r1.x.cpu().numpy())
    st = P.stats_numpy(rb.stats)
    assert np.array_equal(st["system"], np.repeat(np.arange(3), m))
    with pytest.raises(P.PhcError):
        P.track_from(hb, _dev(np.concatenate([R] * 4)), starts_per_system=m)  # a fourth target does not exist


@pytest.mark.parametrize("seed", [71, 72])
def test_example_4_1_membership_on_gpu(seed):
    sys = membership_example()
    rng = rng_for(seed)
    g, hy = embedding_constants(rng, 2, 2, 1)
    gamma = unit_gamma(rng)
    E = P.phc_embed(sys, 1, g, hy)
    h = P.phc_make_homotopy(E, gamma)
    r = P.track(h)
    P.refine(h, r)
    x, c = r.x.cpu().numpy().T, r.cls.cpu().numpy()
    W = x[(c == 0) & oracle.slack_zero(x, 2)]
    assert len(W) == 1
    pts = np.array([[2, 0], [1, 5], [1, 0.3 - 2j]], dtype=complex)
    on, ends = P.membership(E, 1, _dev(W), pts)
    assert on.tolist() == [False, True, True]  # (2, 0) is not on the line x1 = 1 (Example 4.1)
    Eo = oracle.embed(sys, 1, g, hy)
    ono, endso = oracle.membership(Eo, 2, 1, W, pts)
    assert on.tolist() == ono.tolist()
    xg = ends.x.cpu().numpy().T
    for t, (xo, co) in enumerate(endso):
        assert np.max(np.abs(xg[t] - xo[0])) <= RTOL * (1 + np.abs(xo).max())


@pytest.mark.parametrize("seed", [41, 42])
def test_example_4_2_filter_on_gpu(seed):
    """The cascade of Example 3.1 on the GPU, then the filters: witness sets
    of degrees 1, 1, 12 equal to the oracle's, exactly the four isolated
    points, and at dimension 0 the same filter stages (points tested, paths,
    points removed) as the oracle's."""
    sys = multistep_example()
    n, D = 4, 3
    rng = rng_for(seed)
    g, hy = embedding_constants(rng, n, n, D)
    gamma = unit_gamma(rng)
    E = P.phc_embed(sys, D, g, hy)
    h = P.phc_make_homotopy(E, gamma)
    r = P.track(h)
    P.refine(h, r)
    levels = {D: (E, r.x, r.cls)}
    prev, Ek = r, E
    for k in range(D, 0, -1):
        hk = P.phc_make_homotopy(Ek, gamma)
        rk = P.cascade_from(hk, k, prev)
        Ek1 = P.phc_embed(sys, k - 1, g[:, :k - 1], hy[:k - 1]) if k > 1 else sys
        hk1 = P.phc_make_homotopy(Ek1, gamma)
        P.refine(hk1, rk)
        levels[k - 1] = (Ek1, rk.x, rk.cls)
        prev, Ek = rk, Ek1
    witness, isolated, stages = filtering.filter_candidates(levels, n)
    assert {k: len(v) for k, v in witness.items()} == {3: 1, 2: 1, 1: 12}
    ok, err = same_set(isolated, np.array([[3, 2, 2, 1], [3, 3, 2, 1], [4, 3, 2, 1], [4, 2, 2, 1]], complex), RTOL)
    assert ok, err
    # the oracle's cascade and filters from the same constants
    import importlib
    mt = importlib.import_module("tests.test_oracle_membership")
    lev_o = mt._cascade_levels(seed)
    wo, iso_o, st_o = oracle.filter_candidates(lev_o, n)
    # candidates at dimension 0 and the filters they go through are the same;
    # above it a singular endpoint on a higher-dimensional set is accurate to
    # about 1e-4 only, so whether its slack passes the 1e-8 zero test can
    # differ between the two sides (such a point is filtered out either way)
    assert [st for st in stages if st[0] == 0] == [st for st in st_o if st[0] == 0]
    for k in (3, 2, 1):
        ok, err = same_set(witness[k], wo[k], 1e-6)
        assert ok, (k, err)


def test_squared_systems_on_gpu():
    """The squaring of Section 2.1 (phc_square) then tracking on the GPU:
    the oracle's classes and regular endpoints, for an underdetermined and an
    overdetermined system."""
    from workloads import PolySystem
    rng = rng_for(84)
    sphere = PolySystem(1, 3, np.array([4]), np.array([[2, 0, 0], [0, 2, 0], [0, 0, 2], [0, 0, 0]], np.uint8),
                        np.array([1, 1, 1, -1], complex), name="sphere")
    over = PolySystem(3, 2, np.array([2, 2, 2]), np.array([[1, 0], [0, 0], [0, 1], [0, 0], [1, 1], [0, 0]], np.uint8),
                      np.array([1, -1, 1, -2, 1, -2], complex), name="over")
    for sys, shape in [(sphere, (2, 4)), (over, (3, 1))]:
        c = rng.normal(size=shape) + 1j * rng.normal(size=shape)
        g = unit_gamma(rng)
        S = P.phc_square(sys, c)
        r = P.track(P.phc_make_homotopy(S, g))
        xo, co, _ = oracle.track(oracle.total_degree(oracle.square(sys, c), g), threads=1)
        cg = r.cls.cpu().numpy()
        assert np.array_equal(_counts(cg), _counts(co)) and _counts(cg)[0] == 2
        ok, err = same_set(r.x.cpu().numpy().T[cg == 0], xo[co == 0], RTOL)
        assert ok, err
