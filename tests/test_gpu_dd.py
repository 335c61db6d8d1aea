"""Path tracking in complex double double (Section 5, Table 2: the solver in
double double arithmetic) on the GPU, through the C ABI, against the oracle's
double double tracker: equal class counts; regular endpoints matched one to
one on their double parts within 1e-10, and then equal as double double
values within 1e-24 relative; every regular endpoint a root of f to 1e-28 in
exact rational arithmetic."""
import numpy as np
import pytest

import oracle
import paper_1804_03807_gb300 as P
from workloads import configs, cyclic, rng_for, unit_gamma, univariate
from tests._checks import exact_residual, match_sets

pytestmark = pytest.mark.gpu


def _compare(sys, gamma, check_residual=8):
    h = P.phc_make_homotopy(sys, gamma)
    r, xlo = P.track_dd(h)
    xg, lg = r.x.cpu().numpy().T, xlo.cpu().numpy().T
    cg = r.cls.cpu().numpy()
    xo, lo, co, _ = oracle.track_dd(oracle.total_degree(sys, gamma))
    assert np.array_equal(np.bincount(cg, minlength=4), np.bincount(co, minlength=4))
    Rg, Ro = np.where(cg == 0)[0], np.where(co == 0)[0]
    ra, rb, rel = match_sets(xg[Rg], xo[Ro])
    assert len(ra) == len(Rg) and (len(rel) == 0 or rel.max() <= 1e-10)
    for a, b in zip(Rg[ra], Ro[rb]):
        d = np.max(np.abs((xg[a] - xo[b]) + (lg[a] - lo[b])))
        assert d <= 1e-24 * (1 + np.abs(xo[b]).max()), d
    for a in Rg[:check_residual]:
        assert exact_residual(sys, xg[a], lg[a]) <= 1e-28
    return cg


def test_dd_dense4():
    w = configs.dense4()
    cg = _compare(w.systems[0], w.gammas[0], check_residual=16)
    assert np.all(cg == P.PHC_REGULAR)


def test_dd_univariate_and_cyclic():
    rng = rng_for(93)
    c = rng.normal(size=8) + 1j * rng.normal(size=8)
    _compare(univariate(c), unit_gamma(rng))
    for n in (5, 6):
        _compare(cyclic(n), unit_gamma(rng_for(94 + n)))


def test_dd_batch_handle_and_sub_range():
    """A batch handle (cyclic 5 and two random-coefficient copies): a
    sub-range across the system boundary gives, path for path, what the whole
    range gives."""
    w = configs.cyclic_batch(5, 2, seed=804)
    hb = P.phc_make_homotopy_batch(w.systems, w.gammas)
    r, xlo = P.track_dd(hb)
    r2, xlo2 = P.track_dd(hb, first=100, n_paths=50)
    assert np.array_equal(r2.cls.cpu().numpy(), r.cls.cpu().numpy()[100:150])
    assert np.array_equal(r2.x.cpu().numpy(), r.x.cpu().numpy()[:, 100:150])
    assert np.array_equal(xlo2.cpu().numpy(), xlo.cpu().numpy()[:, 100:150])
