"""Path tracking in complex quad double (Section 5, Table 2: the solver in
quad double arithmetic) on the GPU, through the C ABI, against the oracle's
quad double tracker: equal class counts; regular endpoints matched one to one
on their leading parts within 1e-10, then equal as quad double values (the
sums of the four parts, exactly) within 1e-55 relative; every regular
endpoint a root of f to 1e-58 in exact rational arithmetic."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
import paper_1804_03807_gb300 as P
from workloads import configs, cyclic, rng_for, unit_gamma, univariate
from tests._checks import exact_residual_parts, match_sets

pytestmark = pytest.mark.gpu


def _sum_parts(parts):
    return (sum(Fraction(float(v.real)) for v in parts), sum(Fraction(float(v.imag)) for v in parts))


def _compare(sys, gamma, check_residual=8):
    h = P.phc_make_homotopy(sys, gamma)
    r, parts = P.track_qd(h)
    pg = np.transpose(parts.cpu().numpy(), (2, 1, 0))  # [P, n, 4]
    cg = r.cls.cpu().numpy()
    po, co, _ = oracle.track_qd(oracle.total_degree(sys, gamma))
    assert np.array_equal(np.bincount(cg, minlength=4), np.bincount(co, minlength=4))
    Rg, Ro = np.where(cg == 0)[0], np.where(co == 0)[0]
    ra, rb, rel = match_sets(pg[Rg, :, 0], po[Ro, :, 0])
    assert len(ra) == len(Rg) and (len(rel) == 0 or rel.max() <= 1e-10)
    for a, b in zip(Rg[ra], Ro[rb]):
        scale = 1 + np.abs(po[b, :, 0]).max()
        for j in range(sys.n_var):
            ga, oa = _sum_parts(pg[a, j]), _sum_parts(po[b, j])
            d = max(abs(float(ga[0] - oa[0])), abs(float(ga[1] - oa[1])))
            assert d <= 1e-55 * scale, d
    for a in Rg[:check_residual]:
        assert exact_residual_parts(sys, pg[a]) <= 1e-58
    return cg, pg


def test_qd_dense4():
    w = configs.dense4()
    cg, pg = _compare(w.systems[0], w.gammas[0], check_residual=16)
    assert np.all(cg == P.PHC_REGULAR)
    # parts of decreasing magnitude, each below the last bit of the one before
    for k in range(3):
        hi, lo = np.abs(pg[..., k].real), np.abs(pg[..., k + 1].real)
        assert np.all((lo <= hi * 2.0 ** -50) | (lo == 0))


def test_qd_univariate_and_cyclic5():
    rng = rng_for(710)
    c = rng.normal(size=7) + 1j * rng.normal(size=7)
    _compare(univariate(c), unit_gamma(rng))
    _compare(cyclic(5), unit_gamma(rng_for(711)))


def test_qd_sub_range_and_rejections():
    w = configs.cyclic_batch(4, 1, seed=712)
    hb = P.phc_make_homotopy_batch(w.systems, w.gammas)
    r, parts = P.track_qd(hb)
    r2, parts2 = P.track_qd(hb, first=10, n_paths=12)
    assert np.array_equal(r2.cls.cpu().numpy(), r.cls.cpu().numpy()[10:22])
    assert np.array_equal(parts2.cpu().numpy(), parts.cpu().numpy()[:, :, 10:22])
    hp = P.phc_make_parameter_homotopy(w.systems[1], w.systems[0].coefs, 1.0)
    with pytest.raises(P.PhcError, match="total-degree"):
        P.track_qd(hp, n_paths=1)
