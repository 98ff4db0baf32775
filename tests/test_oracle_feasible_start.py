"""The solve's feasible-start rule (a reading where the paper is silent): J is +inf unless
|delta| < 1 in every cell (Eq. 3), so an OT start with a steeper PE difference somewhere is halved
until max |delta| < 1.  Pinned against numpy's max |delta| and the definition of the factor."""
import numpy as np
import pytest

from paper_2403_10706_b300 import phantom as ph

ALPHA, BETA = 300.0, 1e4
BASE = dict(n_ellipsoids=4, n_blobs=3, semi_axes=(3.0, 9.0), smooth=0.5, n_gauss=4,
            sigma=(4.0, 7.0), spacing=(1.0, 1.0, 1.0), bmax=7.0)
# pairs whose blurred OT field has max |delta| of about 1.22 and 1.14 (infeasible starts)
INFEASIBLE = [dict(BASE, dims=(24, 40, 20), pe_dim=1, seed=6043, noise=0.03),
              dict(BASE, dims=(40, 20, 24), pe_dim=0, seed=6036, noise=0.05)]


def expected_factor(b, pe):
    s = np.abs(np.diff(b, axis=pe)).max()
    k = 0
    while s * 2.0 ** -k >= 1.0:
        k += 1
    return 2.0 ** -k


@pytest.mark.parametrize("recipe", INFEASIBLE)
def test_infeasible_ot_start_is_halved_until_feasible(orc, recipe):
    pr = ph.make_pair(recipe)
    P = orc.Problem(pr.dims, pr.spacing, pr.pe_dim, ALPHA, BETA)
    b0 = P.ot_init(pr.Ip, pr.Im, contract=False)
    f = expected_factor(b0, pr.pe_dim)
    assert f < 1.0
    assert np.isinf(P.eval(pr.Ip, pr.Im, b0, contract=False, grad=False)["J"])
    start, status, _ = P.solve(pr.Ip, pr.Im, gn_iters=0, contract=False)
    assert np.array_equal(start, f * b0)
    assert np.abs(np.diff(start, axis=pr.pe_dim)).max() < 1.0
    assert np.isfinite(P.eval(pr.Ip, pr.Im, start, contract=False, grad=False)["J"])
    b, status, st = P.solve(pr.Ip, pr.Im, gn_iters=5, contract=False)
    assert status == 0 and np.all(np.diff(st[:, 0]) <= 0.0)


def test_feasible_start_is_left_unchanged(orc):
    pr = ph.make_pair("tiny")
    P = orc.Problem(pr.dims, pr.spacing, pr.pe_dim, ALPHA, BETA)
    b0 = P.ot_init(pr.Ip, pr.Im, contract=False)
    assert expected_factor(b0, pr.pe_dim) == 1.0
    start, _, _ = P.solve(pr.Ip, pr.Im, gn_iters=0, contract=False)
    assert np.array_equal(start, b0)


def test_factor_definition_at_the_boundary(orc):
    dims, p = (3, 5, 2), 1
    P = orc.Problem(dims, (1.0, 1.0, 1.0), p, ALPHA, BETA)
    fd = ph.field_dims(dims, p)
    b = np.zeros(fd)
    assert P.feasible_start(b)[1] == 1.0
    b[:, 3, :] = 1.0        # a PE difference of exactly 1: infeasible (|delta| < 1 required)
    bb, f = P.feasible_start(b)
    assert f == 0.5 and np.array_equal(bb, 0.5 * b)
    b[:, 3, :] = 4.5        # 4.5 * 2^-3 = 0.5625 < 1 <= 4.5 * 2^-2
    assert P.feasible_start(b)[1] == 0.125
