"""Pins of the oracle's implicit differentiation through the solve: at a stationary point b* of
J, dL/dtheta = -(dg/dtheta)^T v with H v = dL/db* (g = grad J, H the Gauss-Newton Hessian).  Each
piece is checked against exact finite differences of quantities the oracle already computes:
  - v^T dg/dalpha, v^T dg/dbeta: g is affine in alpha and in beta;
  - d(v^T g)/dI+-: v^T g is quadratic in the images (dyadic values and steps make the central
    difference exact up to double rounding);
  - v solves H v = dL/db (residual through the oracle's Hessian-vector product).
"""
import numpy as np
import pytest

from paper_2403_10706_b300 import phantom as ph

ALPHA, BETA = 300.0, 1e4
GEOMS = [((4, 6, 5), (1.0, 1.25, 0.9), 1), ((7, 3, 4), (1.1, 1.0, 1.2), 0),
         ((3, 4, 9), (0.9, 1.3, 1.0), 2)]


def dyadic_images(dims, seed):
    rng = np.random.default_rng(seed)
    return tuple((rng.integers(400, 4096, size=dims) / 4096.0).astype(np.float32) for _ in (0, 1))


def setup(orc, dims, spacing, p, seed):
    Ip, Im = dyadic_images(dims, seed)
    b = ph.random_field(dims, p, seed + 1, scale=2.0, smooth=1.0, max_slope=0.6).astype(np.float64)
    v = np.random.default_rng(seed + 2).normal(size=b.shape)
    return orc.Problem(dims, spacing, p, ALPHA, BETA), Ip, Im, b, v


@pytest.mark.parametrize("contract", [True, False])
@pytest.mark.parametrize("dims,spacing,p", GEOMS)
def test_theta_dots_match_differences_in_the_weights(orc, dims, spacing, p, contract):
    P, Ip, Im, b, v = setup(orc, dims, spacing, p, 100)
    sa, sb = P.theta_dots(Ip, Im, b, v, contract=contract)
    for w, s in ((0, sa), (1, sb)):
        h = 0.25 * (ALPHA, BETA)[w]
        wts = [ALPHA, BETA]
        wts[w] += h
        gp = orc.Problem(dims, spacing, p, *wts).eval(Ip, Im, b, contract=contract)["grad"]
        wts[w] -= 2 * h
        gm = orc.Problem(dims, spacing, p, *wts).eval(Ip, Im, b, contract=contract)["grad"]
        fd = np.sum(v * (gp - gm)) / (2 * h)
        assert abs(fd - s) <= 1e-9 * (abs(s) + np.sum(np.abs(v * gp)) / (ALPHA, BETA)[w])


@pytest.mark.parametrize("contract", [True, False])
@pytest.mark.parametrize("dims,spacing,p", GEOMS)
def test_mixed_image_adjoint_matches_exact_central_differences(orc, dims, spacing, p, contract):
    P, Ip, Im, b, v = setup(orc, dims, spacing, p, 200)
    dIp, dIm = P.mixed_image_adjoint(Ip, Im, b, v, contract=contract)
    h = 2.0 ** -8

    def F(a, c):
        return np.sum(v * P.eval(a, c, b, contract=contract)["grad"])

    scale = max(np.abs(dIp).max(), np.abs(dIm).max())
    for which, got in ((0, dIp), (1, dIm)):
        for k in range(Ip.size):
            imgs = [Ip.copy(), Im.copy()]
            imgs[which].ravel()[k] += h
            Fp = F(*imgs)
            imgs[which].ravel()[k] -= 2 * h
            Fm = F(*imgs)
            fd = (Fp - Fm) / (2 * h)
            assert abs(fd - got.ravel()[k]) <= 1e-9 * scale + 1e-10 * abs(Fp), (which, k)


def test_solve_adjoint_assembles_the_pieces(orc):
    dims, spacing, p = GEOMS[0]
    P, Ip, Im, b, dLdb = setup(orc, dims, spacing, p, 300)
    v, dIp, dIm, da, dbe, it = P.solve_adjoint(Ip, Im, b, dLdb, max_it=500, rtol=1e-12)
    Hv = P.hessvec(Ip, Im, b, v)
    assert np.linalg.norm(Hv - dLdb) <= 1e-9 * np.linalg.norm(dLdb)
    rp, rm = P.mixed_image_adjoint(Ip, Im, b, v)
    sa, sb = P.theta_dots(Ip, Im, b, v)
    assert np.array_equal(dIp, -rp) and np.array_equal(dIm, -rm)
    assert da == -sa and dbe == -sb
