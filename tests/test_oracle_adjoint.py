"""Pins of the oracle's adjoints (vector-Jacobian products) of the corrected images (Eq. 1) and
of J (Eq. 2-5) at fixed b, against what the definitions fix independently of the adjoint code:

  - T+ is linear in I+ and T- in I-: for any image v, <g, T+(v)> = <dI+, v> with the forward
    model evaluated by the oracle's own forward pass (no finite differences needed);
  - the field part: central finite differences of <g+, T+(b)> + <g-, T-(b)> in pure double
    precision, on nodes whose perturbation does not move any interpolation cell (the image model
    is piecewise linear in the position);
  - dJ/dI+-: J is quadratic in the images, so central differences with a dyadic step on dyadic
    images are exact up to double rounding.
"""
import numpy as np
import pytest

from paper_2403_10706_b300 import phantom as ph

ALPHA, BETA = 300.0, 1e4
GEOMS = [  # (dims, spacing, pe)
    ((4, 6, 5), (1.0, 1.25, 0.9), 1),
    ((7, 3, 4), (1.1, 1.0, 1.2), 0),
    ((3, 4, 9), (0.9, 1.3, 1.0), 2),
    ((1, 12, 1), (1.0, 1.0, 1.0), 1),
]


def setup(orc, dims, spacing, p, seed, bscale=2.5):
    P = orc.Problem(dims, spacing, p, ALPHA, BETA)
    Ip, Im = ph.random_images(dims, seed, 0.1, 1.0)
    b = ph.random_field(dims, p, seed + 1, scale=bscale, smooth=1.0, max_slope=0.6)
    rng = np.random.default_rng(seed + 2)
    gp, gm = rng.normal(size=dims), rng.normal(size=dims)
    return P, Ip, Im, b.astype(np.float64), gp, gm


@pytest.mark.parametrize("contract", [True, False])
@pytest.mark.parametrize("dims,spacing,p", GEOMS)
def test_image_adjoint_is_the_transpose_of_the_forward_model(orc, dims, spacing, p, contract):
    P, Ip, Im, b, gp, gm = setup(orc, dims, spacing, p, 11)
    dIp, dIm, _ = P.correct_adjoint(Ip, Im, b, gp, gm, contract=contract)
    rng = np.random.default_rng(5)
    for _ in range(3):
        vp = rng.normal(size=dims).astype(np.float32)
        vm = rng.normal(size=dims).astype(np.float32)
        T = P.eval(vp, vm, b, contract=contract, grad=False, corrected=True)
        lhs = np.sum(gp * T["Tp"]) + np.sum(gm * T["Tm"])
        rhs = np.sum(dIp * vp) + np.sum(dIm * vm)
        assert abs(lhs - rhs) <= 1e-12 * (np.sum(np.abs(gp * T["Tp"])) + np.sum(np.abs(gm * T["Tm"])))
    # each image gets only its own sensitivity
    dIp0, dIm0, _ = P.correct_adjoint(Ip, Im, b, gp, None, contract=contract)
    assert np.array_equal(dIp0, dIp) and not dIm0.any()


@pytest.mark.parametrize("dims,spacing,p", GEOMS)
def test_field_adjoint_matches_finite_differences(orc, dims, spacing, p):
    P, Ip, Im, b, gp, gm = setup(orc, dims, spacing, p, 21)
    _, _, db = P.correct_adjoint(Ip, Im, b, gp, gm, contract=False)

    def L(bb):
        T = P.eval(Ip, Im, bb, contract=False, grad=False, corrected=True, cells=True)
        return np.sum(gp * T["Tp"]) + np.sum(gm * T["Tm"]), T["cell_p"], T["cell_m"]

    h, checked = 1e-6, 0
    scale = np.abs(db).max()
    for k in range(b.size):
        e = np.zeros(b.size)
        e[k] = h
        e = e.reshape(b.shape)
        Lp, cpp, cmp_ = L(b + e)
        Lm, cpm, cmm = L(b - e)
        if not (np.array_equal(cpp, cpm) and np.array_equal(cmp_, cmm)):
            continue   # the perturbation moves a cell: the model has a kink there
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - db.ravel()[k]) <= 1e-6 * scale, (k, fd, db.ravel()[k])
        checked += 1
    assert checked >= 0.9 * b.size


def dyadic_images(dims, seed):
    rng = np.random.default_rng(seed)
    Ip = rng.integers(400, 4096, size=dims) / 4096.0
    Im = rng.integers(400, 4096, size=dims) / 4096.0
    return Ip.astype(np.float32), Im.astype(np.float32)


@pytest.mark.parametrize("contract", [True, False])
@pytest.mark.parametrize("dims,spacing,p", GEOMS)
def test_image_gradient_of_J_matches_exact_central_differences(orc, dims, spacing, p, contract):
    P = orc.Problem(dims, spacing, p, ALPHA, BETA)
    Ip, Im = dyadic_images(dims, 31)
    b = ph.random_field(dims, p, 32, scale=2.0, smooth=1.0, max_slope=0.6).astype(np.float64)
    dIp, dIm = P.image_grad(Ip, Im, b, contract=contract)
    h = 2.0 ** -8   # Ip +- h is exact in single precision for these dyadic values
    scale = max(np.abs(dIp).max(), np.abs(dIm).max())
    for which, grad in ((0, dIp), (1, dIm)):
        for k in range(Ip.size):
            imgs = [Ip.copy(), Im.copy()]
            imgs[which].ravel()[k] += h
            Jp = P.eval(imgs[0], imgs[1], b, contract=contract, grad=False)["J"]
            imgs[which].ravel()[k] -= 2 * h
            Jm = P.eval(imgs[0], imgs[1], b, contract=contract, grad=False)["J"]
            fd = (Jp - Jm) / (2 * h)
            assert abs(fd - grad.ravel()[k]) <= 1e-9 * scale + 1e-9 * abs(Jp), (which, k)


def test_image_gradient_vanishes_for_a_consistent_pair(orc):
    """I+ = I- and b = 0 give r = 0, hence dJ/dI+- = 0 (J = 0 there)."""
    dims, p = (5, 8, 4), 1
    P = orc.Problem(dims, (1.0, 1.0, 1.0), p, ALPHA, BETA)
    I = ph.random_images(dims, 41, 0.1, 1.0)[0]
    b = np.zeros(ph.field_dims(dims, p))
    dIp, dIm = P.image_grad(I, I, b)
    assert not dIp.any() and not dIm.any()
