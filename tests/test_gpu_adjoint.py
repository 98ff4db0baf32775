"""Adjoint kernels (hysco_correct_adjoint, hysco_image_grad) and the torch.autograd wrappers,
against the double-precision oracle's adjoints and against central finite differences.

Tolerances: each adjoint entry is a sum of a few single-precision products (<= 3 cells per voxel,
2 cells per node), so relative 1e-5 in the 2-norm and 2e-4 of the largest magnitude per entry,
as for the gradient.  Finite differences (h = 1e-3, double precision, on single PE columns: a
voxel or node only affects its own column) are exact for the image entries up to rounding (the
loss is quadratic in the images) and for the field entries up to O(h^2) (the model is a low-order
polynomial in b between interpolation kinks; nodes whose perturbation crosses a kink are redrawn).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2403_10706_b300 import phantom as ph  # noqa: E402

ALPHA, BETA = 300.0, 1e4
SHAPES = [
    ((7, 13, 5), (1.0, 1.25, 0.9), 1),
    ((9, 6, 11), (1.1, 1.0, 1.2), 0),
    ((5, 4, 17), (0.9, 1.3, 1.0), 2),
    ((1, 33, 1), (1.0, 1.0, 1.0), 1),
    ((40, 3, 37), (1.0, 1.5, 1.0), 1),
]
DT = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}


@pytest.fixture(scope="module")
def H():
    from paper_2403_10706_b300 import build
    build.build()
    from paper_2403_10706_b300.hysco import Hysco
    return Hysco


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return t if dtype is None else t.to(dtype)


def host(t):
    torch.cuda.synchronize()
    return t.detach().float().cpu().numpy().astype(np.float64)


def check(got, ref, what, rtol=1e-5, etol=2e-4):
    scale = max(np.abs(ref).max(), 1e-30)
    err2 = np.linalg.norm((got - ref).ravel()) / max(np.linalg.norm(ref.ravel()), 1e-30)
    errinf = np.abs(got - ref).max() / scale
    assert err2 <= rtol and errinf <= etol, (what, err2, errinf)


def case(dims, p, seed, bscale=2.0, slope=0.6):
    Ip, Im = ph.random_images(dims, seed, 0.1, 1.0)
    b = ph.random_field(dims, p, seed + 1, scale=bscale, smooth=1.0, max_slope=slope)
    rng = np.random.default_rng(seed + 2)
    return Ip, Im, b, rng.normal(size=dims).astype(np.float32), rng.normal(size=dims).astype(np.float32)


@pytest.mark.parametrize("dtype", list(DT))
@pytest.mark.parametrize("dims,spacing,p", SHAPES)
def test_correct_adjoint_matches_oracle(H, orc, dims, spacing, p, dtype):
    Ip, Im, b, gp, gm = case(dims, p, 500)
    td = DT[dtype]
    Ipq, Imq = dev(Ip, td), dev(Im, td)
    h = H(dims, spacing, p, ALPHA, BETA, dtype=td)
    dIp, dIm, db = h.correct_adjoint(Ipq, Imq, dev(b), dev(gp), dev(gm))
    P = orc.Problem(dims, spacing, p, ALPHA, BETA)
    rp, rm, rb = P.correct_adjoint(host(Ipq), host(Imq), b, gp, gm, contract=True)
    check(host(dIp), rp, "dIp")
    check(host(dIm), rm, "dIm")
    check(host(db), rb, "db")


@pytest.mark.parametrize("dims,spacing,p", SHAPES[:3])
def test_correct_adjoint_with_folding_field(H, orc, dims, spacing, p):
    """A field whose PE slope exceeds 1 folds the column (the cell index decreases along it): the
    kernel's in-place path must still give the oracle's adjoint."""
    Ip, Im, b, gp, gm = case(dims, p, 600, bscale=4.0, slope=3.0)
    assert np.abs(np.diff(b, axis=p)).max() > 1.0
    h = H(dims, spacing, p, ALPHA, BETA)
    dIp, dIm, db = h.correct_adjoint(dev(Ip), dev(Im), dev(b), dev(gp), dev(gm))
    P = orc.Problem(dims, spacing, p, ALPHA, BETA)
    rp, rm, rb = P.correct_adjoint(Ip, Im, b, gp, gm, contract=True)
    check(host(dIp), rp, "dIp")
    check(host(dIm), rm, "dIm")
    check(host(db), rb, "db")


@pytest.mark.parametrize("compress", [False, True])
def test_correct_adjoint_long_columns(H, orc, compress):
    """Columns of the 3T length (168 cells: eight segments of 21 per column and image) with a
    smooth field, and with a stretch of PE slope -0.95 in some columns that squeezes ~20 cells of
    the + image into one voxel (a voxel shared by three segments: those columns take the
    single-thread path, the others the segmented one)."""
    dims, spacing, p = (6, 168, 5), (1.25, 1.25, 1.25), 1
    Ip, Im, b, gp, gm = case(dims, p, 650, bscale=3.0)
    if compress:
        b = b.copy()
        for i0, i2 in ((1, 2), (4, 0), (5, 4)):
            ramp = np.zeros(dims[p] + 1)
            ramp[40:70] = -0.95
            b[i0, :, i2] = np.cumsum(ramp) - np.cumsum(ramp).mean()
        assert np.abs(np.diff(b, axis=p)).max() < 1.0
    h = H(dims, spacing, p, ALPHA, BETA)
    dIp, dIm, db = h.correct_adjoint(dev(Ip), dev(Im), dev(b), dev(gp), dev(gm))
    P = orc.Problem(dims, spacing, p, ALPHA, BETA)
    rp, rm, rb = P.correct_adjoint(Ip, Im, b, gp, gm, contract=True)
    check(host(dIp), rp, "dIp")
    check(host(dIm), rm, "dIm")
    check(host(db), rb, "db")


def test_correct_adjoint_optional_arguments(H, orc):
    dims, spacing, p = SHAPES[0]
    Ip, Im, b, gp, gm = case(dims, p, 700)
    h = H(dims, spacing, p, ALPHA, BETA)
    dIp, dIm, db = h.correct_adjoint(dev(Ip), dev(Im), dev(b), dev(gp), None)
    assert not host(dIm).any()
    P = orc.Problem(dims, spacing, p, ALPHA, BETA)
    rp, _, rb = P.correct_adjoint(Ip, Im, b, gp, None, contract=True)
    check(host(dIp), rp, "dIp")
    check(host(db), rb, "db")
    dIp2, dIm2, db2 = h.correct_adjoint(dev(Ip), dev(Im), dev(b), dev(gp), dev(gm),
                                        want=(False, True, False))
    assert dIp2 is None and db2 is None and dIm2 is not None


@pytest.mark.parametrize("dims,spacing,p", SHAPES)
def test_image_grad_matches_oracle(H, orc, dims, spacing, p):
    Ip, Im, b, _, _ = case(dims, p, 800)
    h = H(dims, spacing, p, ALPHA, BETA)
    dIp, dIm = h.image_grad(dev(Ip), dev(Im), dev(b), 1.0)
    P = orc.Problem(dims, spacing, p, ALPHA, BETA)
    rp, rm = P.image_grad(Ip, Im, b, contract=True)
    check(host(dIp), rp, "dJ/dIp")
    check(host(dIm), rm, "dJ/dIm")
    dIp3, _ = h.image_grad(dev(Ip), dev(Im), dev(b), -2.5, want=(True, False))
    check(host(dIp3), -2.5 * rp, "scaled")


def column(a, col, p):
    """PE column `col` (flat over the two other axes, C order) of an image or field."""
    moved = np.moveaxis(a, p, -1)
    return moved.reshape(-1, moved.shape[-1])[col]


def test_autograd_corrected_image_loss_7t(H, orc):
    """7T-shaped pair (130x130x85, 1.05 mm, PE axis 0): loss = mean((1/2 (T+ + T-) - I_true)^2)
    at the OT initial field, gradients through CorrectedImages with respect to both images and b,
    against the oracle adjoint and against central differences on 64 random voxels / nodes."""
    from paper_2403_10706_b300 import autograd as ag
    pr = ph.make_pair("7t")
    dims, p = pr.dims, pr.pe_dim
    h = H(dims, pr.spacing, p, ALPHA, BETA)
    Ip = dev(pr.Ip).requires_grad_(True)
    Im = dev(pr.Im).requires_grad_(True)
    b0 = h.init_ot(Ip.detach(), Im.detach())
    b = b0.clone().requires_grad_(True)
    It = dev(pr.I_true)
    C = ag.corrected_image(h, Ip, Im, b)
    loss = ((C - It) ** 2).mean()
    loss.backward()
    gIp, gIm, gb = host(Ip.grad), host(Im.grad), host(b.grad)
    bh = host(b0)
    N = float(np.prod(dims))

    # oracle gradient: dL/dT+- = (C - I_true) / N
    P = orc.Problem(dims, pr.spacing, p, ALPHA, BETA)
    T = P.eval(pr.Ip, pr.Im, bh, contract=True, grad=False, corrected=True)
    gT = (0.5 * (T["Tp"] + T["Tm"]) - pr.I_true) / N
    rp, rm, rb = P.correct_adjoint(pr.Ip, pr.Im, bh, gT, gT, contract=True)
    check(gIp, rp, "dL/dIp")
    check(gIm, rm, "dL/dIm")
    check(gb, rb, "dL/db")

    # central differences on single columns (a voxel or node only moves its own column's T)
    m = dims[p]
    P1 = orc.Problem((1, m, 1), (1.0, 1.0, 1.0), 1, ALPHA, BETA)
    ncols = int(np.prod(dims)) // m

    def col_loss(ip, im, bb, It_c):
        T1 = P1.eval(ip.reshape(1, m, 1), im.reshape(1, m, 1), bb.reshape(1, m + 1, 1),
                     contract=False, grad=False, corrected=True, cells=True)
        Cc = 0.5 * (T1["Tp"] + T1["Tm"]).ravel()
        return np.sum((Cc - It_c) ** 2) / N, T1["cell_p"], T1["cell_m"]

    rng = np.random.default_rng(4242)
    hstep = 1e-3
    gscale = {"Ip": np.abs(gIp).max(), "Im": np.abs(gIm).max(), "b": np.abs(gb).max()}
    done = {"Ip": 0, "Im": 0, "b": 0}
    tries = 0
    while min(done.values()) < 64 and tries < 4000:
        tries += 1
        col = int(rng.integers(ncols))
        ipc = column(pr.Ip, col, p).astype(np.float32)
        imc = column(pr.Im, col, p).astype(np.float32)
        bc = column(bh, col, p).astype(np.float64)
        itc = column(pr.I_true, col, p).astype(np.float64)
        for which in ("Ip", "Im", "b"):
            if done[which] >= 64:
                continue
            if which == "b":
                k = int(rng.integers(m + 1))
                e = np.zeros(m + 1)
                e[k] = hstep
                Lp, cp1, cm1 = col_loss(ipc, imc, bc + e, itc)
                Lm, cp2, cm2 = col_loss(ipc, imc, bc - e, itc)
                if not (np.array_equal(cp1, cp2) and np.array_equal(cm1, cm2)):
                    continue   # the step crosses an interpolation kink
                fd = (Lp - Lm) / (2 * hstep)
                g = column(gb, col, p)[k]
            else:
                k = int(rng.integers(m))
                src = ipc if which == "Ip" else imc
                up, dn = src.copy(), src.copy()
                up[k] = np.float32(src[k] + hstep)
                dn[k] = np.float32(src[k] - hstep)
                hp, hm = float(up[k]) - float(src[k]), float(src[k]) - float(dn[k])
                args_up = (up, imc) if which == "Ip" else (ipc, up)
                args_dn = (dn, imc) if which == "Ip" else (ipc, dn)
                Lp = col_loss(*args_up, bc, itc)[0]
                Lm = col_loss(*args_dn, bc, itc)[0]
                fd = (Lp - Lm) / (hp + hm)
                g = column(gIp if which == "Ip" else gIm, col, p)[k]
            assert abs(fd - g) <= 1e-3 * abs(fd) + 1e-4 * gscale[which], (which, col, k, fd, g)
            done[which] += 1
    assert min(done.values()) >= 64, done


def test_autograd_objective_gradients(H, orc):
    """J through Objective: dJ/dIp, dJ/dIm against the oracle, dJ/db = the gradient of
    hysco_eval, dJ/dalpha = S and dJ/dbeta = P against central differences of the oracle's J in
    the weights (J is affine in them)."""
    from paper_2403_10706_b300 import autograd as ag
    dims, spacing, p = SHAPES[4]
    Ip, Im, b, _, _ = case(dims, p, 900)
    h = H(dims, spacing, p, ALPHA, BETA)
    tIp, tIm, tb = (dev(Ip).requires_grad_(True), dev(Im).requires_grad_(True),
                    dev(b).requires_grad_(True))
    a = torch.tensor(ALPHA, dtype=torch.float64, device="cuda", requires_grad=True)
    be = torch.tensor(BETA, dtype=torch.float64, device="cuda", requires_grad=True)
    J = ag.objective(h, tIp, tIm, tb, a, be)
    (3.0 * J).backward()
    P = orc.Problem(dims, spacing, p, ALPHA, BETA)
    e = P.eval(Ip, Im, b, contract=True)
    assert abs(J.item() - e["J"]) <= 1e-5 * abs(e["J"])
    rp, rm = P.image_grad(Ip, Im, b, contract=True)
    check(host(tIp.grad), 3.0 * rp, "dJ/dIp")
    check(host(tIm.grad), 3.0 * rm, "dJ/dIm")
    check(host(tb.grad), 3.0 * e["grad"], "dJ/db")
    for name, t, w in (("alpha", a, 0), ("beta", be, 1)):
        hw = 1e-3 * (ALPHA if w == 0 else BETA)
        wts = [ALPHA, BETA]
        wts[w] += hw
        Jp = orc.Problem(dims, spacing, p, *wts).eval(Ip, Im, b, contract=True, grad=False)["J"]
        wts[w] -= 2 * hw
        Jm = orc.Problem(dims, spacing, p, *wts).eval(Ip, Im, b, contract=True, grad=False)["J"]
        fd = 3.0 * (Jp - Jm) / (2 * hw)
        assert abs(t.grad.item() - fd) <= 1e-5 * abs(fd), (name, t.grad.item(), fd)
    with pytest.raises(ValueError):
        ag.objective(h, tIp, tIm, tb, torch.tensor(1.0, dtype=torch.float64, device="cuda"))


def test_autograd_bf16_images_return_bf16_gradients(H):
    from paper_2403_10706_b300 import autograd as ag
    dims, spacing, p = SHAPES[0]
    Ip, Im, b, _, _ = case(dims, p, 950)
    h = H(dims, spacing, p, ALPHA, BETA, dtype=torch.bfloat16)
    tIp = dev(Ip, torch.bfloat16).requires_grad_(True)
    tIm = dev(Im, torch.bfloat16).requires_grad_(True)
    C = ag.corrected_image(h, tIp, tIm, dev(b))
    C.square().sum().backward()
    assert tIp.grad.dtype == torch.bfloat16 and tIm.grad.dtype == torch.bfloat16
    assert torch.isfinite(tIp.grad.float()).all()


@pytest.mark.parametrize("dims,spacing,p", SHAPES)
@pytest.mark.parametrize("dt", ["f32", "bf16"])
def test_corrected_mean_and_its_adjoint(H, orc, dims, spacing, p, dt):
    """hysco_correct_mean against the oracle's 1/2 (T+ + T-) (1e-5 of the largest intensity), and
    its adjoint against hysco_correct_adjoint with both sensitivities gT / 2: halving is exact, so
    the two adjoints agree bit for bit."""
    Ip, Im, b, gT, _ = case(dims, p, 8100 + 7 * p)
    h = H(dims, spacing, p, ALPHA, BETA, dtype=DT[dt])
    tIp, tIm = dev(Ip, DT[dt]), dev(Im, DT[dt])
    T = host(h.correct_mean(tIp, tIm, dev(b)))
    P = orc.Problem(dims, spacing, p, ALPHA, BETA)
    ev = P.eval(host(tIp).astype(np.float32), host(tIm).astype(np.float32), b.astype(np.float64),
                contract=True, grad=False, corrected=True)
    ref = 0.5 * (ev["Tp"] + ev["Tm"])
    assert np.abs(T - ref).max() <= 1e-5 * np.abs(ref).max()
    tgT = dev(gT)
    a = h.correct_mean_adjoint(tIp, tIm, dev(b), tgT)
    half = (0.5 * tgT).contiguous()
    r = h.correct_adjoint(tIp, tIm, dev(b), half, half)
    for x, y in zip(a, r):
        assert torch.equal(x, y)
