"""Implicit differentiation through the solve on the GPU (hysco_implicit_parts,
hysco_solve_adjoint, autograd.SolvedField) against the double-precision oracle.

Tolerances: the parts for a given v are sums of a few single-precision products per entry
(relative 1e-5 in the 2-norm, 2e-4 of the largest per entry, as for the gradient); the two weight
sums cancel (v has both signs), so their error is bounded by 1e-5 of the sum of the terms'
magnitudes.  Where v comes from each side's own PCG (single precision to relative
residual 1e-6 on the GPU, double to 1e-12 in the oracle), v and everything after it agree to
relative 1e-3.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2403_10706_b300 import phantom as ph  # noqa: E402

ALPHA, BETA = 300.0, 1e4
SHAPES = [((7, 13, 5), (1.0, 1.25, 0.9), 1), ((9, 6, 11), (1.1, 1.0, 1.2), 0),
          ((5, 4, 17), (0.9, 1.3, 1.0), 2), ((40, 3, 37), (1.0, 1.5, 1.0), 1)]


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
    return t.detach().double().cpu().numpy()


def rel(a, b):
    return np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300)


def check(got, ref, what, rtol=1e-5, etol=2e-4):
    err2 = rel(got, ref)
    errinf = np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-30)
    assert err2 <= rtol and errinf <= etol, (what, err2, errinf)


@pytest.mark.parametrize("dims,spacing,p", SHAPES)
def test_implicit_parts_match_oracle(H, orc, dims, spacing, p):
    Ip, Im = ph.random_images(dims, 1200, 0.1, 1.0)
    b = ph.random_field(dims, p, 1201, scale=2.0, smooth=1.0, max_slope=0.6)
    v = np.random.default_rng(1202).normal(size=b.shape).astype(np.float32)
    h = H(dims, spacing, p, ALPHA, BETA)
    dIp, dIm, dth = h.implicit_parts(dev(Ip), dev(Im), dev(b), dev(v))
    P = orc.Problem(dims, spacing, p, ALPHA, BETA)
    rp, rm = P.mixed_image_adjoint(Ip, Im, b, v, contract=True)
    sa, sb = P.theta_dots(Ip, Im, b, v, contract=True)
    check(host(dIp), -rp, "dIp")
    check(host(dIm), -rm, "dIm")
    # the weight sums cancel (v has both signs): bound their error by the sum of |terms|, the
    # per-node terms v dg/dtheta taken exactly from the oracle (g is affine in alpha and beta)
    t = host(dth)
    for w, s_ref in ((0, sa), (1, sb)):
        wts = [ALPHA, BETA]
        wts[w] += 1.0
        gp = orc.Problem(dims, spacing, p, *wts).eval(Ip, Im, b, contract=True)["grad"]
        wts[w] -= 2.0
        gm = orc.Problem(dims, spacing, p, *wts).eval(Ip, Im, b, contract=True)["grad"]
        scale = np.sum(np.abs(v * (gp - gm) / 2.0))
        assert abs(t[w] + s_ref) <= 1e-5 * scale, (w, t[w], s_ref, scale)


def test_solve_adjoint_at_a_solution_matches_oracle(H, orc):
    pr = ph.make_pair("tiny")
    h = H(pr.dims, pr.spacing, pr.pe_dim, ALPHA, BETA)
    Ip, Im = dev(pr.Ip), dev(pr.Im)
    b, _ = h.solve(Ip, Im, gn_iters=10)
    dLdb = np.random.default_rng(1300).normal(size=h.field_dims).astype(np.float32)
    v, dIp, dIm, dth = h.solve_adjoint(Ip, Im, b, dev(dLdb), max_iters=1000, rtol=1e-6)
    P = orc.Problem(pr.dims, pr.spacing, pr.pe_dim, ALPHA, BETA)
    rv, rp, rm, ra, rb, it = P.solve_adjoint(pr.Ip, pr.Im, host(b), dLdb, max_it=2000, rtol=1e-12)
    assert rel(host(v), rv) <= 1e-3
    assert rel(host(dIp), rp) <= 1e-3 and rel(host(dIm), rm) <= 1e-3
    t = host(dth)
    assert abs(t[0] - ra) <= 1e-3 * abs(ra) and abs(t[1] - rb) <= 1e-3 * abs(rb), (t, ra, rb)


def test_solved_field_autograd_matches_oracle_composition(H, orc):
    """L = mean((1/2 (T+ + T-)(b*) - I_true)^2) with b* = SolvedField(Ip, Im, alpha): dL/dI+-
    (direct through the corrected image + implicit through b*) and dL/dalpha (implicit only)."""
    from paper_2403_10706_b300 import autograd as ag
    pr = ph.make_pair("tiny")
    h = H(pr.dims, pr.spacing, pr.pe_dim, ALPHA, BETA)
    Ip = dev(pr.Ip).requires_grad_(True)
    Im = dev(pr.Im).requires_grad_(True)
    a = torch.tensor(ALPHA, dtype=torch.float64, device="cuda", requires_grad=True)
    b = ag.solved_field(h, Ip, Im, alpha=a, gn_iters=10, adjoint_iters=1000, adjoint_rtol=1e-6)
    C = ag.corrected_image(h, Ip, Im, b)
    It = dev(pr.I_true)
    loss = ((C - It) ** 2).mean()
    loss.backward()
    bh = host(b)
    P = orc.Problem(pr.dims, pr.spacing, pr.pe_dim, ALPHA, BETA)
    T = P.eval(pr.Ip, pr.Im, bh, contract=True, grad=False, corrected=True)
    gT = (0.5 * (T["Tp"] + T["Tm"]) - pr.I_true) / pr.I_true.size
    dp, dm, db = P.correct_adjoint(pr.Ip, pr.Im, bh, gT, gT, contract=True)
    _, ip_, im_, da, _, _ = P.solve_adjoint(pr.Ip, pr.Im, bh, db, max_it=2000, rtol=1e-12)
    assert rel(host(Ip.grad), dp + ip_) <= 1e-3
    assert rel(host(Im.grad), dm + im_) <= 1e-3
    assert abs(a.grad.item() - da) <= 1e-3 * abs(da), (a.grad.item(), da)
