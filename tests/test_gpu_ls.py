"""Least-squares correction (hysco_ls_correct) against the double-precision oracle.

Tolerances: the GPU assembles the normal equations and factors them (banded LDL^T) in single
precision, the oracle in double with a dense Cholesky.  On fields whose column ends stay in place
(no mass leaves: the normal matrix is well conditioned) the corrected images agree to 1e-5 of the
largest intensity; where mass leaves the column the weakly determined end cells amplify rounding,
and the comparison is relative 1e-3 in the 2-norm.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2403_10706_b300 import phantom as ph  # noqa: E402

ALPHA, BETA = 300.0, 1e4
SHAPES = [((7, 13, 5), (1.0, 1.25, 0.9), 1), ((9, 6, 11), (1.1, 1.0, 1.2), 0),
          ((5, 4, 17), (0.9, 1.3, 1.0), 2), ((40, 3, 37), (1.0, 1.5, 1.0), 1)]
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
    return t.detach().double().cpu().numpy()


def pinned_field(dims, p, seed, amp=2.0, slope=0.45):
    """Column fields that vanish at both ends (no mass leaves) with |delta| <= slope."""
    rng = np.random.default_rng(seed)
    m = dims[p]
    fd = ph.field_dims(dims, p)
    b = np.moveaxis(np.zeros(fd), p, -1)
    x = np.linspace(0.0, np.pi, m + 1)
    for idx in np.ndindex(*b.shape[:-1]):
        col = rng.uniform(0.3, 1.0) * amp * np.sin(x) * (1 + 0.3 * np.sin(3 * x + rng.uniform(0, 6)))
        b[idx] = col * min(1.0, slope / np.abs(np.diff(col)).max())
    return np.ascontiguousarray(np.moveaxis(b, -1, p)).astype(np.float32)


@pytest.mark.parametrize("dtype", list(DT))
@pytest.mark.parametrize("dims,spacing,p", SHAPES)
def test_ls_correct_matches_oracle(H, orc, dims, spacing, p, dtype):
    Ip, Im = ph.random_images(dims, 1400, 0.1, 1.0)
    b = pinned_field(dims, p, 1401)
    td = DT[dtype]
    Ipq, Imq = dev(Ip, td), dev(Im, td)
    h = H(dims, spacing, p, ALPHA, BETA, dtype=td)
    out, nbad = h.ls_correct(Ipq, Imq, dev(b), lam=1e-6)
    assert int(nbad.item()) == 0
    P = orc.Problem(dims, spacing, p, ALPHA, BETA)
    ref, bad = P.ls_correct(host(Ipq), host(Imq), b, lam=1e-6)
    assert bad == 0
    err = np.abs(host(out) - ref).max() / np.abs(ref).max()
    assert err <= 1e-5, err


@pytest.mark.parametrize("dims,spacing,p", SHAPES)
def test_ls_correct_with_mass_leaving_the_columns(H, orc, dims, spacing, p):
    Ip, Im = ph.random_images(dims, 1500, 0.1, 1.0)
    b = ph.random_field(dims, p, 1501, scale=2.0, smooth=1.0, max_slope=0.5)
    h = H(dims, spacing, p, ALPHA, BETA)
    out, nbad = h.ls_correct(dev(Ip), dev(Im), dev(b), lam=1e-6)
    P = orc.Problem(dims, spacing, p, ALPHA, BETA)
    ref, bad = P.ls_correct(Ip, Im, b, lam=1e-6)
    assert int(nbad.item()) == bad == 0
    rel = np.linalg.norm(host(out) - ref) / np.linalg.norm(ref)
    assert rel <= 1e-3, rel


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_ls_correct_strongly_compressed_columns(H, orc, dtype):
    """Fields with |delta| up to 0.9 (compression in both directions: a true cell's mapped interval
    shrinks to 0.1 voxel, so true cells up to ten apart share a distorted cell and the normal
    matrix needs a band of half-width about 10): no column is skipped, and the correction matches
    the oracle's dense solve."""
    dims, spacing, p = (3, 40, 4), (1.0, 1.25, 1.0), 1
    Ip, Im = ph.random_images(dims, 1700, 0.1, 1.0)
    m = dims[p]
    x = np.linspace(0.0, np.pi, m + 1)
    b = np.zeros(ph.field_dims(dims, p), np.float32)
    rng = np.random.default_rng(1701)
    for i0 in range(dims[0]):
        for i2 in range(dims[2]):
            col = np.sin(x) * (1.0 + 0.2 * np.sin(2 * x + rng.uniform(0, 6)))
            col *= 0.9 / np.abs(np.diff(col)).max() * rng.choice([-1.0, 1.0])
            b[i0, :, i2] = col.astype(np.float32)
    assert np.abs(np.diff(b, axis=p)).max() >= 0.89
    td = DT[dtype]
    Ipq, Imq = dev(Ip, td), dev(Im, td)
    h = H(dims, spacing, p, ALPHA, BETA, dtype=td)
    out, nbad = h.ls_correct(Ipq, Imq, dev(b), lam=1e-6)
    assert int(nbad.item()) == 0
    P = orc.Problem(dims, spacing, p, ALPHA, BETA)
    ref, bad = P.ls_correct(host(Ipq), host(Imq), b, lam=1e-6)
    assert bad == 0
    rel = np.linalg.norm(host(out) - ref) / np.linalg.norm(ref)
    assert rel <= 1e-3, rel


def test_ls_correct_skips_infeasible_and_too_steep_columns(H, orc):
    dims, spacing, p = (2, 12, 3), (1.0, 1.0, 1.0), 1
    Ip, Im = ph.random_images(dims, 1600, 0.1, 1.0)
    b = pinned_field(dims, p, 1601)
    b[0, 5, 0] = b[0, 4, 0] + 1.2     # |delta| >= 1 in column (0, 0)
    h = H(dims, spacing, p, ALPHA, BETA)
    out, nbad = h.ls_correct(dev(Ip), dev(Im), dev(b))
    assert int(nbad.item()) == 1
    o = host(out)
    assert not o[0, :, 0].any() and np.abs(o[1]).max() > 0


def test_ls_correct_recovers_the_phantom(H):
    """The tiny phantom at its true field: the correction is close to the true image (the
    residual is the phantom's noise, N(0, 0.01), propagated)."""
    pr = ph.make_pair("tiny")
    h = H(pr.dims, pr.spacing, pr.pe_dim, ALPHA, BETA)
    out, nbad = h.ls_correct(dev(pr.Ip), dev(pr.Im), dev(pr.b_true))
    assert int(nbad.item()) == 0
    err = host(out) - pr.I_true
    assert np.sqrt(np.mean(err ** 2)) <= 0.02
