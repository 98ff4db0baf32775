"""Pins of the oracle's least-squares correction (Sec. 2.4 "Image Correction"): the true image
minimising |P+ I - I+|^2 + |P- I - I-|^2 (+ a tiny lambda |I|^2), P+- the push-forward matrices of
the field, per PE column.  Checked against what fixes it independently of the oracle's code:
  - P+- against the phantom generator's push-forward (its own numpy implementation, cumulative
    mass interpolation), and mass conservation;
  - exact recovery of a known image from its noise-free pushed-forward pair;
  - on noisy data, numpy.linalg.lstsq of the stacked system (a textbook routine).
"""
import numpy as np
import pytest

from paper_2403_10706_b300 import phantom as ph

ALPHA, BETA = 300.0, 1e4


def smooth_column_field(m, seed, amp=2.0, slope=0.45):
    """A column field whose ends are 0 (no mass leaves the column) with |delta| <= slope."""
    rng = np.random.default_rng(seed)
    x = np.linspace(0.0, np.pi, m + 1)
    b = amp * np.sin(x) * (1.0 + 0.3 * np.sin(3 * x + rng.uniform(0, 6)))
    d = np.abs(np.diff(b)).max()
    return b * min(1.0, slope / d)


@pytest.mark.parametrize("sign", [1.0, -1.0])
@pytest.mark.parametrize("m", [5, 16, 40])
def test_pushforward_matrix_matches_the_phantom_generator(orc, m, sign):
    b = smooth_column_field(m, 10 + m)
    b[0] += 0.3 * sign      # some mass leaves at one end
    I = np.random.default_rng(m).uniform(0.1, 1.0, m)
    P = orc.pushforward_matrix(b, sign)
    ref = ph.push_forward(I.reshape(1, m, 1), b.reshape(1, m + 1, 1), 1, sign).ravel()
    assert np.allclose(P @ I, ref, rtol=0, atol=1e-12)


def test_pushforward_conserves_mass_inside_the_column(orc):
    m = 30
    b = smooth_column_field(m, 3)
    for sign in (1.0, -1.0):
        P = orc.pushforward_matrix(b, sign)
        assert np.allclose(P.sum(axis=0), 1.0, atol=1e-12)
        assert (P >= 0).all()


@pytest.mark.parametrize("dims,p", [((3, 24, 4), 1), ((20, 2, 3), 0), ((2, 3, 18), 2)])
def test_noise_free_pair_is_corrected_exactly(orc, dims, p):
    m = dims[p]
    rng = np.random.default_rng(7)
    I = rng.uniform(0.2, 1.0, dims)
    fd = ph.field_dims(dims, p)
    b = np.moveaxis(np.zeros(fd), p, -1)
    for idx in np.ndindex(*b.shape[:-1]):
        b[idx] = smooth_column_field(m, 100 + sum(idx), amp=rng.uniform(0.5, 3.0))
    b = np.ascontiguousarray(np.moveaxis(b, -1, p))
    Ip = ph.push_forward(I, b, p, +1.0).astype(np.float32)
    Im = ph.push_forward(I, b, p, -1.0).astype(np.float32)
    P = orc.Problem(dims, (1.0, 1.0, 1.0), p, ALPHA, BETA)
    out, bad = P.ls_correct(Ip, Im, b, lam=1e-12)
    assert bad == 0
    assert np.abs(out - I).max() <= 1e-5 * np.abs(I).max()


def test_noisy_pair_matches_lstsq(orc):
    dims, p = (2, 20, 3), 1
    m = dims[p]
    rng = np.random.default_rng(11)
    Ip = rng.uniform(0.2, 1.0, dims).astype(np.float32)
    Im = rng.uniform(0.2, 1.0, dims).astype(np.float32)
    b = ph.random_field(dims, p, 12, scale=2.0, smooth=1.0, max_slope=0.5).astype(np.float64)
    lam = 1e-3
    P = orc.Problem(dims, (1.0, 1.0, 1.0), p, ALPHA, BETA)
    out, bad = P.ls_correct(Ip, Im, b, lam=lam)
    assert bad == 0
    for c0 in range(dims[0]):
        for c2 in range(dims[2]):
            bc = b[c0, :, c2]
            A = np.vstack([orc.pushforward_matrix(bc, 1.0), orc.pushforward_matrix(bc, -1.0),
                           np.sqrt(lam) * np.eye(m)])
            y = np.concatenate([Ip[c0, :, c2], Im[c0, :, c2], np.zeros(m)]).astype(np.float64)
            ref = np.linalg.lstsq(A, y, rcond=None)[0]
            assert np.allclose(out[c0, :, c2], ref, rtol=0, atol=1e-10)


def test_infeasible_column_is_skipped(orc):
    dims, p = (1, 6, 2), 1
    b = np.zeros(ph.field_dims(dims, p))
    b[0, 3, 0] = 1.5            # |delta| >= 1 in column 0 only
    Ip = np.ones(dims, np.float32)
    P = orc.Problem(dims, (1.0, 1.0, 1.0), p, ALPHA, BETA)
    out, bad = P.ls_correct(Ip, Ip, b)
    assert bad == 1 and not out[0, :, 0].any() and np.allclose(out[0, :, 1], 1.0, atol=1e-6)
