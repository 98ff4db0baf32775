"""Pins of the double-precision oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed forms (J = 0 at an
exactly explained pair), finite differences, high-precision numerical differentiation, a library
routine (numpy.linalg.solve, scipy's Gaussian filter), Krylov-space optimality of CG, and exact
shift recovery of the 1D optimal-transport map.  No GPU is used.
"""
import numpy as np
import pytest

from paper_2403_10706_b300 import phantom as ph

ALPHA, BETA = 300.0, 1e4


def problem(orc, dims=(5, 9, 4), spacing=(1.0, 1.25, 0.8), p=1, alpha=ALPHA, beta=BETA):
    return orc.Problem(dims, spacing, p, alpha, beta)


def smooth_case(dims, p, seed, bscale=1.5):
    Ip, Im = ph.random_images(dims, seed, 0.2, 1.0)
    b = ph.random_field(dims, p, seed + 1, scale=bscale, smooth=1.0)
    return Ip, Im, b.astype(np.float64)


# --------------------------------------------------------------------------------------------
# reversing the phase-encoding direction (Eq. 1): the two acquisitions trade places
# --------------------------------------------------------------------------------------------

@pytest.mark.parametrize("p", [0, 1, 2])
def test_polarity_swap_symmetry(orc, p):
    """Swapping the two images and negating the field maps T+ to T- and back (Eq. 1): the
    residual changes sign, the smoothness and barrier terms are even in b, so J, D, S, P are
    unchanged, the gradient changes sign and the Gauss-Newton Hessian is unchanged.  A wrong sign
    of b or of the modulation in either image's term breaks this."""
    dims = (5, 9, 6)
    P = problem(orc, dims, (1.0, 1.25, 0.8), p)
    Ip, Im, b = smooth_case(dims, p, 40)
    v = np.random.default_rng(41).normal(size=b.shape)
    for contract in (True, False):
        e1 = P.eval(Ip, Im, b, contract=contract)
        e2 = P.eval(Im, Ip, -b, contract=contract)
        for k in "JDSP":
            assert abs(e2[k] - e1[k]) <= 1e-13 * abs(e1[k]), (k, contract)
        assert np.abs(e2["grad"] + e1["grad"]).max() <= 1e-13 * np.abs(e1["grad"]).max()
        h1 = P.hessvec(Ip, Im, b, v, contract=contract)
        h2 = P.hessvec(Im, Ip, -b, v, contract=contract)
        assert np.abs(h2 - h1).max() <= 1e-13 * np.abs(h1).max()
    # the whole GN solve from the OT start: the swapped pair's field is the negated field
    b1, s1, st1 = P.solve(Ip, Im, gn_iters=3)
    b2, s2, st2 = P.solve(Im, Ip, gn_iters=3)
    assert s1 == 0 and s2 == 0
    assert np.abs(b2 + b1).max() <= 1e-12 * np.abs(b1).max()
    assert np.allclose(st2[:, 0], st1[:, 0], rtol=1e-12)


# --------------------------------------------------------------------------------------------
# the barrier function (Eq. 3)
# --------------------------------------------------------------------------------------------

def test_phi_and_derivatives_match_mpmath(orc):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    f = lambda z: z ** 4 / (1 - z ** 2)
    for z in [-0.95, -0.7, -0.3, -1e-3, 0.0, 0.05, 0.5, 0.8, 0.99]:
        v, d1, d2 = orc.phi(z)
        zz = mp.mpf(z)
        assert abs(v - float(f(zz))) <= 1e-13 * max(1.0, abs(v))
        assert abs(d1 - float(mp.diff(f, zz, 1))) <= 1e-11 * max(1.0, abs(d1))
        assert abs(d2 - float(mp.diff(f, zz, 2))) <= 1e-10 * max(1.0, abs(d2))
        if z != 0.0:
            assert d2 > 0.0          # phi is strictly convex on (-1, 1) away from 0
    for z in [1.0, -1.0, 1.5, -3.0]:
        assert orc.phi(z)[0] == np.inf


# --------------------------------------------------------------------------------------------
# closed forms of the objective
# --------------------------------------------------------------------------------------------

@pytest.mark.parametrize("p", [0, 1, 2])
def test_zero_field_equal_images_gives_zero(orc, p):
    dims = (4, 6, 5)
    P = problem(orc, dims, (1.1, 0.9, 1.3), p)
    I = ph.random_images(dims, 3)[0]
    b = np.zeros(orc.field_dims(dims, p))
    for contract in (True, False):
        e = P.eval(I, I, b, contract=contract)
        assert e["J"] == 0.0 and e["D"] == 0.0 and e["S"] == 0.0 and e["P"] == 0.0
        assert np.all(e["grad"] == 0.0)


@pytest.mark.parametrize("p,s", [(0, 1), (1, 2), (2, 3), (1, -2)])
def test_exactly_shifted_pair_is_explained_by_constant_field(orc, p, s):
    """I+(y) = G(y - s), I-(y) = G(y + s) with integer s: the constant field b = s corrects both
    images back to G exactly (Eq. 1), so D = S = P = 0 and the gradient vanishes; the opposite
    sign does not.  Pins the sign of b in t+-, the cell-centre convention and L's null space."""
    dims = [4, 5, 6]
    dims[p] = 24
    dims = tuple(dims)
    m = dims[p]
    rng = np.random.default_rng(11)
    G = np.zeros(dims)
    sl = [slice(None)] * 3
    sl[p] = slice(abs(s) + 2, m - abs(s) - 2)
    G[tuple(sl)] = rng.uniform(0.2, 1.0, size=G[tuple(sl)].shape)
    Ip = np.roll(G, s, axis=p)     # Ip[j] = G[j - s]
    Im = np.roll(G, -s, axis=p)    # Im[j] = G[j + s]
    P = problem(orc, dims, (1.0, 1.2, 0.9), p)
    b = np.full(orc.field_dims(dims, p), float(s))
    e = P.eval(Ip, Im, b, contract=False)
    assert abs(e["J"]) < 1e-12 and np.abs(e["grad"]).max() < 1e-10
    bad = P.eval(Ip, Im, -b, contract=False)
    assert bad["D"] > 1e-3


def test_modulation_of_a_linear_field(orc):
    """b_k = kappa*k has delta = kappa in every cell.  Constant images 1/(1+kappa) and
    1/(1-kappa) are then both corrected to exactly 1 wherever t+- stay inside the image: pins the
    (1 +- delta) intensity modulation of Eq. 1."""
    m, kappa = 32, 0.1
    dims = (1, m, 1)
    P = problem(orc, dims, (1.0, 1.0, 1.0), 1, 0.0, 0.0)
    Ip = np.full(dims, 1.0 / (1.0 + kappa), np.float32)
    Im = np.full(dims, 1.0 / (1.0 - kappa), np.float32)
    b = (kappa * np.arange(m + 1, dtype=np.float64)).reshape(1, m + 1, 1)
    e = P.eval(Ip, Im, b, contract=False, corrected=True)
    j = np.arange(m)
    inside = (j * (1 + kappa) + kappa / 2 <= m - 1) & (j * (1 - kappa) - kappa / 2 >= 0)
    Tp, Tm = e["Tp"][0, :, 0], e["Tm"][0, :, 0]
    # the images are single precision: agreement to their rounding
    assert np.allclose(Tp[inside], 1.0, rtol=0, atol=1e-7)
    assert np.allclose(Tm[inside], 1.0, rtol=0, atol=1e-7)


def test_smoothness_null_space_symmetry_and_edge_form(orc):
    dims, p = (5, 7, 6), 2
    P = problem(orc, dims, (1.1, 0.7, 1.3), p)
    rng = np.random.default_rng(5)
    b = rng.normal(size=orc.field_dims(dims, p))
    I0 = np.zeros(dims, np.float32)
    S = P.eval(I0, I0, b, contract=False, grad=False)["S"]
    assert abs(P.eval(I0, I0, b + 3.7, contract=False, grad=False)["S"] - S) <= 1e-12 * S
    assert np.abs(P.laplacian(np.ones_like(b))).max() < 1e-12
    x, y = rng.normal(size=b.shape), rng.normal(size=b.shape)
    assert abs(x.ravel() @ P.laplacian(y).ravel() - y.ravel() @ P.laplacian(x).ravel()) < 1e-10
    # Eq. 5 as an integral of |grad b_mm|^2 over edges (b in PE voxels, b_mm = h_p b)
    h = (1.1, 0.7, 1.3)
    vol = h[0] * h[1] * h[2]
    edge = sum(((np.diff(b, axis=a) * h[p] / h[a]) ** 2).sum() for a in range(3))
    assert abs(0.5 * vol * edge - S) <= 1e-12 * S


# --------------------------------------------------------------------------------------------
# derivatives
# --------------------------------------------------------------------------------------------

@pytest.mark.parametrize("p", [0, 1, 2])
def test_gradient_matches_central_differences(orc, p):
    dims = (6, 7, 5)
    P = problem(orc, dims, (1.2, 1.0, 0.9), p)
    Ip, Im, b = smooth_case(dims, p, 20 + p)
    g = P.eval(Ip, Im, b, contract=False)["grad"]
    rng = np.random.default_rng(3)
    eps = 1e-6
    for _ in range(4):
        v = rng.normal(size=b.shape)
        Jp = P.eval(Ip, Im, b + eps * v, contract=False, grad=False)["J"]
        Jm = P.eval(Ip, Im, b - eps * v, contract=False, grad=False)["J"]
        fd = (Jp - Jm) / (2 * eps)
        assert abs(fd - g.ravel() @ v.ravel()) <= 1e-6 * abs(fd) + 1e-6
    # node-wise, away from interpolation kinks
    cells = P.eval(Ip, Im, b, contract=False, grad=False, cells=True)
    checked = 0
    for k in rng.choice(b.size, 40, replace=False):
        e = np.zeros(b.size); e[k] = 1e-5
        e = e.reshape(b.shape)
        up = P.eval(Ip, Im, b + e, contract=False, grad=False, cells=True)
        dn = P.eval(Ip, Im, b - e, contract=False, grad=False, cells=True)
        if any(np.any(x["cell_p"] != cells["cell_p"]) or np.any(x["cell_m"] != cells["cell_m"])
               for x in (up, dn)):
            continue
        fd = (up["J"] - dn["J"]) / 2e-5
        gk = g.ravel()[k]
        assert abs(fd - gk) <= 1e-5 * max(abs(gk), 1e-3 * np.abs(g).max())
        checked += 1
    assert checked >= 25


def _dense(P, fdims, fn):
    n = int(np.prod(fdims))
    H = np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n); e[k] = 1.0
        H[:, k] = fn(e.reshape(fdims)).ravel()
    return H


def test_gauss_newton_data_term_is_JtJ_of_fd_residual_jacobian(orc):
    """alpha = beta = 0: the GN Hessian is vol * Jr^T Jr; Jr from central differences of the
    corrected images' difference r(b) = T+ - T- (Eq. 1)."""
    dims, p = (3, 8, 2), 1
    P = problem(orc, dims, (1.0, 1.5, 0.8), p, 0.0, 0.0)
    Ip, Im, b = smooth_case(dims, p, 31, bscale=0.7)
    fd = orc.field_dims(dims, p)
    n = int(np.prod(fd))
    eps = 1e-7
    Jr = np.zeros((int(np.prod(dims)), n))
    for k in range(n):
        e = np.zeros(n); e[k] = eps
        up = P.eval(Ip, Im, b + e.reshape(fd), contract=False, grad=False, corrected=True)
        dn = P.eval(Ip, Im, b - e.reshape(fd), contract=False, grad=False, corrected=True)
        Jr[:, k] = (((up["Tp"] - up["Tm"]) - (dn["Tp"] - dn["Tm"])) / (2 * eps)).ravel()
    vol = 1.0 * 1.5 * 0.8
    H = _dense(P, fd, lambda v: P.hessvec(Ip, Im, b, v, contract=False))
    assert np.allclose(H, vol * Jr.T @ Jr, rtol=1e-6, atol=1e-6 * np.abs(H).max())


@pytest.mark.parametrize("alpha,beta", [(0.0, 2.0), (3.0, 0.0)])
def test_regulariser_hessians_match_fd_of_gradient(orc, alpha, beta):
    """With zero images only alpha*S + beta*P remains; both are exactly second-order in b
    (phi(D b) with D linear, and a quadratic), so the GN Hessian equals the true Hessian."""
    dims, p = (4, 6, 3), 1
    P = problem(orc, dims, (1.0, 1.3, 0.7), p, alpha, beta)
    I0 = np.zeros(dims, np.float32)
    b = ph.random_field(dims, p, 44, scale=1.2, smooth=1.0).astype(np.float64)
    rng = np.random.default_rng(9)
    eps = 1e-6
    for _ in range(3):
        v = rng.normal(size=b.shape)
        gp = P.eval(I0, I0, b + eps * v, contract=False)["grad"]
        gm = P.eval(I0, I0, b - eps * v, contract=False)["grad"]
        Hv = P.hessvec(I0, I0, b, v, contract=False)
        assert np.allclose(Hv, (gp - gm) / (2 * eps), rtol=1e-5,
                           atol=1e-6 * np.abs(Hv).max())


def test_hessian_symmetric_psd_diag_and_column_blocks(orc):
    dims, p = (3, 6, 4), 1
    P = problem(orc, dims, (1.0, 1.2, 0.9), p)
    Ip, Im, b = smooth_case(dims, p, 51, bscale=1.0)
    fd = orc.field_dims(dims, p)
    H = _dense(P, fd, lambda v: P.hessvec(Ip, Im, b, v))
    assert np.allclose(H, H.T, rtol=0, atol=1e-10 * np.abs(H).max())
    assert np.linalg.eigvalsh(H).min() > -1e-9 * np.abs(H).max()
    assert np.allclose(P.hessdiag(Ip, Im, b).ravel(), np.diag(H), rtol=1e-12)
    # per-column diagonal blocks (block-diagonal preconditioner) = H restricted to the column
    idx = np.arange(H.shape[0]).reshape(fd)
    cols = [idx[c0, :, c1] for c0 in range(dims[0]) for c1 in range(dims[2])]
    for col, nodes in enumerate(cols):
        dia, off = P.column_block(Ip, Im, b, col)
        Hc = H[np.ix_(nodes, nodes)]
        assert np.allclose(np.diag(Hc), dia, rtol=1e-12)
        assert np.allclose(np.diag(Hc, 1), off, rtol=1e-12, atol=1e-12 * np.abs(Hc).max())
        assert np.abs(np.triu(Hc, 2)).max() == 0.0


def test_preconditioners_are_exact_solves_of_their_matrices(orc):
    dims, p = (3, 7, 3), 1
    P = problem(orc, dims, (1.0, 1.2, 0.9), p)
    Ip, Im, b = smooth_case(dims, p, 61, bscale=1.0)
    fd = orc.field_dims(dims, p)
    H = _dense(P, fd, lambda v: P.hessvec(Ip, Im, b, v))
    r = np.random.default_rng(2).normal(size=fd)
    zj = P.precond(Ip, Im, b, r, 0)
    assert np.allclose(zj.ravel(), r.ravel() / np.diag(H), rtol=1e-12)
    zc = P.precond(Ip, Im, b, r, 1)
    idx = np.arange(H.shape[0]).reshape(fd)
    for c0 in range(dims[0]):
        for c1 in range(dims[2]):
            nodes = idx[c0, :, c1]
            ref = np.linalg.solve(H[np.ix_(nodes, nodes)], r.ravel()[nodes])
            assert np.allclose(zc.ravel()[nodes], ref, rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("precond", [0, 1])
def test_pcg_iterates_minimise_energy_over_krylov_space(orc, precond):
    """The i-th PCG iterate (x0 = 0) minimises the H-energy error over
    span{z0, (M^-1 H) z0, ...} (Hestenes & Stiefel); n iterations solve the system."""
    dims, p = (2, 6, 3), 1
    P = problem(orc, dims, (1.0, 1.2, 0.9), p)
    Ip, Im, b = smooth_case(dims, p, 71, bscale=1.0)
    fd = orc.field_dims(dims, p)
    n = int(np.prod(fd))
    H = _dense(P, fd, lambda v: P.hessvec(Ip, Im, b, v))
    Minv = _dense(P, fd, lambda v: P.precond(Ip, Im, b, v, precond))
    rhs = np.random.default_rng(4).normal(size=n)
    for it in (1, 2, 4, 7):
        q, used, _ = P.pcg(Ip, Im, b, rhs.reshape(fd), precond, max_it=it, rtol=0.0)
        assert used == it
        K = [Minv @ rhs]
        for _ in range(it - 1):
            K.append(Minv @ (H @ K[-1]))
        V, _ = np.linalg.qr(np.array(K).T)
        x = V @ np.linalg.solve(V.T @ H @ V, V.T @ rhs)
        assert np.allclose(q.ravel(), x, rtol=1e-6, atol=1e-8 * np.abs(x).max())
    q, used, rel = P.pcg(Ip, Im, b, rhs.reshape(fd), precond, max_it=4 * n, rtol=1e-12)
    assert np.allclose(q.ravel(), np.linalg.solve(H, rhs), rtol=1e-7, atol=1e-10)


# --------------------------------------------------------------------------------------------
# optimal-transport initialisation (Sec. 2.2)
# --------------------------------------------------------------------------------------------

def _gauss_columns(m, s, ncols=3, sigma=4.0):
    y = np.arange(m, dtype=np.float64)
    c = (m - 1) / 2.0
    G = lambda t: np.exp(-0.5 * ((t - c) / sigma) ** 2)
    Ip = np.stack([G(y - s)] * ncols)          # I+(y) = G(y - s)
    Im = np.stack([G(y + s)] * ncols)          # I-(y) = G(y + s)
    return Ip.reshape(ncols, 1, m).astype(np.float32), Im.reshape(ncols, 1, m).astype(np.float32)


@pytest.mark.parametrize("s", [1, 2, 3])
def test_ot_recovers_integer_shift_of_translated_gaussians(orc, s):
    m = 96   # long enough that both shifted Gaussians keep all of their mass
    Ip, Im = _gauss_columns(m, s)
    P = orc.Problem(Ip.shape, (1.0, 1.0, 1.0), 2, ALPHA, BETA)
    b0 = P.ot_init(Ip, Im, eps=0.0, contract=False, blur=False)
    C = np.concatenate([[0.0], np.cumsum(Ip[0, 0].astype(np.float64))])
    C /= C[-1]
    mask = (C >= 1e-6) & (C <= 1 - 1e-6)
    assert mask.sum() > 20
    assert np.abs(b0[:, 0, mask] - s).max() <= 1e-9


@pytest.mark.parametrize("s", [0.5, 1.3, 2.7])
def test_ot_recovers_fractional_shift_approximately(orc, s):
    m = 96
    Ip, Im = _gauss_columns(m, s)
    P = orc.Problem(Ip.shape, (1.0, 1.0, 1.0), 2, ALPHA, BETA)
    b0 = P.ot_init(Ip, Im, eps=0.0, contract=False, blur=False)
    C = np.concatenate([[0.0], np.cumsum(Ip[0, 0].astype(np.float64))])
    C /= C[-1]
    mask = (C >= 1e-3) & (C <= 1 - 1e-3)
    assert np.abs(b0[:, 0, mask] - s).max() <= 0.05


def test_ot_identity_and_antisymmetry(orc):
    dims, p = (5, 20, 4), 1
    Ip, Im = ph.random_images(dims, 8, 0.1, 1.0)
    P = problem(orc, dims, (1.0, 1.0, 1.0), p)
    for contract in (True, False):
        assert np.all(P.ot_init(Ip, Ip, 1e-3, contract, blur=False) == 0.0)
        a = P.ot_init(Ip, Im, 1e-3, contract, blur=False)
        b = P.ot_init(Im, Ip, 1e-3, contract, blur=False)
        assert np.array_equal(a, -b)


def test_ot_merge_index_is_the_spline_inverse_bracket(orc):
    """k* = min{k : C(k+1) >= r}: check against numpy.searchsorted on the same single-precision
    CDFs (formed in numpy float32, left to right)."""
    dims, p = (3, 17, 2), 1
    Ip, Im = ph.random_images(dims, 12, 0.0, 1.0)
    P = problem(orc, dims, (1.0, 1.0, 1.0), p)
    b0, kp, km = P.ot_init(Ip, Im, 1e-3, contract=True, blur=False, indices=True)
    allv = np.concatenate([Ip.ravel(), Im.ravel()])
    s = np.float32(max(np.float32(0), -allv.min())) + np.float32(1e-3) * np.abs(allv).max()
    for c0 in range(dims[0]):
        for c1 in range(dims[2]):
            cdf = []
            for I in (Ip, Im):
                acc = np.float32(0)
                c = [np.float32(0)]
                for v in I[c0, :, c1]:
                    acc = np.float32(acc + np.float32(v + s))
                    c.append(acc)
                c = np.array(c, np.float32)
                cdf.append(c / c[-1])
            Cp, Cm = cdf
            m = dims[p]
            for k in range(m + 1):
                for r, Cinv, got in ((Cp[k], Cm, kp[c0, k, c1]), (Cm[k], Cp, km[c0, k, c1])):
                    want = 0 if r <= 0 else min(int(np.searchsorted(Cinv[1:], r, "left")), m - 1)
                    assert got == want


def test_blur_is_the_truncated_gaussian_filter(orc):
    ndimage = pytest.importorskip("scipy.ndimage")
    dims, p = (6, 5, 7), 0
    P = problem(orc, dims, (1.0, 1.0, 1.0), p)
    b = np.random.default_rng(1).normal(size=orc.field_dims(dims, p))
    ref = ndimage.gaussian_filter(b, sigma=1.0, truncate=1.0, mode="nearest")
    assert np.allclose(P.blur(b), ref, rtol=0, atol=1e-13)


# --------------------------------------------------------------------------------------------
# contract mode and the full solve
# --------------------------------------------------------------------------------------------

def test_contract_mode_cell_index_is_single_precision_floor(orc):
    dims, p = (4, 12, 5), 1
    P = problem(orc, dims, (1.0, 1.0, 1.0), p)
    Ip, Im, _ = smooth_case(dims, p, 81)
    b = (np.random.default_rng(0).uniform(-3, 3, size=orc.field_dims(dims, p))
         .astype(np.float32))
    e = P.eval(Ip, Im, b.astype(np.float64), contract=True, grad=False, cells=True)
    bb = np.moveaxis(b, p, -1)
    bc = (bb[..., :-1] + bb[..., 1:]) * np.float32(0.5)
    j = np.arange(dims[p], dtype=np.float32)
    tp, tm = j + bc, j - bc
    assert tp.dtype == np.float32
    assert np.array_equal(np.moveaxis(e["cell_p"], p, -1), np.floor(tp).astype(np.int32))
    assert np.array_equal(np.moveaxis(e["cell_m"], p, -1), np.floor(tm).astype(np.int32))


def test_gn_solve_decreases_objective_and_explains_shifted_pair(orc):
    pr = ph.make_pair("tiny")
    P = orc.Problem(pr.dims, pr.spacing, pr.pe_dim, ALPHA, BETA)
    b, status, stats = P.solve(pr.Ip, pr.Im, gn_iters=6)
    assert status == 0
    J = stats[:, 0]
    assert np.all(np.diff(J) <= 0.0)
    gam = stats[:, 6]
    assert np.all(np.isin(gam, [0.0] + [2.0 ** -t for t in range(10)]))
    # final J matches a fresh evaluation at the returned field
    e = P.eval(pr.Ip, pr.Im, b, contract=False, grad=False)
    assert e["J"] <= J[-1]


def test_brute_force_8_voxel_column(orc):
    """One column of 8 cells (9 nodes): J by an independent 50-digit mpmath evaluation of
    Eq. 1-5 and the gradient by mpmath numerical differentiation of that evaluation."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    m = 8
    rng = np.random.default_rng(2024)
    Ip = rng.uniform(0.1, 1.0, m).astype(np.float32)
    Im = rng.uniform(0.1, 1.0, m).astype(np.float32)
    b = np.cumsum(np.r_[0.4, rng.uniform(-0.5, 0.5, m)])  # |delta| < 1
    h = (1.0, 1.7, 1.0)      # PE spacing 1.7 mm
    alpha, beta = 0.3, 0.02

    def J_mp(bv):
        vol = mp.mpf(h[0]) * mp.mpf(h[1]) * mp.mpf(h[2])
        def img(I, t):
            i = int(mp.floor(t)); w = t - i
            v0 = mp.mpf(float(I[i])) if 0 <= i < m else mp.mpf(0)
            v1 = mp.mpf(float(I[i + 1])) if 0 <= i + 1 < m else mp.mpf(0)
            return (1 - w) * v0 + w * v1
        D = mp.mpf(0); Pp = mp.mpf(0)
        for j in range(m):
            bc = (bv[j] + bv[j + 1]) / 2
            dl = bv[j + 1] - bv[j]
            r = img(Ip, j + bc) * (1 + dl) - img(Im, j - bc) * (1 - dl)
            D += r * r
            Pp += dl ** 4 / (1 - dl ** 2)
        # |grad b_mm|^2 along the single PE column: ((b_{k+1} - b_k) h / h) ^2
        S = sum((bv[k + 1] - bv[k]) ** 2 for k in range(m))
        return vol / 2 * D + alpha * vol / 2 * S + beta * vol / 2 * Pp

    P = orc.Problem((1, m, 1), h, 1, alpha, beta)
    e = P.eval(Ip.reshape(1, m, 1), Im.reshape(1, m, 1), b.reshape(1, m + 1, 1), contract=False)
    bm = [mp.mpf(float(x)) for x in b]
    Jref = J_mp(bm)
    assert abs(e["J"] - float(Jref)) <= 1e-13 * abs(float(Jref))
    for k in range(m + 1):
        def f(x, k=k):
            bb = list(bm); bb[k] = x
            return J_mp(bb)
        gk = float(mp.diff(f, bm[k]))
        assert abs(e["grad"].ravel()[k] - gk) <= 1e-11 * max(1.0, abs(gk))
