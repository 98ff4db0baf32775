"""Pins of the oracle's ADMM (Sec. 2.3.2) against what the mathematics fixes, no GPU.

  - the split: F(b) + G(b) = J(b) term by term (S3 + S1 + S2 = S, same D and P);
  - the gradient of the b-subproblem F_c = F + rho vol/2 ||b - c||^2 against central finite
    differences (pure double precision);
  - its per-column GN block against one assembled from a finite-difference residual Jacobian;
  - BlockPCG run to convergence against numpy.linalg.solve on every column's dense block, and the
    per-column stop (each column's own relative residual) against a column-by-column textbook CG;
  - the z-update against a dense solve with explicitly assembled periodic 2D Laplacians;
  - the driver: the rho rule of Boyd et al. (factors tau only when a residual exceeds mu times
    the other), the stop rule, and descent of J on the tiny workload.
"""
import numpy as np
import pytest

from paper_2403_10706_b300 import phantom as ph

ALPHA, BETA = 300.0, 1e4


def case(orc, dims=(5, 9, 4), spacing=(1.0, 1.25, 0.8), p=1, seed=11, bscale=1.5, rho=40.0):
    P = orc.Problem(dims, spacing, p, ALPHA, BETA)
    Ip, Im = ph.random_images(dims, seed, 0.2, 1.0)
    b = ph.random_field(dims, p, seed + 1, scale=bscale, smooth=1.0).astype(np.float64)
    c = ph.random_field(dims, p, seed + 2, scale=bscale, smooth=1.0).astype(np.float64)
    return P, Ip, Im, b, c, rho


def inplane_smoothness(P, b):
    """vol/2 h_p^2 sum over the in-plane axes a of sum (forward difference / h_a)^2"""
    vol = np.prod(P.spacing)
    hp = P.spacing[P.pe_dim]
    s = 0.0
    for a in P.inplane_axes():
        d = np.diff(b, axis=a)
        s += (hp / P.spacing[a]) ** 2 * np.sum(d * d)
    return 0.5 * vol * s


@pytest.mark.parametrize("p", [0, 1, 2])
def test_split_adds_up_to_the_objective(orc, p):
    P, Ip, Im, b, c, rho = case(orc, (6, 5, 7), (1.1, 0.9, 1.3), p, seed=21)
    e = P.eval(Ip, Im, b, contract=False, grad=False)
    f = P.admm_eval(Ip, Im, b, 0.0, c, contract=False, grad=False)
    assert f["D"] == pytest.approx(e["D"], rel=1e-14)
    assert f["P"] == pytest.approx(e["P"], rel=1e-14)
    assert f["S3"] + inplane_smoothness(P, b) == pytest.approx(e["S"], rel=1e-12)
    assert f["F_c"] == pytest.approx(f["D"] + ALPHA * f["S3"] + BETA * f["P"], rel=1e-14)
    g = P.admm_eval(Ip, Im, b, rho, c, contract=False, grad=False)
    vol = np.prod(P.spacing)
    assert g["prox"] == pytest.approx(0.5 * vol * np.sum((b - c) ** 2), rel=1e-13)
    assert g["F_c"] - f["F_c"] == pytest.approx(rho * g["prox"], rel=1e-12)


@pytest.mark.parametrize("p", [0, 1, 2])
def test_bsubproblem_gradient_matches_finite_differences(orc, p):
    P, Ip, Im, b, c, rho = case(orc, (4, 6, 5), (1.0, 1.2, 0.9), p, seed=31, bscale=0.8)
    g = P.admm_eval(Ip, Im, b, rho, c, contract=False)["grad"]
    rng = np.random.default_rng(5)
    h = 1e-6
    for _ in range(12):
        idx = tuple(rng.integers(0, n) for n in P.fdims)
        bp, bm = b.copy(), b.copy()
        bp[idx] += h
        bm[idx] -= h
        fp = P.admm_eval(Ip, Im, bp, rho, c, contract=False, grad=False)["F_c"]
        fm = P.admm_eval(Ip, Im, bm, rho, c, contract=False, grad=False)["F_c"]
        fd = (fp - fm) / (2 * h)
        assert abs(fd - g[idx]) <= 1e-6 * max(1.0, abs(g[idx])), (idx, fd, g[idx])


def test_column_block_from_finite_difference_jacobian(orc):
    """The per-column GN block assembled independently: the residual Jacobian by central finite
    differences of r = T+ - T- (the corrected images, pure double precision, at a field whose
    cell positions are away from the interpolation kinks), the barrier's second derivative from
    phi, and the PE difference operator written out:
      vol [Jr^T Jr + alpha D^T D + beta/2 D^T diag(phi''(D b)) D + rho I]."""
    dims, p = (3, 7, 4), 1
    P, Ip, Im, b, c, rho = case(orc, dims, (1.0, 1.3, 0.9), p, seed=41, bscale=0.7, rho=25.0)
    m = dims[p]
    vol = np.prod(P.spacing)
    h = 1e-6

    def resid(bb):
        e = P.eval(Ip, Im, bb, contract=False, grad=False, corrected=True)
        return e["Tp"] - e["Tm"]

    Dop = np.zeros((m, m + 1))
    for j in range(m):
        Dop[j, j], Dop[j, j + 1] = -1.0, 1.0
    cols = [(i0, i2) for i0 in range(dims[0]) for i2 in range(dims[2])]
    for col, (i0, i2) in enumerate(cols):
        Jr = np.zeros((m, m + 1))
        for k in range(m + 1):
            bp, bm = b.copy(), b.copy()
            bp[i0, k, i2] += h
            bm[i0, k, i2] -= h
            Jr[:, k] = (resid(bp)[i0, :, i2] - resid(bm)[i0, :, i2]) / (2 * h)
        delta = Dop @ b[i0, :, i2]
        d2 = np.array([orc.phi(x)[2] for x in delta])
        H = vol * (Jr.T @ Jr + ALPHA * Dop.T @ Dop + 0.5 * BETA * Dop.T @ np.diag(d2) @ Dop
                   + rho * np.eye(m + 1))
        dia, off = P.admm_column_block(Ip, Im, b, rho, col, contract=False)
        np.testing.assert_allclose(dia, np.diag(H), rtol=1e-6)
        np.testing.assert_allclose(off, np.diag(H, 1), rtol=1e-6, atol=1e-6 * np.abs(H).max())


@pytest.mark.parametrize("p", [0, 2])
def test_block_pcg_converges_to_each_columns_dense_solve(orc, p):
    dims = (4, 5, 6)
    P, Ip, Im, b, c, rho = case(orc, dims, (1.0, 1.1, 0.9), p, seed=51)
    rhs = -P.admm_eval(Ip, Im, b, rho, c)["grad"]
    m = dims[p]
    q, it = P.block_pcg(Ip, Im, b, rho, rhs, max_it=4 * (m + 1), rtol=1e-13)
    axes = [a for a in range(3) if a != p]
    for col in range(dims[axes[0]] * dims[axes[1]]):
        c0, c1 = divmod(col, dims[axes[1]])
        sl = [slice(None)] * 3
        sl[axes[0]], sl[axes[1]] = c0, c1
        dia, off = P.admm_column_block(Ip, Im, b, rho, col)
        H = np.diag(dia) + np.diag(off, 1) + np.diag(off, -1)
        np.testing.assert_allclose(q[tuple(sl)], np.linalg.solve(H, rhs[tuple(sl)]), rtol=1e-9,
                                   atol=1e-12)


def test_block_pcg_stops_each_column_on_its_own_residual(orc):
    """Textbook Jacobi CG per column with the column's own stop reproduces BlockPCG exactly."""
    dims, p = (3, 8, 3), 1
    P, Ip, Im, b, c, rho = case(orc, dims, (1.0, 1.0, 1.0), p, seed=61)
    rhs = -P.admm_eval(Ip, Im, b, rho, c)["grad"]
    q, it = P.block_pcg(Ip, Im, b, rho, rhs, max_it=10, rtol=0.1)
    total = 0
    for col in range(dims[0] * dims[2]):
        i0, i2 = divmod(col, dims[2])
        dia, off = P.admm_column_block(Ip, Im, b, rho, col)
        H = np.diag(dia) + np.diag(off, 1) + np.diag(off, -1)
        r = rhs[i0, :, i2].copy()
        x = np.zeros_like(r)
        rr0 = r @ r
        if rr0 > 0:
            z = r / dia
            pp, rz = z.copy(), r @ z
            for _ in range(10):
                Hp = H @ pp
                a = rz / (pp @ Hp)
                x += a * pp
                r -= a * Hp
                total += 1
                if np.sqrt(r @ r) / np.sqrt(rr0) < 0.1:
                    break
                z = r / dia
                rz_new = r @ z
                pp = z + rz_new / rz * pp
                rz = rz_new
        np.testing.assert_allclose(q[i0, :, i2], x, rtol=1e-12, atol=1e-15)
    assert it == total


def periodic_laplacian(n):
    L = 2.0 * np.eye(n)
    for i in range(n):
        L[i, (i + 1) % n] -= 1.0
        L[i, (i - 1) % n] -= 1.0
    return L


@pytest.mark.parametrize("p", [0, 1, 2])
def test_z_update_matches_dense_periodic_solve(orc, p):
    dims = (5, 6, 4)
    P = orc.Problem(dims, (1.2, 0.9, 1.1), p, ALPHA, BETA)
    rng = np.random.default_rng(71)
    rhs = rng.standard_normal(P.fdims)
    rho = 13.0
    z = P.admm_z_solve(rhs, rho)
    a0, a1 = P.inplane_axes()
    n0, n1 = P.fdims[a0], P.fdims[a1]
    hp = P.spacing[p]
    A = (rho * np.eye(n0 * n1)
         + ALPHA * (hp / P.spacing[a0]) ** 2 * np.kron(periodic_laplacian(n0), np.eye(n1))
         + ALPHA * (hp / P.spacing[a1]) ** 2 * np.kron(np.eye(n0), periodic_laplacian(n1)))
    for k in range(P.fdims[p]):
        plane = np.take(rhs, k, axis=p)          # (n0, n1), a0 slower than a1
        zk = np.linalg.solve(A, plane.ravel()).reshape(n0, n1)
        np.testing.assert_allclose(np.take(z, k, axis=p), zk, rtol=1e-11, atol=1e-12)


def test_admm_driver_rules_and_descent(orc):
    pr = ph.make_pair("tiny")
    P = orc.Problem(pr.dims, pr.spacing, pr.pe_dim, ALPHA, BETA)
    tau, mu = 2.0, 10.0
    b, z, u, status, st = P.admm(pr.Ip, pr.Im, admm_iters=12, gn_iters=2, tau=tau, mu=mu,
                                 tol=1e-12)
    assert status == 0
    F = {f: i for i, f in enumerate(orc.ADMM_FIELDS)}
    assert st[0, F["rho"]] == ALPHA                 # rho0 defaults to alpha
    for k in range(1, len(st)):
        r, s, rho_prev = st[k - 1, F["r_primal"]], st[k - 1, F["s_dual"]], st[k - 1, F["rho"]]
        want = rho_prev * tau if r > mu * s else (rho_prev / tau if s > mu * r else rho_prev)
        assert st[k, F["rho"]] == want
    assert st[-1, F["J"]] < 0.01 * st[0, F["J"]]   # descent on the tiny workload
    assert np.isinf(st[0, F["rel_du"]])             # u starts at 0
    # the stop rule: a loose tolerance ends the run after the first iteration below it
    b2, z2, u2, status2, st2 = P.admm(pr.Ip, pr.Im, admm_iters=40, gn_iters=2, tol=0.05)
    done = np.where(~np.isnan(st2[:, 0]))[0]
    last = done[-1]
    assert last < 39
    rel = st2[last, [F["rel_db"], F["rel_dz"], F["rel_du"]]]
    assert np.all(rel < 0.05)
    for k in done[:-1]:
        assert not np.all(st2[k, [F["rel_db"], F["rel_dz"], F["rel_du"]]] < 0.05)
