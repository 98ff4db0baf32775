"""ADMM (Sec. 2.3.2, hysco_admm) against the double-precision oracle's ADMM on the same inputs.

Every decision of a run is compared first: the rho sequence (the residual-balancing rule) and
the stopping iteration must be identical, and the BlockPCG iteration counts (summed over
columns) may differ only where a column's relative residual sits at the 0.1 threshold (within
1%).  Values: J and the b-subproblem's objective at every iterate relative 1e-4 and the final
field relative 1e-3 in the 2-norm
(single-precision arithmetic through the same iterations, as for the GN solve); the residuals
r, s and the relative changes, whose single-precision values are differences of nearby fields,
relative 1e-2.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2403_10706_b300 import _lib  # noqa: E402
from paper_2403_10706_b300 import phantom as ph  # noqa: E402

ALPHA, BETA = 300.0, 1e4


@pytest.fixture(scope="module")
def H():
    from paper_2403_10706_b300 import build
    build.build()
    from paper_2403_10706_b300.hysco import Hysco
    return Hysco


def rel(a, b):
    return np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300)


def run_both(H, orc, pr, iters, gn_iters=2, **kw):
    h = H(pr.dims, pr.spacing, pr.pe_dim, ALPHA, BETA)
    b, st = h.admm(torch.from_numpy(pr.Ip).cuda(), torch.from_numpy(pr.Im).cuda(),
                   admm_iters=iters, gn_iters=gn_iters, **kw)
    torch.cuda.synchronize()
    assert h.last_status() == 0
    P = orc.Problem(pr.dims, pr.spacing, pr.pe_dim, ALPHA, BETA)
    okw = {k: v for k, v in kw.items() if k in ("tol", "mu", "tau", "rho0")}
    rb, rz, ru, status, rst = P.admm(pr.Ip, pr.Im, admm_iters=iters, gn_iters=gn_iters,
                                     contract=True, **okw)
    assert status == 0
    return b.cpu().numpy(), st.cpu().numpy(), rb, rst, orc.ADMM_FIELDS


def check(gs, rs, fields, gb, rb, what):
    F = {f: i for i, f in enumerate(fields)}
    done_g = ~np.isnan(gs[:, F["J"]])
    done_r = ~np.isnan(rs[:, F["J"]])
    assert np.array_equal(done_g, done_r), (what, done_g, done_r)
    gs, rs = gs[done_g], rs[done_r]
    assert np.array_equal(gs[:, F["rho"]], rs[:, F["rho"]]), (what, gs[:, F["rho"]], rs[:, F["rho"]])
    np.testing.assert_allclose(gs[:, F["J"]], rs[:, F["J"]], rtol=1e-4, err_msg=what)
    np.testing.assert_allclose(gs[:, F["F_c"]], rs[:, F["F_c"]], rtol=1e-4, err_msg=what)
    np.testing.assert_allclose(gs[:, F["block_pcg_iters"]], rs[:, F["block_pcg_iters"]],
                               rtol=1e-2, err_msg=what)
    for f in ("r_primal", "s_dual", "rel_db", "rel_dz"):
        np.testing.assert_allclose(gs[:, F[f]], rs[:, F[f]], rtol=1e-2, err_msg=f"{what} {f}")
    assert rel(gb, rb) <= 1e-3, (what, rel(gb, rb))


def test_one_iteration_matches_oracle(H, orc):
    pr = ph.make_pair("tiny")
    gb, gs, rb, rs, fields = run_both(H, orc, pr, 1, gn_iters=1)
    check(gs, rs, fields, gb, rb, "tiny, 1 iteration")


def test_tiny_run_matches_oracle(H, orc):
    pr = ph.make_pair("tiny")
    gb, gs, rb, rs, fields = run_both(H, orc, pr, 10)
    check(gs, rs, fields, gb, rb, "tiny, 10 iterations")


@pytest.mark.parametrize("name", ["small", "7t"])
def test_larger_volumes_match_oracle(H, orc, name):
    """96x96x60 (PE axis 1) and 130x130x85 (PE axis 0), 4 iterations."""
    pr = ph.make_pair(name)
    gb, gs, rb, rs, fields = run_both(H, orc, pr, 4)
    check(gs, rs, fields, gb, rb, name)


def test_pe_axis_2_and_ragged_planes(H, orc):
    recipe = dict(dims=(21, 19, 40), spacing=(1.1, 0.9, 1.0), pe_dim=2, seed=7001, n_ellipsoids=3,
                  n_blobs=2, semi_axes=(3.0, 8.0), smooth=0.5, n_gauss=3, sigma=(4.0, 6.0),
                  bmax=2.5, noise=0.01)
    pr = ph.make_pair(recipe)
    gb, gs, rb, rs, fields = run_both(H, orc, pr, 5)
    check(gs, rs, fields, gb, rb, "pe 2")


def test_stop_rule_matches_oracle(H, orc):
    pr = ph.make_pair("tiny")
    gb, gs, rb, rs, fields = run_both(H, orc, pr, 30, tol=0.05)
    assert np.isnan(gs[-1, 0])   # stopped before the cap
    check(gs, rs, fields, gb, rb, "tol 0.05")


def test_graph_replay_equals_direct_launches(H):
    pr = ph.make_pair("tiny")
    h = H(pr.dims, pr.spacing, pr.pe_dim, ALPHA, BETA)
    Ip, Im = torch.from_numpy(pr.Ip).cuda(), torch.from_numpy(pr.Im).cuda()
    outs = []
    b = h._new_fld()
    for no_graph in (1, 0, 0):
        b, st = h.admm(Ip, Im, b=b, init=1, admm_iters=6, no_graph=no_graph)
        torch.cuda.synchronize()
        outs.append((b.cpu().numpy().copy(), st.cpu().numpy().copy()))
    for k in (1, 2):
        assert np.array_equal(outs[0][0], outs[k][0])
        assert np.array_equal(outs[0][1], outs[k][1], equal_nan=True)


def test_rejects_long_columns_and_bad_options(H):
    h = H((4, 300, 3), (1.0, 1.0, 1.0), 1, ALPHA, BETA)   # 301 PE nodes > 256
    Ip = torch.zeros((4, 300, 3), device="cuda")
    with pytest.raises(_lib.HyscoError):
        h.admm(Ip, Ip, admm_iters=1)
    h2 = H((8, 8, 8), (1.0, 1.0, 1.0), 1, ALPHA, BETA)
    I2 = torch.zeros((8, 8, 8), device="cuda")
    for bad in (dict(tau=1.0), dict(mu=0.5), dict(gn_iters=0), dict(pcg_max_iters=65),
                dict(tol=-1.0)):
        with pytest.raises(_lib.HyscoError):
            h2.admm(I2, I2, admm_iters=1, **bad)


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
def test_half_precision_images_match_oracle_on_the_same_values(H, orc, dtype):
    """Images stored in bf16 / f16 (the prox evaluation kernels are templated on the storage
    type): against the oracle's ADMM on the same quantised values."""
    td = {"bf16": torch.bfloat16, "f16": torch.float16}[dtype]
    pr = ph.make_pair("tiny")
    Ipq = torch.from_numpy(pr.Ip).cuda().to(td)
    Imq = torch.from_numpy(pr.Im).cuda().to(td)
    h = H(pr.dims, pr.spacing, pr.pe_dim, ALPHA, BETA, dtype=td)
    b, st = h.admm(Ipq, Imq, admm_iters=6)
    torch.cuda.synchronize()
    assert h.last_status() == 0
    P = orc.Problem(pr.dims, pr.spacing, pr.pe_dim, ALPHA, BETA)
    rb, rz, ru, status, rst = P.admm(Ipq.float().cpu().numpy(), Imq.float().cpu().numpy(),
                                     admm_iters=6, contract=True)
    check(st.cpu().numpy(), rst, orc.ADMM_FIELDS, b.cpu().numpy(), rb, dtype)


def test_start_from_a_given_field(H, orc):
    """init = 0: the run starts from the caller's b (here the oracle's 3-iteration GN field)."""
    pr = ph.make_pair("tiny")
    P = orc.Problem(pr.dims, pr.spacing, pr.pe_dim, ALPHA, BETA)
    b0, status, _ = P.solve(pr.Ip, pr.Im, gn_iters=3)
    assert status == 0
    h = H(pr.dims, pr.spacing, pr.pe_dim, ALPHA, BETA)
    b = torch.from_numpy(b0.astype(np.float32)).cuda()
    b, st = h.admm(torch.from_numpy(pr.Ip).cuda(), torch.from_numpy(pr.Im).cuda(), b=b, init=0,
                   admm_iters=5, rho0=50.0)
    torch.cuda.synchronize()
    assert h.last_status() == 0
    rb, rz, ru, status, rst = P.admm(pr.Ip, pr.Im, b=b0.astype(np.float32).astype(np.float64),
                                     init=False, admm_iters=5, rho0=50.0, contract=True)
    assert status == 0
    assert st.cpu().numpy()[0, 2] == 50.0
    check(st.cpu().numpy(), rst, orc.ADMM_FIELDS, b.cpu().numpy(), rb, "init 0, rho0 50")


@pytest.mark.parametrize("name,p", [("tiny", None), ("pe0", 0), ("pe2", 2)])
def test_block_pcg_matches_oracle(H, orc, name, p):
    """BlockPCG alone (hysco_block_pcg) against the oracle's per-column CG on the same
    linearisation: q relative 1e-4 (single-precision CG through <= 10 iterations per column, as
    for the global PCG step), iterations summed over columns within 1% (a column whose relative
    residual sits at 0.1 may stop one iteration apart)."""
    if p is None:
        pr = ph.make_pair("tiny")
        dims, spacing, pe, Ip, Im = pr.dims, pr.spacing, pr.pe_dim, pr.Ip, pr.Im
    else:
        dims, spacing, pe = ((9, 6, 11), (1.1, 1.0, 1.2), 0) if p == 0 else \
            ((5, 4, 17), (0.9, 1.3, 1.0), 2)
        Ip, Im = ph.random_images(dims, 801, 0.1, 1.0)
    b = ph.random_field(dims, pe, 802, scale=1.2, smooth=1.0)
    P = orc.Problem(dims, spacing, pe, ALPHA, BETA)
    rng = np.random.default_rng(803)
    rhs = rng.standard_normal(P.fdims).astype(np.float32)
    rho = 40.0
    h = H(dims, spacing, pe, ALPHA, BETA)
    q, it = h.block_pcg(torch.from_numpy(Ip).cuda(), torch.from_numpy(Im).cuda(),
                        torch.from_numpy(b).cuda(), rho, torch.from_numpy(rhs).cuda())
    torch.cuda.synchronize()
    qref, itref = P.block_pcg(Ip, Im, b.astype(np.float64), rho, rhs.astype(np.float64))
    assert rel(q.cpu().numpy(), qref) <= 1e-4, rel(q.cpu().numpy(), qref)
    assert abs(int(it.item()) - itref) <= 0.01 * itref, (int(it.item()), itref)


@pytest.mark.parametrize("path", [0, 1])
@pytest.mark.parametrize("dims,spacing,p", [((32, 32, 16), (1.0, 1.0, 1.0), 1),
                                            ((9, 6, 11), (1.1, 1.0, 1.2), 0),
                                            ((5, 4, 17), (0.9, 1.3, 1.0), 2),
                                            ((1, 7, 6), (1.0, 1.0, 1.0), 1),
                                            ((40, 33, 150), (1.0, 1.2, 0.9), 0)])
def test_z_update_matches_the_oracles_fft(H, orc, dims, spacing, p, path):
    """The z-update alone (hysco_admm_zsolve, real Fourier bases) against the oracle's numpy 2D
    FFT inversion, on the tensor cores (path 0: TF32 split pairs, three products each, FP32
    accumulation) and on the CUDA cores (path 1, FP32): relative 2e-5 (single precision through
    four transforms; the tensor-core products drop only the lo x lo term, below 2^-21 relative).
    The shapes cover ragged tiles (rows and contraction lengths not multiples of the tile), a
    one-node in-plane axis, the PE axis innermost (the other row order of the last product) and
    in-plane axes of 150 and 40 nodes."""
    P = orc.Problem(dims, spacing, p, ALPHA, BETA)
    rng = np.random.default_rng(901)
    v = rng.standard_normal(P.fdims).astype(np.float32)
    rho = 7.5
    h = H(dims, spacing, p, ALPHA, BETA)
    h.set_zsolve_path(path)
    assert h.zsolve_path() == path
    z = h.admm_zsolve(torch.from_numpy(v).cuda(), rho)
    torch.cuda.synchronize()
    zref = P.admm_z_solve(rho * v.astype(np.float64), rho)
    assert rel(z.cpu().numpy(), zref) <= 2e-5, rel(z.cpu().numpy(), zref)


@pytest.mark.parametrize("rho", [0.5, 40.0])
def test_z_update_full_3t_size_on_the_tensor_cores(H, orc, rho):
    """The 3T plane size (144 x 111 in-plane, 169 PE planes) on the tensor-core path, the default
    there, against the oracle's FFT inversion, and the two paths against each other."""
    dims, spacing, p = (144, 168, 111), (1.25, 1.25, 1.25), 1
    P = orc.Problem(dims, spacing, p, ALPHA, BETA)
    rng = np.random.default_rng(902)
    v = rng.standard_normal(P.fdims).astype(np.float32)
    h = H(dims, spacing, p, ALPHA, BETA)
    assert h.zsolve_path() == 0
    vd = torch.from_numpy(v).cuda()
    z0 = h.admm_zsolve(vd, rho).cpu().numpy()
    h.set_zsolve_path(1)
    z1 = h.admm_zsolve(vd, rho).cpu().numpy()
    zref = P.admm_z_solve(rho * v.astype(np.float64), rho)
    assert rel(z0, zref) <= 2e-5, rel(z0, zref)
    assert rel(z1, zref) <= 2e-5, rel(z1, zref)
    assert h.last_status() == 0


def test_z_update_7t_plane_size_and_the_cuda_core_fallback(H, orc):
    """The 7T plane (200 x 132 in-plane, PE axis 0: a 208-column tile, five 16-column stages) on
    the tensor cores against the oracle; an in-plane axis of 300 nodes (past the MMA's largest N)
    runs on the CUDA cores, where path 0 is refused."""
    dims, spacing, p = (132, 200, 200), (1.2, 1.0, 1.0), 0
    P = orc.Problem(dims, spacing, p, ALPHA, BETA)
    v = np.random.default_rng(903).standard_normal(P.fdims).astype(np.float32)
    h = H(dims, spacing, p, ALPHA, BETA)
    assert h.zsolve_path() == 0
    z = h.admm_zsolve(torch.from_numpy(v).cuda(), 12.0).cpu().numpy()
    zref = P.admm_z_solve(12.0 * v.astype(np.float64), 12.0)
    assert rel(z, zref) <= 2e-5, rel(z, zref)
    dims2 = (300, 6, 5)
    P2 = orc.Problem(dims2, (1.0, 1.0, 1.0), 1, ALPHA, BETA)
    v2 = np.random.default_rng(904).standard_normal(P2.fdims).astype(np.float32)
    h2 = H(dims2, (1.0, 1.0, 1.0), 1, ALPHA, BETA)
    assert h2.zsolve_path() == 1
    with pytest.raises(_lib.HyscoError):
        h2.set_zsolve_path(0)
    z2 = h2.admm_zsolve(torch.from_numpy(v2).cuda(), 3.0).cpu().numpy()
    zref2 = P2.admm_z_solve(3.0 * v2.astype(np.float64), 3.0)
    assert rel(z2, zref2) <= 2e-5, rel(z2, zref2)


def test_z_update_path_switch_rejects_unknown_paths_and_rebuilds_the_graph(H):
    """Path 2 and -1 are rejected; switching paths between two graph-captured ADMM runs gives
    results that agree to single precision (the cached graph is rebuilt, not replayed)."""
    pr = ph.make_pair("tiny")
    h = H(pr.dims, pr.spacing, pr.pe_dim, ALPHA, BETA)
    for bad in (-1, 2):
        with pytest.raises(_lib.HyscoError):
            h.set_zsolve_path(bad)
    Ip, Im = torch.from_numpy(pr.Ip).cuda(), torch.from_numpy(pr.Im).cuda()
    outs = []
    for path in (0, 1, 0):
        h.set_zsolve_path(path)
        b, _ = h.admm(Ip, Im, init=1, admm_iters=4)
        torch.cuda.synchronize()
        outs.append(b.cpu().numpy().copy())
    assert np.array_equal(outs[0], outs[2])
    assert rel(outs[1], outs[0]) <= 1e-4
    assert not np.array_equal(outs[1], outs[0])
