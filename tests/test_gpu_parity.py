"""Parity of the CUDA path (through the C ABI) with the double-precision oracle.

Tolerances (derived from single-precision arithmetic, unit roundoff u = 6e-8):
  - cell indices and OT merge indices: bit-exact (both sides take those decisions in the same
    single-precision operations);
  - J, D, S, P: relative 1e-5 (sums of non-negative single-precision terms);
  - gradient, Hessian-vector product, preconditioner: relative 1e-5 in the 2-norm, and every
    element within 2e-4 of the largest magnitude (a handful of roundings of terms that cancel);
  - corrected images: 1e-5 of the largest intensity;
  - OT field: 2e-4 voxel before / after blur (single-precision spline inversion, the CDF
    decisions being identical);
  - final field after the full GN solve: relative 1e-3 in the 2-norm.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2403_10706_b300 import phantom as ph  # noqa: E402

ALPHA, BETA = 300.0, 1e4
SHAPES = [  # (dims, spacing, pe): ragged sizes, every PE axis, single columns
    ((7, 13, 5), (1.0, 1.25, 0.9), 1),
    ((9, 6, 11), (1.1, 1.0, 1.2), 0),
    ((5, 4, 17), (0.9, 1.3, 1.0), 2),
    ((1, 33, 1), (1.0, 1.0, 1.0), 1),
    ((40, 3, 37), (1.0, 1.5, 1.0), 1),
    ((2, 2, 2), (1.0, 1.0, 1.0), 0),
    ((4, 2, 5), (1.0, 1.2, 0.9), 1),    # the shortest PE extent the handle accepts (m = 2)
    ((3, 4, 2), (1.1, 1.0, 0.8), 2),    # PE innermost, m = 2: three nodes in a 4-wide pitch
]


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
    return t.detach().cpu().numpy()


def rel(a, b):
    return np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300)


def case(dims, p, seed, bscale=2.0):
    Ip, Im = ph.random_images(dims, seed, 0.1, 1.0)
    b = ph.random_field(dims, p, seed + 1, scale=bscale, smooth=1.0)
    return Ip, Im, b


def check_field(got, ref, what, rtol=1e-5, etol=2e-4):
    r = rel(got, ref)
    e = np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300)
    assert r <= rtol and e <= etol, f"{what}: rel {r:.3e}, max elem {e:.3e}"


# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("dims,spacing,p", SHAPES)
def test_cell_indices_bit_exact(H, orc, dims, spacing, p):
    Ip, Im, b = case(dims, p, 100)
    b = (np.random.default_rng(1).uniform(-4, 4, size=b.shape)).astype(np.float32)
    h = H(dims, spacing, p, ALPHA, BETA)
    cp, cm = h.cell_indices(dev(b))
    P = orc.Problem(dims, spacing, p, ALPHA, BETA)
    e = P.eval(Ip, Im, b, contract=True, grad=False, cells=True)
    m = dims[p]
    assert np.array_equal(host(cp), np.clip(e["cell_p"], -2, m + 1))
    assert np.array_equal(host(cm), np.clip(e["cell_m"], -2, m + 1))


@pytest.mark.parametrize("dims,spacing,p", SHAPES)
def test_eval_matches_oracle(H, orc, dims, spacing, p):
    Ip, Im, b = case(dims, p, 200)
    h = H(dims, spacing, p, ALPHA, BETA)
    terms, g = h.eval(dev(Ip), dev(Im), dev(b))
    P = orc.Problem(dims, spacing, p, ALPHA, BETA)
    e = P.eval(Ip, Im, b, contract=True)
    t = host(terms)
    for i, k in enumerate("JDSP"):
        assert abs(t[i] - e[k]) <= 1e-5 * abs(e[k]) + 1e-12, (k, t[i], e[k])
    assert h.last_status() == 0
    check_field(host(g), e["grad"], "grad")


@pytest.mark.parametrize("dims,spacing,p", SHAPES)
def test_hessvec_and_preconditioners_match_oracle(H, orc, dims, spacing, p):
    Ip, Im, b = case(dims, p, 300)
    v = np.random.default_rng(7).normal(size=b.shape).astype(np.float32)
    h = H(dims, spacing, p, ALPHA, BETA)
    h.eval(dev(Ip), dev(Im), dev(b))
    P = orc.Problem(dims, spacing, p, ALPHA, BETA)
    check_field(host(h.hessvec(dev(v))), P.hessvec(Ip, Im, b, v), "Hv")
    check_field(host(h.precond(dev(v), 0)), P.precond(Ip, Im, b, v, 0), "jacobi")
    # column blocks: FP32 Thomas is backward stable; its forward error grows with the block's
    # condition number (a lone column has only the weak data term against the constant null
    # space of alpha * L), so the check is on the residual of the oracle's blocks
    # (backward error  max|M z - r| / max(|M| |z| + |r|), M = the oracle's blocks)
    zc = host(h.precond(dev(v), 1)).astype(np.float64)
    dia, off = P.column_blocks(Ip, Im, b)
    Mz, Maz = dia * zc, np.abs(dia * zc)
    lo = [slice(None)] * 3; hi = [slice(None)] * 3
    lo[p] = slice(0, -1); hi[p] = slice(1, None)
    lo, hi = tuple(lo), tuple(hi)
    Mz[lo] += off[lo] * zc[hi]; Maz[lo] += np.abs(off[lo] * zc[hi])
    Mz[hi] += off[lo] * zc[lo]; Maz[hi] += np.abs(off[lo] * zc[lo])
    eta = np.abs(Mz - v).max() / (Maz + np.abs(v)).max()
    assert eta <= 1e-5, eta
    if dims[0] * dims[1] * dims[2] // dims[p] > 1:
        check_field(zc, P.precond(Ip, Im, b, v, 1), "column", 1e-4, 1e-3)


@pytest.mark.parametrize("dims,spacing,p", SHAPES)
def test_corrected_images_match_oracle(H, orc, dims, spacing, p):
    Ip, Im, b = case(dims, p, 400)
    h = H(dims, spacing, p, ALPHA, BETA)
    Tp, Tm = h.correct(dev(Ip), dev(Im), dev(b))
    P = orc.Problem(dims, spacing, p, ALPHA, BETA)
    e = P.eval(Ip, Im, b, contract=True, grad=False, corrected=True)
    assert np.abs(host(Tp) - e["Tp"]).max() <= 1e-5 * np.abs(e["Tp"]).max()
    assert np.abs(host(Tm) - e["Tm"]).max() <= 1e-5 * np.abs(e["Tm"]).max()


@pytest.mark.parametrize("dims,spacing,p", SHAPES[:5] + SHAPES[6:])
@pytest.mark.parametrize("blur", [False, True])
def test_ot_init_matches_oracle(H, orc, dims, spacing, p, blur):
    pr_I = ph.random_images(dims, 500, -0.05, 1.0)
    Ip, Im = pr_I
    h = H(dims, spacing, p, ALPHA, BETA)
    b0 = host(h.init_ot(dev(Ip), dev(Im), blur=blur, eps=1e-3))
    kp, km = h.ot_indices(dev(Ip), dev(Im), eps=1e-3)
    P = orc.Problem(dims, spacing, p, ALPHA, BETA)
    ref, rkp, rkm = P.ot_init(Ip, Im, 1e-3, contract=True, blur=blur, indices=True)
    assert np.array_equal(host(kp), rkp)
    assert np.array_equal(host(km), rkm)
    assert np.abs(b0 - ref).max() <= 2e-4


def test_infeasible_and_nonfinite_status(H, orc):
    dims, p = (6, 10, 5), 1
    Ip, Im, b = case(dims, p, 600)
    h = H(dims, (1.0, 1.0, 1.0), p, ALPHA, BETA)
    bad = b.copy()
    bad[2, 4, 3] += 1.5     # one PE difference beyond the barrier
    terms, _ = h.eval(dev(Ip), dev(Im), dev(bad))
    assert h.last_status() == 1
    assert np.isinf(host(terms)[0])
    Ipn = Ip.copy()
    Ipn[1, 1, 1] = np.nan
    h.eval(dev(Ipn), dev(Im), dev(b))
    assert h.last_status() == -4


@pytest.mark.parametrize("dtype", ["bfloat16", "float16"])
def test_half_precision_images_match_oracle_on_the_same_values(H, orc, dtype):
    dims, spacing, p = (9, 14, 7), (1.0, 1.25, 1.0), 1
    Ip, Im, b = case(dims, p, 700)
    td = getattr(torch, dtype)
    Ipq, Imq = dev(Ip, td), dev(Im, td)
    h = H(dims, spacing, p, ALPHA, BETA, dtype=td)
    terms, g = h.eval(Ipq, Imq, dev(b))
    P = orc.Problem(dims, spacing, p, ALPHA, BETA)
    e = P.eval(host(Ipq.float()), host(Imq.float()), b, contract=True)
    assert abs(host(terms)[0] - e["J"]) <= 1e-5 * abs(e["J"])
    check_field(host(g), e["grad"], "grad " + dtype)


@pytest.mark.parametrize("precond,path", [(0, 1), (0, 2), (0, 3), (0, 4), (1, 0)])
def test_tiny_solve_matches_oracle(H, orc, precond, path):
    """Tiny case: 32x32x16, OT init, 10 GN-PCG iterations (path 1: separate PCG kernels,
    path 2: the persistent cooperative PCG kernel, path 3: its one-barrier form, path 4: the
    whole GN loop in one persistent kernel)."""
    pr = ph.make_pair("tiny")
    h = H(pr.dims, pr.spacing, pr.pe_dim, ALPHA, BETA)
    b, st = h.solve(dev(pr.Ip), dev(pr.Im), gn_iters=10, precond=precond, pcg_path=path)
    assert h.last_status() == 0
    P = orc.Problem(pr.dims, pr.spacing, pr.pe_dim, ALPHA, BETA)
    ref, status, rst = P.solve(pr.Ip, pr.Im, gn_iters=10, precond=precond, contract=False)
    gs = host(st)
    assert status == 0
    assert np.array_equal(gs[:, 6], rst[:, 6]), (gs[:, 6], rst[:, 6])        # accepted steps
    assert np.array_equal(gs[:, 7], rst[:, 7]), (gs[:, 7], rst[:, 7])        # PCG iterations
    assert np.allclose(gs[:, 0], rst[:, 0], rtol=1e-4)
    assert rel(host(b), ref) <= 1e-3


@pytest.mark.parametrize("name", ["small", "7t"])
def test_both_pcg_paths_match_oracle_on_larger_volumes(H, orc, name):
    """Small (96x96x60, PE axis 1) and 7T-shaped (130x130x85, PE axis 0) pairs, OT init + 4 GN
    iterations, through the separate PCG kernels, both persistent PCG kernels and the persistent
    GN loop, against the oracle's own double-precision trajectory."""
    pr = ph.make_pair(name)
    P = orc.Problem(pr.dims, pr.spacing, pr.pe_dim, ALPHA, BETA)
    ref, status, rst = P.solve(pr.Ip, pr.Im, gn_iters=4, contract=False)
    assert status == 0
    h = H(pr.dims, pr.spacing, pr.pe_dim, ALPHA, BETA)
    for path in (1, 2, 3, 4):
        b, st = h.solve(dev(pr.Ip), dev(pr.Im), gn_iters=4, pcg_path=path)
        assert h.last_status() == 0
        gs = host(st)
        assert np.allclose(gs[:, 0], rst[:, 0], rtol=1e-4), (path, gs[:, 0], rst[:, 0])
        assert rel(host(b), ref) <= 1e-3, (path, rel(host(b), ref), gs[:, 6], rst[:, 6])


@pytest.mark.parametrize("precond,path", [(0, 1), (0, 2), (0, 3), (1, 0)])
@pytest.mark.parametrize("dims,spacing,p", [SHAPES[0], SHAPES[1], SHAPES[2], SHAPES[4]])
def test_pcg_step_matches_oracle(H, orc, precond, path, dims, spacing, p):
    """hysco_pcg: q ~= H^{-1} rhs with <= 10 PCG iterations, against the oracle's PCG on the same
    linearisation (the two differ only by single-precision rounding through 10 iterations)."""
    Ip, Im, b = case(dims, p, 900)
    h = H(dims, spacing, p, ALPHA, BETA)
    terms, g = h.eval(dev(Ip), dev(Im), dev(b))
    rhs = -host(g).astype(np.float32)
    q = host(h.pcg(dev(rhs), precond=precond, max_iters=10, rtol=0.1, pcg_path=path))
    P = orc.Problem(dims, spacing, p, ALPHA, BETA)
    qref, it, relres = P.pcg(Ip, Im, b, rhs.astype(np.float64), precond=precond, max_it=10,
                             rtol=0.1)
    assert rel(q, qref) <= 1e-4, (rel(q, qref), it, relres)


def test_graph_replay_equals_direct_launches(H):
    """The CUDA graph of a solve replays exactly the kernels a direct solve launches, and the
    kernels are deterministic: the fields and statistics are bit-identical, also on a second
    replay of the cached graph."""
    pr = ph.make_pair("small")
    h = H(pr.dims, pr.spacing, pr.pe_dim, ALPHA, BETA)
    Ip, Im = dev(pr.Ip), dev(pr.Im)
    out = []
    for graph in (False, True, True):
        b = torch.empty(h.field_dims, dtype=torch.float32, device="cuda")
        st = torch.empty((5, 10), dtype=torch.float64, device="cuda")
        if out:   # same buffers for the two graph calls, so the second one replays the cache
            b, st = out[-1][2], out[-1][3]
        h.solve(Ip, Im, b=b, gn_iters=5, init=True, graph=graph)
        assert h.last_status() == 0
        bb, ss = h.solve(Ip, Im, b=b, gn_iters=5, init=True, graph=graph)
        out.append((host(bb).copy(), host(ss).copy(), b, st))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[1][0], out[2][0])
    assert np.array_equal(out[0][1], out[1][1], equal_nan=True)


INFEASIBLE = [dict(n_ellipsoids=4, n_blobs=3, semi_axes=(3.0, 9.0), smooth=0.5, n_gauss=4,
                   sigma=(4.0, 7.0), spacing=(1.0, 1.0, 1.0), bmax=7.0, dims=(24, 40, 20),
                   pe_dim=1, seed=6043, noise=0.03),
              dict(n_ellipsoids=4, n_blobs=3, semi_axes=(3.0, 9.0), smooth=0.5, n_gauss=4,
                   sigma=(4.0, 7.0), spacing=(1.0, 1.0, 1.0), bmax=7.0, dims=(40, 20, 24),
                   pe_dim=0, seed=6036, noise=0.05)]


@pytest.mark.parametrize("recipe", INFEASIBLE)
def test_infeasible_ot_start_is_halved_like_the_oracle(H, orc, recipe):
    """Blurred OT fields with max |delta| ~ 1.2 and 1.1: the solve starts from the OT field halved
    until feasible (exact power-of-two factor, the oracle's), then follows the oracle."""
    pr = ph.make_pair(recipe)
    h = H(pr.dims, pr.spacing, pr.pe_dim, ALPHA, BETA)
    Ip, Im = dev(pr.Ip), dev(pr.Im)
    b0 = host(h.init_ot(Ip, Im))
    start, _ = h.solve(Ip, Im, gn_iters=0)
    P = orc.Problem(pr.dims, pr.spacing, pr.pe_dim, ALPHA, BETA)
    _, f = P.feasible_start(P.ot_init(pr.Ip, pr.Im, contract=True))
    assert f < 1.0
    assert np.array_equal(host(start), (f * b0).astype(np.float32))
    b, st = h.solve(Ip, Im, gn_iters=5)
    assert h.last_status() == 0
    ref, status, rst = P.solve(pr.Ip, pr.Im, gn_iters=5, contract=False)
    assert status == 0
    gs = host(st)
    assert np.allclose(gs[:, 0], rst[:, 0], rtol=1e-4), (gs[:, 0], rst[:, 0])
    assert rel(host(b), ref) <= 1e-3


def test_persistent_gn_loop_matches_the_separate_kernels(H):
    """pcg_path 4 (the whole GN loop in one persistent launch) against pcg_path 2 (the same PCG
    kernel body, every other step its own kernel) on the small pair: the same accepted steps and
    PCG iteration counts, objective histories within 1e-6 and fields within 1e-5 (only the
    grouping of J's partial sums differs); a second call, and a graph replay, bit-identical."""
    pr = ph.make_pair("small")
    h = H(pr.dims, pr.spacing, pr.pe_dim, ALPHA, BETA)
    Ip, Im = dev(pr.Ip), dev(pr.Im)
    b2, s2 = h.solve(Ip, Im, gn_iters=8, pcg_path=2)
    b2, s2 = host(b2).copy(), host(s2).copy()
    runs = []
    for graph in (False, True, True):
        b4, s4 = h.solve(Ip, Im, gn_iters=8, pcg_path=4, graph=graph)
        assert h.last_status() == 0
        runs.append((host(b4).copy(), host(s4).copy()))
    b4, s4 = runs[0]
    assert np.array_equal(s4[:, 6], s2[:, 6]) and np.array_equal(s4[:, 7], s2[:, 7])
    assert np.array_equal(s4[:, 9], s2[:, 9])
    assert np.allclose(s4[:, 0], s2[:, 0], rtol=1e-6)
    assert rel(b4, b2) <= 1e-5
    for bb, ss in runs[1:]:
        assert np.array_equal(bb, b4) and np.array_equal(ss, s4, equal_nan=True)


def test_persistent_gn_loop_stops_on_a_non_finite_objective_like_the_separate_kernels(H):
    """A NaN image voxel makes J NaN at the first evaluation: both forms stop there with status
    -4, keep the objective row and fill every statistic after it with NaN, and leave b as the
    start."""
    dims, spacing, p = (24, 40, 20), (1.0, 1.0, 1.0), 1
    Ip, Im, b = case(dims, p, 710)
    Ipn = Ip.copy()
    Ipn[3, 5, 7] = np.nan
    h = H(dims, spacing, p, ALPHA, BETA)
    out = {}
    for path in (2, 4):
        bb, st = h.solve(dev(Ipn), dev(Im), b=dev(b), gn_iters=3, init=False, pcg_path=path)
        out[path] = (host(bb).copy(), host(st).copy(), h.last_status())
    for path in (2, 4):
        bb, st, status = out[path]
        assert status == -4, path
        assert np.array_equal(bb, b), path
        assert np.isnan(st[0, 0]) and np.all(np.isnan(st[0, 4:])) and np.all(np.isnan(st[1:])), path


@pytest.mark.parametrize("dtype", ["bfloat16", "float16"])
@pytest.mark.parametrize("dims,spacing,p", [SHAPES[0], SHAPES[1], SHAPES[2]])
def test_persistent_gn_loop_half_precision_images_every_pe_axis(H, orc, dtype, dims, spacing, p):
    """pcg_path 4 with bf16 / f16 image storage on each PE axis: the same accepted steps, PCG and
    line-search counts as pcg_path 2 on the same quantised images, and both within the solve
    tolerance of the FP64 oracle run on those quantised values."""
    Ip, Im, b0 = case(dims, p, 720)
    td = getattr(torch, dtype)
    Ipq, Imq = dev(Ip, td), dev(Im, td)
    h = H(dims, spacing, p, ALPHA, BETA, dtype=td)
    runs = {}
    for path in (2, 4):
        bb, st = h.solve(Ipq, Imq, b=dev(b0), gn_iters=5, init=False, pcg_path=path)
        assert h.last_status() == 0, path
        runs[path] = (host(bb).copy(), host(st).copy())
    (b2, s2), (b4, s4) = runs[2], runs[4]
    assert np.array_equal(s4[:, 6], s2[:, 6]) and np.array_equal(s4[:, 7], s2[:, 7])
    assert np.array_equal(s4[:, 9], s2[:, 9])
    assert rel(b4, b2) <= 1e-5
    P = orc.Problem(dims, spacing, p, ALPHA, BETA)
    ref, status, rst = P.solve(host(Ipq.float()), host(Imq.float()), b=b0.astype(np.float64),
                               gn_iters=5, init=False, contract=False)
    assert status == 0
    assert np.array_equal(s4[:, 6], rst[:, 6])
    assert rel(b4, ref) <= 1e-3
