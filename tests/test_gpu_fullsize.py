"""Parity at the full 3T workload size the throughput benchmark solves (144x168x111 at 1.25 mm,
PE axis 1: 2.7 M field nodes), in the launch configuration it times (the persistent PCG on 148
blocks of 768 threads, every vector slot on chip), against the double-precision oracle on the
same seeded phantom.  Same tolerances as the small-size parity tests:
  - OT merge indices and interpolation cell indices: bit-exact;
  - J, D, S, P: relative 1e-5; gradient and H v: relative 1e-5 in the 2-norm, every element
    within 2e-4 of the largest magnitude; OT field: 2e-4 voxel;
  - one PCG solve of a GN step: relative 1e-4 (ten single-precision iterations);
  - two GN iterations from the OT start: the same accepted steps and PCG iteration counts,
    J within 1e-4, field relative 1e-3;
  - a property that holds at any size: reversing the phase-encoding direction (Eq. 1) negates
    the OT field exactly and the gradient and the 20-iteration solve within those tolerances.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

from paper_2403_10706_b300 import phantom as ph  # noqa: E402

ALPHA, BETA = 300.0, 1e4


@pytest.fixture(scope="module")
def H():
    from paper_2403_10706_b300 import build
    build.build()
    from paper_2403_10706_b300.hysco import Hysco
    return Hysco


@pytest.fixture(scope="module")
def pair():
    return ph.make_pair("3t")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def rel(a, b):
    return np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300)


def check_field(got, ref, what, rtol=1e-5, etol=2e-4):
    r = rel(got, ref)
    e = np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300)
    assert r <= rtol and e <= etol, f"{what}: rel {r:.3e}, max elem {e:.3e}"


def test_3t_launch_configuration(H, pair):
    h = H(pair.dims, pair.spacing, pair.pe_dim, ALPHA, BETA)
    grid, onchip, slots, block = h.pcg_plan()
    assert (onchip, slots, block) == (6, 6, 768), (grid, onchip, slots, block)
    assert grid == torch.cuda.get_device_properties(0).multi_processor_count


def test_3t_ot_cells_eval_hessvec_match_oracle(H, orc, pair):
    h = H(pair.dims, pair.spacing, pair.pe_dim, ALPHA, BETA)
    P = orc.Problem(pair.dims, pair.spacing, pair.pe_dim, ALPHA, BETA)
    Ip, Im = dev(pair.Ip), dev(pair.Im)
    # OT start: merge indices bit-exact, field within the spline-inversion bound
    b0 = host(h.init_ot(Ip, Im, blur=True, eps=1e-3))
    kp, km = h.ot_indices(Ip, Im, eps=1e-3)
    ref, rkp, rkm = P.ot_init(pair.Ip, pair.Im, 1e-3, contract=True, blur=True, indices=True)
    assert np.array_equal(host(kp), rkp)
    assert np.array_equal(host(km), rkm)
    assert np.abs(b0 - ref).max() <= 2e-4
    # J, its terms, the gradient and the cell indices at the GPU's OT field (same FP32 input)
    cp, cm = h.cell_indices(dev(b0))
    terms, g = h.eval(Ip, Im, dev(b0))
    e = P.eval(pair.Ip, pair.Im, b0, contract=True, cells=True)
    m = pair.dims[pair.pe_dim]
    assert np.array_equal(host(cp), np.clip(e["cell_p"], -2, m + 1))
    assert np.array_equal(host(cm), np.clip(e["cell_m"], -2, m + 1))
    t = host(terms)
    for i, k in enumerate("JDSP"):
        assert abs(t[i] - e[k]) <= 1e-5 * abs(e[k]) + 1e-12, (k, t[i], e[k])
    assert h.last_status() == 0
    check_field(host(g), e["grad"], "grad")
    # Gauss-Newton Hessian-vector product at that linearisation
    v = np.random.default_rng(11).normal(size=b0.shape).astype(np.float32)
    check_field(host(h.hessvec(dev(v))), P.hessvec(pair.Ip, pair.Im, b0, v), "Hv")


def test_3t_persistent_pcg_step_matches_oracle(H, orc, pair):
    h = H(pair.dims, pair.spacing, pair.pe_dim, ALPHA, BETA)
    Ip, Im = dev(pair.Ip), dev(pair.Im)
    b0 = host(h.init_ot(Ip, Im, blur=True, eps=1e-3))
    _, g = h.eval(Ip, Im, dev(b0))
    rhs = -host(g).astype(np.float32)
    q = host(h.pcg(dev(rhs), precond=0, max_iters=10, rtol=0.1, pcg_path=2))
    P = orc.Problem(pair.dims, pair.spacing, pair.pe_dim, ALPHA, BETA)
    qref, it, relres = P.pcg(pair.Ip, pair.Im, b0, rhs.astype(np.float64), precond=0,
                             max_it=10, rtol=0.1)
    assert rel(q, qref) <= 1e-4, (rel(q, qref), it, relres)


def test_3t_two_gn_iterations_match_oracle(H, orc, pair):
    h = H(pair.dims, pair.spacing, pair.pe_dim, ALPHA, BETA)
    b, st = h.solve(dev(pair.Ip), dev(pair.Im), gn_iters=2)
    assert h.last_status() == 0
    P = orc.Problem(pair.dims, pair.spacing, pair.pe_dim, ALPHA, BETA)
    ref, status, rst = P.solve(pair.Ip, pair.Im, gn_iters=2, contract=False)
    assert status == 0
    gs = host(st)
    assert np.array_equal(gs[:, 6], rst[:, 6]), (gs[:, 6], rst[:, 6])        # accepted steps
    assert np.array_equal(gs[:, 7], rst[:, 7]), (gs[:, 7], rst[:, 7])        # PCG iterations
    assert np.allclose(gs[:, 0], rst[:, 0], rtol=1e-4), (gs[:, 0], rst[:, 0])
    assert rel(host(b), ref) <= 1e-3, rel(host(b), ref)


def test_3t_polarity_swap_symmetry(H, pair):
    """Reversing the phase-encoding direction (swapping the images, negating the field) maps T+ to
    T- and back (Eq. 1): J and its terms are unchanged, the gradient and the solved field change
    sign.  The OT field is exactly antisymmetric (its operations only exchange operands); the
    objective holds the symmetry up to single-precision rounding, because fused multiply-adds
    round the two images' products in the other order on the swapped pair, so the tolerances are
    the parity ones: terms 1e-5, gradient 1e-5 / 2e-4, the 20-iteration solve 1e-3 with the
    objective history 1e-4 and the same accepted steps and PCG iteration counts."""
    h = H(pair.dims, pair.spacing, pair.pe_dim, ALPHA, BETA)
    Ip, Im = dev(pair.Ip), dev(pair.Im)
    b0 = host(h.init_ot(Ip, Im))
    assert np.array_equal(host(h.init_ot(Im, Ip)), -b0)
    t1, g1 = (host(x).copy() for x in h.eval(Ip, Im, dev(b0)))
    t2, g2 = (host(x).copy() for x in h.eval(Im, Ip, dev(-b0)))
    assert np.all(np.abs(t2 - t1) <= 1e-5 * np.abs(t1)), (t1, t2)
    check_field(-g2, g1, "swapped gradient")
    b1, st1 = (host(x).copy() for x in h.solve(Ip, Im, gn_iters=20))
    b2, st2 = (host(x).copy() for x in h.solve(Im, Ip, gn_iters=20))
    assert np.array_equal(st2[:, 6], st1[:, 6]) and np.array_equal(st2[:, 7], st1[:, 7])
    assert np.allclose(st2[:, 0], st1[:, 0], rtol=1e-4), (st1[:, 0], st2[:, 0])
    assert rel(-b2, b1) <= 1e-3, rel(-b2, b1)
