"""Failure detection without a GPU fault: the persistent kernels' device-wide barrier gives up
after a bounded spin and reports HYSCO_ETIMEOUT; the context stays usable.  The wait is made to
run out by a block that never arrives (hysco_selftest_barrier), with a ~10 ms budget.  The same
for the tensor-core z-update's mbarrier waits: a launch whose copies are never issued
(hysco_selftest_zsolve) gives up on its unfilled stages."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2403_10706_b300 import _lib  # noqa: E402
from paper_2403_10706_b300 import phantom as ph  # noqa: E402


@pytest.fixture(scope="module")
def lib():
    from paper_2403_10706_b300 import build
    build.build()
    torch.cuda.init()
    return _lib.load()


def stream():
    return torch.cuda.current_stream().cuda_stream


def test_barrier_completes_when_every_block_arrives(lib):
    for grid in (1, 2, 8, 64):
        assert lib.hysco_selftest_barrier(grid, -1, 2_000_000_000, stream()) == _lib.OK


@pytest.mark.parametrize("missing", [0, 3, 7])
def test_barrier_times_out_when_a_block_never_arrives(lib, missing):
    assert lib.hysco_selftest_barrier(8, missing, 20_000_000, stream()) == _lib.ETIMEOUT


def test_zsolve_waits_run_out_and_the_handle_recovers(lib, orc):
    """The tensor-core product launch whose stages never fill records HYSCO_ETIMEOUT (a ~10 ms
    budget per wait); the same handle's z-update then matches the oracle again."""
    from paper_2403_10706_b300.hysco import Hysco
    dims, spacing, p = (32, 40, 24), (1.0, 1.1, 0.9), 1
    h = Hysco(dims, spacing, p, 300.0, 1e4)
    assert h.zsolve_path() == 0
    assert lib.hysco_selftest_zsolve(h._h, 20_000_000, stream()) == _lib.ETIMEOUT
    assert lib.hysco_selftest_zsolve(h._h, 0, stream()) == _lib.EINVAL
    P = orc.Problem(dims, spacing, p, 300.0, 1e4)
    v = np.random.default_rng(905).standard_normal(P.fdims).astype(np.float32)
    z = h.admm_zsolve(torch.from_numpy(v).cuda(), 5.0).cpu().numpy()
    zref = P.admm_z_solve(5.0 * v.astype(np.float64), 5.0)
    assert np.linalg.norm(z - zref) <= 2e-5 * np.linalg.norm(zref)
    assert h.last_status() == 0


def test_context_is_usable_after_a_timeout(lib, orc):
    from paper_2403_10706_b300.hysco import Hysco
    assert lib.hysco_selftest_barrier(16, 5, 20_000_000, stream()) == _lib.ETIMEOUT
    pr = ph.make_pair("tiny")
    h = Hysco(pr.dims, pr.spacing, pr.pe_dim, 300.0, 1e4)
    Ip, Im = torch.from_numpy(pr.Ip).cuda(), torch.from_numpy(pr.Im).cuda()
    b = h.init_ot(Ip, Im)
    terms, _ = h.eval(Ip, Im, b)
    P = orc.Problem(pr.dims, pr.spacing, pr.pe_dim, 300.0, 1e4)
    ref = P.eval(pr.Ip, pr.Im, b.cpu().numpy(), contract=True, grad=False)["J"]
    assert abs(terms[0].item() - ref) <= 1e-5 * abs(ref)
    assert h.last_status() == 0
    assert lib.hysco_selftest_barrier(16, -1, 2_000_000_000, stream()) == _lib.OK
