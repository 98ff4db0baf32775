"""The persistent PCG keeps r, p and H p of each thread's own float4 groups in shared memory for
the whole launch (on-chip slots) and the remaining slots in global memory.  Where a vector lives
changes no arithmetic: solves with every slot on chip, with none, and with a split give
bit-identical fields and statistics, and on one B300 the plan puts the whole field of the 3T
(144x168x111), 7T-shaped and small workloads on chip."""
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


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("name", ["3t", "7t", "small"])
def test_onchip_placement_is_bit_identical(H, name):
    pr = ph.make_pair(name)
    h = H(pr.dims, pr.spacing, pr.pe_dim, ALPHA, BETA)
    grid, onchip, slots, block = h.pcg_plan()
    assert grid > 0 and slots >= 1 and block >= 32
    assert onchip == slots, (grid, onchip, slots)
    Ip = torch.from_numpy(pr.Ip).cuda()
    Im = torch.from_numpy(pr.Im).cuda()
    outs = []
    for k in sorted({0, onchip // 2, onchip}):
        h.set_pcg_onchip(k)
        assert h.pcg_plan()[1] == k
        b, st = h.solve(Ip, Im, gn_iters=6, pcg_path=2)
        assert h.last_status() == 0
        outs.append((k, host(b).copy(), host(st).copy()))
    for k, b, st in outs[1:]:
        assert np.array_equal(b, outs[0][1]), (k, outs[0][0])
        assert np.array_equal(st, outs[0][2], equal_nan=True), (k, outs[0][0])
    h.set_pcg_onchip(-1)
    assert h.pcg_plan()[1] == onchip
    with pytest.raises(_lib.HyscoError):
        h.set_pcg_onchip(onchip + 1)
