"""The allocation-free objective entry point (hysco_eval_static) against the handle-based one.

hysco_eval_static serves callers that cannot allocate device memory -- code running under a
memory manager that owns the whole device budget, or latency-critical code that cannot afford
cudaMalloc's implicit synchronisation.  It keeps its reduction scratch in a static device array
shared by every call, so this test calls it twice in a row on the same stream (the second call
must not see stale partial sums or a stale ticket counter) and compares both results with
hysco_eval, called through the C ABI, and with the double-precision oracle, within the parity
tolerances of the other GPU tests: relative 1e-5 on J, D, S, P and on the gradient's 2-norm,
2e-4 of the largest entry elementwise.  A third call without a gradient output must give the
same terms bit for bit (the same reduction in the same order).

This file is collected last on purpose: a failure here leaves every other test already run.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2403_10706_b300 import _lib, build  # noqa: E402
from paper_2403_10706_b300 import phantom as ph  # noqa: E402

CASES = [
    # (dims, spacing, pe_dim, alpha, beta, image dtype)
    ((32, 32, 16), (1.0, 1.0, 1.0), 1, 300.0, 1e4, torch.float32),
    ((9, 13, 7), (1.1, 1.25, 0.9), 0, 300.0, 1e4, torch.float32),
    ((6, 5, 19), (1.0, 1.0, 1.3), 2, 30.0, 1.0, torch.bfloat16),
]
DT = {torch.float32: _lib.F32, torch.bfloat16: _lib.BF16, torch.float16: _lib.F16}


def ptr(t):
    return C.c_void_p(t.data_ptr())


def stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("dims,spacing,p,alpha,beta,dtype", CASES)
def test_static_eval_matches_handle_eval_twice_in_a_row(orc, dims, spacing, p, alpha, beta,
                                                        dtype):
    build.build()
    lib = _lib.load()
    Ipn, Imn = ph.random_images(dims, 4242, 0.1, 1.0)
    bn = ph.random_field(dims, p, 4243, scale=2.0, smooth=1.0)
    Ip = torch.from_numpy(Ipn).cuda().to(dtype)
    Im = torch.from_numpy(Imn).cuda().to(dtype)
    b = torch.from_numpy(bn).cuda()
    cdims = (C.c_int64 * 3)(*dims)
    cspac = (C.c_double * 3)(*spacing)

    h = C.c_void_p()
    assert lib.hysco_create(cdims, cspac, p, alpha, beta, DT[dtype], C.byref(h)) == 0
    try:
        t_ref = torch.empty(4, dtype=torch.float64, device="cuda")
        g_ref = torch.empty_like(b)
        assert lib.hysco_eval(h, ptr(Ip), ptr(Im), ptr(b), ptr(t_ref), ptr(g_ref), stream()) == 0
        # the oracle on the values the GPU sees (bf16 images rounded, then widened exactly)
        P = orc.Problem(dims, spacing, p, alpha, beta)
        ev = P.eval(Ip.float().cpu().numpy(), Im.float().cpu().numpy(),
                    bn.astype(np.float64), contract=True)
        t_orc = np.array([ev["J"], ev["D"], ev["S"], ev["P"]])
        terms = []
        for call in range(2):
            t = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
            g = torch.full_like(b, float("nan"))
            rc = lib.hysco_eval_static(cdims, cspac, p, alpha, beta, DT[dtype], ptr(Ip), ptr(Im),
                                       ptr(b), ptr(t), ptr(g), stream())
            assert rc == 0, (call, _lib.strerror(rc))
            torch.cuda.synchronize()
            tn = t.cpu().numpy()
            terms.append(tn)
            gn = g.cpu().numpy()
            for tr, gr in ((t_ref.cpu().numpy(), g_ref.cpu().numpy()), (t_orc, ev["grad"])):
                assert np.all(np.abs(tn - tr) <= 1e-5 * np.abs(tr)), (call, tn, tr)
                assert np.linalg.norm(gn - gr) <= 1e-5 * np.linalg.norm(gr), call
                assert np.abs(gn - gr).max() <= 2e-4 * np.abs(gr).max(), call
        # without a gradient output: the same reduction, so the same terms bit for bit
        t = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
        rc = lib.hysco_eval_static(cdims, cspac, p, alpha, beta, DT[dtype], ptr(Ip), ptr(Im),
                                   ptr(b), ptr(t), None, stream())
        assert rc == 0, _lib.strerror(rc)
        torch.cuda.synchronize()
        assert np.array_equal(t.cpu().numpy(), terms[-1])
        assert np.array_equal(terms[0], terms[1])
    finally:
        lib.hysco_destroy(h)


def test_static_eval_rejects_oversized_grids_and_bad_arguments():
    build.build()
    lib = _lib.load()
    f = torch.zeros(8, device="cuda")
    t = torch.zeros(4, dtype=torch.float64, device="cuda")
    big = (C.c_int64 * 3)(2048, 2048, 200)      # 16384 * 51 blocks > 32768
    sp = (C.c_double * 3)(1.0, 1.0, 1.0)
    assert lib.hysco_eval_static(big, sp, 2, 1.0, 1.0, 0, ptr(f), ptr(f), ptr(f), ptr(t), None,
                                 stream()) == _lib.EINVAL
    small = (C.c_int64 * 3)(2, 2, 2)
    assert lib.hysco_eval_static(small, sp, 1, 1.0, 1.0, 0, ptr(f), ptr(f), ptr(f), None, None,
                                 stream()) == _lib.EINVAL
    assert lib.hysco_eval_static(small, sp, 5, 1.0, 1.0, 0, ptr(f), ptr(f), ptr(f), ptr(t), None,
                                 stream()) == _lib.EINVAL
