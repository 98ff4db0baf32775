"""The oracle's OpenMP loops change no result: every sum has a fixed order (per-column sums in
column order, fixed chunks in chunk order), so one thread and several give identical bits."""
import numpy as np

from paper_2403_10706_b300 import phantom as ph


def run(orc, pr, threads):
    orc.set_threads(threads)
    P = orc.Problem(pr.dims, pr.spacing, pr.pe_dim, 300.0, 1e4)
    b0 = P.ot_init(pr.Ip, pr.Im, 1e-3, contract=True, blur=True)
    ev = P.eval(pr.Ip, pr.Im, b0, contract=True)
    b, status, st = P.solve(pr.Ip, pr.Im, gn_iters=3, contract=True)
    return b0, ev, b, st


def test_one_thread_and_many_give_identical_bits(orc):
    pr = ph.make_pair("tiny")
    try:
        b0a, eva, ba, sta = run(orc, pr, 1)
        b0b, evb, bb, stb = run(orc, pr, 4)
    finally:
        orc.set_threads(orc.max_threads())
    assert np.array_equal(b0a, b0b)
    for k in ("J", "D", "S", "P"):
        assert eva[k] == evb[k]
    assert np.array_equal(eva["grad"], evb["grad"])
    assert np.array_equal(ba, bb)
    assert np.array_equal(sta, stb, equal_nan=True)
