"""Batched solve (hysco_batch_*): pairs of uneven sizes and PE axes advancing through the GN loop
together, with one cooperative PCG launch per GN step for the whole batch.  Every pair is checked
against the double-precision oracle's own solve of that pair (same tolerances as a single solve:
objective history relative 1e-4, final field relative 1e-3, the accepted-step and PCG-iteration
sequences equal).  The batch's PCG sums each pair's dot products over its own block range, so a
pair's iterates differ from a single solve only by the order of single-precision additions.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2403_10706_b300 import _lib  # noqa: E402
from paper_2403_10706_b300 import phantom as ph  # noqa: E402

ALPHA, BETA = 300.0, 1e4
GN = 6
BASE = dict(n_ellipsoids=3, n_blobs=2, semi_axes=(3.0, 9.0), smooth=0.5, n_gauss=3,
            sigma=(4.0, 6.0), noise=0.01)
RECIPES = [
    dict(BASE, dims=(32, 32, 16), spacing=(1.0, 1.0, 1.0), pe_dim=1, seed=5001, bmax=3.0),
    dict(BASE, dims=(24, 40, 20), spacing=(1.2, 1.0, 1.1), pe_dim=0, seed=5002, bmax=2.5),
    dict(BASE, dims=(20, 18, 36), spacing=(1.0, 1.0, 1.0), pe_dim=2, seed=5003, bmax=2.0),
    dict(BASE, dims=(48, 56, 30), spacing=(1.5, 1.5, 1.5), pe_dim=1, seed=5004, bmax=3.5),
    dict(BASE, dims=(33, 27, 21), spacing=(1.0, 1.25, 1.0), pe_dim=1, seed=5005, bmax=2.0),
]


@pytest.fixture(scope="module")
def mods():
    from paper_2403_10706_b300 import build
    build.build()
    from paper_2403_10706_b300.hysco import Hysco, HyscoBatch
    return Hysco, HyscoBatch


@pytest.fixture(scope="module")
def problem(mods, orc):
    Hysco, HyscoBatch = mods
    pairs = [ph.make_pair(r) for r in RECIPES]
    refs = []
    for pr in pairs:
        P = orc.Problem(pr.dims, pr.spacing, pr.pe_dim, ALPHA, BETA)
        b, status, st = P.solve(pr.Ip, pr.Im, gn_iters=GN, contract=False)
        assert status == 0
        refs.append((b, st))
    hs = [Hysco(pr.dims, pr.spacing, pr.pe_dim, ALPHA, BETA) for pr in pairs]
    Ips = [torch.from_numpy(pr.Ip).cuda() for pr in pairs]
    Ims = [torch.from_numpy(pr.Im).cuda() for pr in pairs]
    return pairs, refs, hs, Ips, Ims


def rel(a, b):
    return np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300)


def check_against_oracle(bs, sts, refs, hs, what):
    for i, (b, st) in enumerate(zip(bs, sts)):
        assert hs[i].last_status() == 0, (what, i)
        ref_b, ref_st = refs[i]
        gs = st.cpu().numpy()
        assert np.array_equal(gs[:, 6], ref_st[:, 6]), (what, i, gs[:, 6], ref_st[:, 6])
        assert np.array_equal(gs[:, 7], ref_st[:, 7]), (what, i, gs[:, 7], ref_st[:, 7])
        assert np.allclose(gs[:, 0], ref_st[:, 0], rtol=1e-4), (what, i)
        assert rel(b.cpu().numpy(), ref_b) <= 1e-3, (what, i, rel(b.cpu().numpy(), ref_b))


def test_batch_matches_oracle_per_pair(mods, problem):
    _, HyscoBatch = mods
    pairs, refs, hs, Ips, Ims = problem
    batch = HyscoBatch(hs)
    bs, sts = batch.solve(Ips, Ims, gn_iters=GN)
    torch.cuda.synchronize()
    check_against_oracle(bs, sts, refs, hs, "default schedule")
    branches, policy, grid = batch.schedule()
    assert 1 <= branches <= 8 and 0 <= policy <= 8 and grid >= len(hs)


def test_batch_graph_replay_equals_direct_launches(mods, problem):
    _, HyscoBatch = mods
    pairs, refs, hs, Ips, Ims = problem
    batch = HyscoBatch(hs)
    outs = []
    bs = [h._new_fld() for h in hs]
    for graph in (False, True, True):
        bs, sts = batch.solve(Ips, Ims, bs=bs, init=True, gn_iters=GN, graph=graph)
        torch.cuda.synchronize()
        outs.append(([b.cpu().numpy().copy() for b in bs], [s.cpu().numpy() for s in sts]))
    for k in (1, 2):
        for i in range(len(hs)):
            assert np.array_equal(outs[0][0][i], outs[k][0][i])
            assert np.array_equal(outs[0][1][i], outs[k][1][i], equal_nan=True)


@pytest.mark.parametrize("branches,policy",
                         [(1, 0), (4, 1), (2, 2), (5, 2), (1, 3), (4, 3), (2, 4), (3, 5),
                          (1, 6), (4, 6), (2, 7), (3, 8)])
def test_every_schedule_matches_oracle(mods, problem, branches, policy):
    """Each PCG policy (shared launch with either block share, the pairs' own persistent kernels
    one after another, waves of pairs sharing one launch per GN step with barriers per pair, or
    waves whose pairs run their whole GN loops in one launch) and branch count gives every pair
    the oracle's trajectory.  The five small pairs of this batch fit one wave, so with policy 3
    all five PCGs, and with policy 6 all five GN loops, run in the same cooperative launch."""
    _, HyscoBatch = mods
    pairs, refs, hs, Ips, Ims = problem
    batch = HyscoBatch(hs)
    batch.set_schedule(branches, policy)
    assert batch.schedule()[:2] == (branches, policy)
    bs, sts = batch.solve(Ips, Ims, gn_iters=GN)
    torch.cuda.synchronize()
    check_against_oracle(bs, sts, refs, hs, f"schedule {(branches, policy)}")


def test_batch_tuner_picks_a_schedule_that_still_matches(mods, problem):
    _, HyscoBatch = mods
    pairs, refs, hs, Ips, Ims = problem
    batch = HyscoBatch(hs)
    sched = batch.tune(Ips, Ims, gn_iters=GN)
    assert sched == batch.schedule()
    assert 1 <= sched[0] <= 8 and 0 <= sched[1] <= 8
    bs, sts = batch.solve(Ips, Ims, gn_iters=GN)
    torch.cuda.synchronize()
    check_against_oracle(bs, sts, refs, hs, f"tuned {sched}")


def test_batch_rejects_bad_arguments(mods, problem):
    Hysco, HyscoBatch = mods
    pairs, refs, hs, Ips, Ims = problem
    lib = _lib.load()
    out = C.c_void_p()
    dup = (C.c_void_p * 2)(hs[0]._h.value, hs[0]._h.value)
    assert lib.hysco_batch_create(2, dup, C.byref(out)) == _lib.EINVAL
    batch = HyscoBatch(hs[:2])
    o = _lib.Opts(2, 10, 10, _lib.PC_COLUMN, 1, 1, 0.1, 1e-4, 1e-3, 0, 0)
    arr = lambda ts: (C.c_void_p * 2)(*[t.data_ptr() for t in ts])   # noqa: E731
    bs = [h._new_fld() for h in hs[:2]]
    rc = lib.hysco_batch_solve(batch._b, arr(Ips[:2]), arr(Ims[:2]), arr(bs), C.byref(o), None,
                               None)
    assert rc == _lib.EINVAL   # the batched PCG is Jacobi only
    with pytest.raises(ValueError):
        batch.solve(Ips[:2], Ims[::-1][:2])   # pair 1's images have the wrong shape
    for br, pol in ((0, 0), (3, 0), (1, 9), (1, -1)):   # 3 branches exceed the 2 pairs
        assert lib.hysco_batch_set_schedule(batch._b, br, pol) == _lib.EINVAL
