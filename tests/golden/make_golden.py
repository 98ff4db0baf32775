"""Writes tests/golden/oracle_fixtures.json: oracle outputs on two small fixed inputs.

Regression fixtures for the oracle itself (the paper prints no worked example): any later change
to the oracle's arithmetic shows up here and must name the passage of the paper that justifies
it.  Calls only oracle/ and the seeded input generator.
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2403_10706_b300 import phantom as ph  # noqa: E402


def fixtures():
    out = {}
    # one 8-cell column, PE spacing 1.7 mm
    rng = np.random.default_rng(2024)
    m = 8
    Ip = rng.uniform(0.1, 1.0, m).astype(np.float32)
    Im = rng.uniform(0.1, 1.0, m).astype(np.float32)
    b = np.cumsum(np.r_[0.4, rng.uniform(-0.5, 0.5, m)]).astype(np.float32)
    P = oracle.Problem((1, m, 1), (1.0, 1.7, 1.0), 1, 0.3, 0.02)
    e = P.eval(Ip.reshape(1, m, 1), Im.reshape(1, m, 1), b.reshape(1, m + 1, 1), contract=True)
    out["column8"] = dict(Ip=Ip.tolist(), Im=Im.tolist(), b=b.tolist(), spacing=[1.0, 1.7, 1.0],
                          alpha=0.3, beta=0.02, J=e["J"], D=e["D"], S=e["S"], P=e["P"],
                          grad=e["grad"].ravel().tolist())
    # the tiny phantom: terms at the OT initial field and after 3 GN iterations
    pr = ph.make_pair("tiny")
    P = oracle.Problem(pr.dims, pr.spacing, pr.pe_dim, 300.0, 1e4)
    b0 = P.ot_init(pr.Ip, pr.Im, 1e-3, contract=True, blur=True)
    e0 = P.eval(pr.Ip, pr.Im, b0, contract=True, grad=False)
    bs, st, stats = P.solve(pr.Ip, pr.Im, gn_iters=3, contract=True)
    out["tiny"] = dict(b0_sum=float(b0.sum()), b0_absmax=float(np.abs(b0).max()), J0=e0["J"],
                       J_iters=stats[:, 0].tolist(), gamma=stats[:, 6].tolist(),
                       final_norm=float(np.linalg.norm(bs)))
    return out


if __name__ == "__main__":
    with open(os.path.join(HERE, "oracle_fixtures.json"), "w") as f:
        json.dump(fixtures(), f, indent=1)
