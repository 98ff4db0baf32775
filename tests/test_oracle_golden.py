"""The oracle reproduces its committed fixtures (tests/golden/make_golden.py wrote them)."""
import json
import os

import numpy as np

from paper_2403_10706_b300 import phantom as ph

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_oracle_reproduces_fixtures(orc):
    with open(os.path.join(HERE, "oracle_fixtures.json")) as f:
        gold = json.load(f)
    c = gold["column8"]
    m = len(c["Ip"])
    P = orc.Problem((1, m, 1), c["spacing"], 1, c["alpha"], c["beta"])
    e = P.eval(np.array(c["Ip"], np.float32).reshape(1, m, 1),
               np.array(c["Im"], np.float32).reshape(1, m, 1),
               np.array(c["b"], np.float32).reshape(1, m + 1, 1), contract=True)
    for k in ("J", "D", "S", "P"):
        assert abs(e[k] - c[k]) <= 1e-14 * abs(c[k])
    assert np.allclose(e["grad"].ravel(), c["grad"], rtol=1e-13, atol=0)
    t = gold["tiny"]
    pr = ph.make_pair("tiny")
    P = orc.Problem(pr.dims, pr.spacing, pr.pe_dim, 300.0, 1e4)
    b0 = P.ot_init(pr.Ip, pr.Im, 1e-3, contract=True, blur=True)
    assert abs(b0.sum() - t["b0_sum"]) <= 1e-12 * max(1.0, abs(t["b0_sum"]))
    _, st, stats = P.solve(pr.Ip, pr.Im, gn_iters=3, contract=True)
    assert np.allclose(stats[:, 0], t["J_iters"], rtol=1e-12)
    assert np.array_equal(stats[:, 6], t["gamma"])
