"""The Armijo backtracking rule of the Gauss-Newton driver (Sec. 2.3.1), pinned on a case whose
objective along the search direction is known in closed form.

One PE column of two cells (three field nodes), both images zero and alpha = 0, so only the
barrier term of Eq. 3 is left: J(b) = beta vol/2 [phi(b1 - b0) + phi(b2 - b1)].  At b = (0, z, 0)
the two cells have delta = +z and -z; phi is even, so J = beta vol phi(z).  The gradient is
beta vol/2 phi'(z) (-1, 2, -1) and the (exact) Gauss-Newton Hessian beta vol/2 phi''(z) D^T D, for
which (-1, 2, -1) is an eigenvector with eigenvalue 3.  The solved direction is therefore
q = -phi'(z) / (3 phi''(z)) (-1, 2, -1), and along it both cells move together:
    J(b + gamma q) = beta vol phi(z - gamma s),   s = phi'(z) / phi''(z),
    grad^T q = -beta vol phi'(z)^2 / phi''(z).
The expected step is computed here from these closed forms and phi(z) = z^4 / (1 - z^2) alone:
the largest gamma = 2^-t with J(b + gamma q) <= J(b) + c1 gamma grad^T q.

With z = 1/2 and a demanding c1 the full step decreases J but not by enough, so a rule that drops
the sufficient-decrease term would take gamma = 1, and one that drops the gamma factor from it
would take none; both fail these tests.
"""
import numpy as np
import pytest

Z = 0.5
BETA = 1e4
SPACING = (1.0, 1.25, 1.0)
VOL = float(np.prod(SPACING))


def phi(z):
    return z ** 4 / (1.0 - z ** 2)


def dphi(z):
    return 2.0 * z ** 3 * (2.0 - z ** 2) / (1.0 - z ** 2) ** 2


def d2phi(z):
    return 2.0 * z ** 2 * (6.0 - 3.0 * z ** 2 + z ** 4) / (1.0 - z ** 2) ** 3


def expected_step(c1, ls_max=10):
    """(gamma, trials) of backtracking from gamma = 1 on the closed-form line J(gamma)."""
    s = dphi(Z) / d2phi(Z)
    J0 = BETA * VOL * phi(Z)
    gq = -BETA * VOL * dphi(Z) ** 2 / d2phi(Z)
    for t in range(ls_max):
        gam = 2.0 ** -t
        if BETA * VOL * phi(Z - gam * s) <= J0 + c1 * gam * gq:
            return gam, t + 1
    return 0.0, ls_max


def problem(orc):
    dims = (1, 2, 1)
    P = orc.Problem(dims, SPACING, 1, 0.0, BETA)
    zero = np.zeros(dims, np.float32)
    b = np.zeros((1, 3, 1))
    b[0, 1, 0] = Z
    return P, zero, b


# c1 and the step it must give: 1e-4 (the default) accepts the full step; 0.7 and 0.8 reject it
CASES = [(1e-4, 1.0), (0.7, 0.5), (0.8, 0.25)]


@pytest.mark.parametrize("c1,gamma", CASES)
def test_closed_form_line_search(c1, gamma):
    # the hand computation itself: the stated steps, with no near-ties at any trial
    assert expected_step(c1)[0] == gamma
    s = dphi(Z) / d2phi(Z)
    J0, gq = phi(Z), -dphi(Z) ** 2 / d2phi(Z)
    for t in range(4):
        gam = 2.0 ** -t
        assert abs(phi(Z - gam * s) - (J0 + c1 * gam * gq)) > 3e-3 * J0


@pytest.mark.parametrize("c1,gamma", CASES)
def test_oracle_armijo_matches_closed_form(orc, c1, gamma):
    P, zero, b0 = problem(orc)
    ev = P.eval(zero, zero, b0, contract=False)
    assert ev["J"] == pytest.approx(BETA * VOL * phi(Z), rel=1e-14)
    g = ev["grad"].ravel()
    assert np.allclose(g, 0.5 * BETA * VOL * dphi(Z) * np.array([-1.0, 2.0, -1.0]), rtol=1e-13)
    b, status, st = P.solve(zero, zero, b=b0, gn_iters=1, init=False, contract=False,
                            pcg_rtol=1e-12, armijo_c1=c1)
    assert status == 0
    exp_gamma, exp_trials = expected_step(c1)
    assert st[0, 6] == exp_gamma == gamma
    assert st[0, 9] == exp_trials
    # the GN direction is the closed-form one up to a constant (the Hessian's null space, which
    # moves neither J nor delta), so the new cell slopes are those of b0 + gamma q: +-(z - gamma s)
    s = dphi(Z) / d2phi(Z)
    assert st[0, 5] == pytest.approx(-BETA * VOL * dphi(Z) ** 2 / d2phi(Z), rel=1e-10)
    delta = np.diff(b.ravel())
    assert np.allclose(delta, [Z - gamma * s, -(Z - gamma * s)], rtol=0, atol=1e-12)


@pytest.mark.gpu
@pytest.mark.parametrize("path", [1, 2, 4])
@pytest.mark.parametrize("c1,gamma", CASES)
def test_gpu_armijo_matches_closed_form(c1, gamma, path):
    """The same line through hysco_solve: the device-side Armijo decision (gamma = 1 as a full
    trial evaluation, then the halvings) takes the closed-form step, with the separate-kernel and
    the persistent PCG, and inside the persistent GN loop."""
    import torch
    from paper_2403_10706_b300.hysco import Hysco
    dev = torch.device("cuda", 0)
    h = Hysco((1, 2, 1), SPACING, 1, 0.0, BETA, device=dev)
    zero = torch.zeros((1, 2, 1), dtype=torch.float32, device=dev)
    b = torch.tensor([0.0, Z, 0.0], dtype=torch.float32, device=dev).reshape(1, 3, 1)
    b, st = h.solve(zero, zero, b=b, gn_iters=1, init=False, pcg_rtol=1e-6, armijo_c1=c1,
                    pcg_path=path)
    st = st.cpu().numpy()
    exp_gamma, exp_trials = expected_step(c1)
    assert h.last_status() == 0
    assert st[0, 6] == exp_gamma == gamma
    assert st[0, 9] == exp_trials
    s = dphi(Z) / d2phi(Z)
    assert st[0, 5] == pytest.approx(-BETA * VOL * dphi(Z) ** 2 / d2phi(Z), rel=1e-4)
    delta = np.diff(b.cpu().numpy().ravel().astype(np.float64))
    assert np.allclose(delta, [Z - gamma * s, -(Z - gamma * s)], rtol=0, atol=1e-5)
