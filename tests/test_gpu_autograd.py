"""Differentiation through the library: torch.autograd.Function whose backward
is cd_chol_rev, on the Gaussian-process negative log marginal likelihood
(inputs on [0,1]^4, targets iid N(0,1), theta = (s, l, sigma) = (1, 0.3, 0.1)),
at the GP configuration's sizes N = 2048 and 4096 and at a small N = 300."""
import numpy as np
import pytest

import oracle
from paper_1602_07527_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
THETA = (1.0, 0.3, 0.1)


@pytest.fixture(scope="module")
def ag():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_07527_gb300 import autograd
    return autograd


def _grad(ag, X, y, theta, nb=0):
    th = torch.tensor(theta, dtype=torch.float64, device=DEV, requires_grad=True)
    f = ag.gp_nlml(th, X, y, nb=nb)
    f.backward()
    return float(f.item()), th.grad.cpu().numpy()


@pytest.mark.parametrize("n", [300, 2048, 4096])
def test_gp_gradient_matches_oracle_and_fd(ag, n):
    Xn, yn = W.gp_case(n)
    X = torch.tensor(Xn, device=DEV)
    y = torch.tensor(yn, device=DEV)
    f, g = _grad(ag, X, y, THETA)
    # the CPU oracle: NLML and its gradient via chol_unblocked / chol_unblocked_rev
    assert abs(f - oracle.gp_nlml(THETA, Xn, yn)) <= 1e-9 * abs(f)
    g_ref = oracle.gp_nlml_grad(THETA, Xn, yn)
    assert np.max(np.abs(g - g_ref)) <= 1e-8 * np.max(np.abs(g_ref))
    # central finite differences, step 1e-6, through the library forward
    h = 1e-6
    fd = []
    with torch.no_grad():
        for t in range(3):
            tp = list(THETA)
            tm = list(THETA)
            tp[t] += h
            tm[t] -= h
            fp = ag.gp_nlml(torch.tensor(tp, dtype=torch.float64, device=DEV), X, y)
            fm = ag.gp_nlml(torch.tensor(tm, dtype=torch.float64, device=DEV), X, y)
            fd.append(float((fp - fm).item()) / (2 * h))
    assert np.max(np.abs(g - np.array(fd))) <= 1e-5 * np.max(np.abs(fd))


def test_cholesky_gradient_matches_torch(ag):
    """The symmetric gradient agrees with torch.linalg.cholesky's own backward."""
    n = 200
    S = torch.tensor(W.wishart(n, 40), device=DEV, requires_grad=True)
    Lb = torch.tensor(W.lbar(n, 40), device=DEV)
    (ag.cholesky(S, nb=64) * Lb).sum().backward()
    g1 = S.grad.clone()
    S.grad = None
    (torch.linalg.cholesky(S) * Lb).sum().backward()
    assert torch.allclose(g1, S.grad, rtol=1e-10, atol=1e-12)


def test_not_positive_definite_raises(ag):
    S = torch.eye(8, dtype=torch.float64, device=DEV)
    S[5, 5] = -1.0
    with pytest.raises(torch.linalg.LinAlgError):
        ag.cholesky(S)
