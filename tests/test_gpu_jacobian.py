"""The explicit Jacobian of Eq. delements on the GPU (cd_chol_jacobian).

Small n: element by element against the oracle's Eq. delements tensor
(itself pinned against finite differences and exact sympy derivatives).
Larger n, including n > 128 where the inverse of L is formed blockwise: the
exact contractions that define forward and reverse mode,
    sum_{k>=l} J[i,j,k,l] Sigma_dot[k,l] = L_dot[i,j]          (Sec. 2),
    sum_{i>=j} L_bar[i,j] J[i,j,k,l]     = tril(Sigma_bar)[k,l] (Eq. symrevtril),
against the oracle's chol_unblocked_fwd and chol_unblocked_rev.
"""
import numpy as np
import pytest

import oracle
from paper_1602_07527_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TOL = 1e-11


@pytest.fixture(scope="module")
def nat():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_07527_gb300 import native
    return native


def factor(n, seed):
    L, info = oracle.chol_unblocked(W.wishart(n, seed))
    assert info == 0
    return L


@pytest.mark.parametrize("n", [1, 2, 5, 8])
def test_jacobian_matches_oracle_tensor(nat, n):
    L = factor(n, 3000 + n)
    J = nat.chol_jacobian(torch.tensor(L, device=DEV)).cpu().numpy()
    ref = oracle.dchol_jacobian(L)
    assert np.max(np.abs(J - ref)) <= TOL * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("n", [33, 64, 129])
def test_jacobian_contractions(nat, n):
    L = factor(n, 3100 + n)
    Lb = W.lbar(n, 3100 + n)
    Sd = W.sigma_dot(n, 3100 + n)
    Jt = nat.chol_jacobian(torch.tensor(L, device=DEV))
    Lb_t = torch.tensor(Lb, device=DEV)
    Sd_t = torch.tensor(np.tril(Sd), device=DEV)
    rev = torch.einsum("ij,ijkl->kl", Lb_t, Jt).cpu().numpy()
    fwd = torch.einsum("ijkl,kl->ij", Jt, Sd_t).cpu().numpy()
    assert oracle.rel_fro(rev, oracle.chol_unblocked_rev(L, Lb)) <= TOL
    assert oracle.rel_fro(fwd, oracle.chol_unblocked_fwd(L, Sd)) <= TOL
    # zero outside i >= j, k >= l
    i, j = (torch.tensor(a, device=DEV) for a in np.triu_indices(n, 1))
    assert not bool(torch.any(Jt[i, j] != 0))
    assert not bool(torch.any(Jt[:, :, i, j] != 0))


def test_jacobian_empty_and_invalid(nat):
    z = torch.zeros((0, 0), dtype=torch.float64, device=DEV)
    assert nat.chol_jacobian(z).numel() == 0
    with pytest.raises(TypeError):
        nat.chol_jacobian(torch.zeros((3, 3), dtype=torch.float32, device=DEV))
