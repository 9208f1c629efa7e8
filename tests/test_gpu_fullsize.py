"""Parity at the benchmark's sizes.

N = 8192 (the timed configuration: SE covariance ell 0.3 on [0,1]^3 + 1e-4 I,
default options): each result on sampled columns against the equation that
defines it (Sigma = L L^T; Sigma_dot = L_dot L^T + L L_dot^T from Eq. symfwd;
L^T (T + T^T) L = P + P^T from Eq. symrevtril), O(N^2) per column; and
element by element against the full oracle (about a minute per routine on
the host's cores), at the benchmark's jitter and at the jitter that keeps the
condition number below 1e6.
N = 2048 (same recipe): element by element against the full oracle.
"""
import numpy as np
import pytest

import oracle
from paper_1602_07527_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
RES_TOL = 1e-11    # column residual, relative to the size of the terms (see oracle docstrings)


@pytest.fixture(scope="module")
def cd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1602_07527_gb300 as m
    return m


def test_n8192_bench_configuration_column_residuals(cd):
    n = 8192
    S, Lb = W.large_se_case(n, 2)
    Sd = W.sigma_dot(n, 2)
    A = torch.tensor(np.tril(S), device=DEV)
    assert int(cd.chol_fwd(A).item()) == 0
    Ad = torch.tensor(np.tril(Sd), device=DEV)
    cd.chol_fwd_sens(A, Ad)
    Ab = torch.tensor(Lb, device=DEV)
    cd.chol_rev(A, Ab)
    torch.cuda.synchronize()
    L, Ld, T = A.cpu().numpy(), Ad.cpu().numpy(), Ab.cpu().numpy()
    cols = sorted(set([0, 1, 127, 128, 4095, 6000, n - 129, n - 1]))
    r_fwd = oracle.fwd_residual_columns(S, L, cols)
    r_sens = oracle.sens_residual_columns(Sd, L, Ld, cols)
    r_rev = oracle.rev_residual_columns(L, Lb, T, cols)
    print(f"column residuals at N={n}: fwd {r_fwd:.2e} sens {r_sens:.2e} rev {r_rev:.2e}")
    assert r_fwd <= RES_TOL and r_sens <= RES_TOL and r_rev <= RES_TOL


@pytest.mark.parametrize("diag", ["symbolic", "level2"])
def test_n2048_se_against_full_oracle(cd, diag):
    n = 2048
    S, Lb = W.large_se_case(n, 2)
    Sd = W.sigma_dot(n, 2)
    L, info = oracle.chol_unblocked(S)
    assert info == 0
    A = torch.tensor(np.tril(S), device=DEV)
    assert int(cd.chol_fwd(A).item()) == 0
    Ld = torch.tensor(L, device=DEV)
    Ab = torch.tensor(Lb, device=DEV)
    cd.chol_rev(Ld, Ab, diag=diag)
    Ad = torch.tensor(np.tril(Sd), device=DEV)
    cd.chol_fwd_sens(Ld, Ad, diag=diag)
    torch.cuda.synchronize()
    e_fwd = oracle.rel_fro(A.cpu().numpy(), L)
    e_rev = oracle.rel_fro(Ab.cpu().numpy(), oracle.chol_unblocked_rev(L, Lb))
    e_sens = oracle.rel_fro(Ad.cpu().numpy(), oracle.chol_unblocked_fwd(L, Sd))
    print(f"N={n} SE diag={diag}: fwd {e_fwd:.2e} rev {e_rev:.2e} sens {e_sens:.2e}")
    assert max(e_fwd, e_rev, e_sens) <= 1e-11


@pytest.mark.slow
@pytest.mark.parametrize("jitter,with_sens", [(2e-3, True), (1e-4, False)])
def test_n8192_against_full_oracle(cd, jitter, with_sens):
    """N = 8192 element by element against the full oracle (Sec. 4.1
    chol_unblocked, chol_unblocked_rev, chol_unblocked_fwd; about a minute
    each on the host's cores).  Jitter 2e-3 gives the condition number below
    1e6 that the FP64 target is stated for (about 8.5e5); jitter 1e-4 is the
    benchmark's own recipe (condition number about 1.7e7).  The derivative
    passes take the oracle's factor as their input, so that they are compared
    on the same L."""
    n = 8192
    S, Lb = W.large_se_case(n, 2, jitter=jitter)
    L, info = oracle.chol_unblocked(S)
    assert info == 0
    A = torch.tensor(np.tril(S), device=DEV)
    assert int(cd.chol_fwd(A).item()) == 0
    Ld = torch.tensor(L, device=DEV)
    Ab = torch.tensor(Lb, device=DEV)
    cd.chol_rev(Ld, Ab)
    if with_sens:
        Sd = W.sigma_dot(n, 2)
        Ad = torch.tensor(np.tril(Sd), device=DEV)
        cd.chol_fwd_sens(Ld, Ad)
    torch.cuda.synchronize()
    errs = {"fwd": oracle.rel_fro(A.cpu().numpy(), L),
            "rev": oracle.rel_fro(Ab.cpu().numpy(), oracle.chol_unblocked_rev(L, Lb))}
    if with_sens:
        errs["sens"] = oracle.rel_fro(Ad.cpu().numpy(), oracle.chol_unblocked_fwd(L, Sd))
    print(f"N={n} SE jitter {jitter:g}: " + " ".join(f"{k} {v:.2e}" for k, v in errs.items()))
    assert max(errs.values()) <= 1e-11, errs
