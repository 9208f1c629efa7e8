"""Accuracy of the mixed-precision path at the sizes of its target workload.

The mixed-precision target: every result of the split-BF16 path within a
relative Frobenius error of 1e-5 of FP64, on the Matern-5/2 covariance
(ell 0.2 on [0,1]^4, jitter 1e-3, condition number below 1e6) at
N = 8192 and 16384.  The FP64 path these errors are taken against is pinned
to the CPU oracle element by element (test_gpu_parity, test_gpu_fullsize).

CD_MIXED_FIXED4 runs the factorisation's products (Sec. 4.2 chol_blocked:
the Schur updates of the diagonal block and the panel, and the panel solve)
on fixed-point slices and the derivative passes on the three-term split;
the errors checked are those of L, of L_dot and Sigma_bar given the FP64
factor, and of the whole mixed pipeline (L_dot and Sigma_bar computed from
the mixed factor).  The fixed-point product itself is checked alone: bit
for bit on integer operands, where every partial sum is exact, and against
FP64 on the rows of a Cholesky factor.
"""
import numpy as np
import pytest

from paper_1602_07527_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5
DEV = "cuda:0"


@pytest.fixture(scope="module")
def cd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1602_07527_gb300 as m
    return m


def _rel(x, ref):
    x, ref = torch.tril(x), torch.tril(ref)
    return (torch.linalg.norm(x - ref) / torch.linalg.norm(ref)).item()


def test_fixed_product_exact_on_integer_operands(cd):
    from paper_1602_07527_gb300 import native
    g = np.random.default_rng(11)
    for M, N, K, lower in ((300, 200, 1000, False), (129, 65, 64, False), (1024, 512, 4096, False),
                           (384, 384, 2000, True)):
        A = g.integers(-127, 128, (M, K)).astype(np.float64)
        B = A if lower else g.integers(-127, 128, (N, K)).astype(np.float64)
        ref = A @ B.T  # integers below 2^53: exact
        C = torch.zeros((M, B.shape[0]), dtype=torch.float64, device=DEV)
        native.mixed_gemm_debug(torch.tensor(A, device=DEV), torch.tensor(B, device=DEV), C, prec="fixed4",
                                lower=lower)
        torch.cuda.synchronize()
        got = C.cpu().numpy()
        if lower:
            assert np.count_nonzero(np.triu(got, 1)) == 0
            got, ref = np.tril(got), np.tril(ref)
        assert np.array_equal(got, ref), (M, N, K, lower)


def test_fixed_product_on_factor_rows(cd):
    from paper_1602_07527_gb300 import native
    n = 2048
    S, _ = W.mixed_matern_case(n)
    L = np.linalg.cholesky(S)
    for j in (256, 1024, 1536):
        k = j + 128
        B, R = L[k:, :j].copy(), L[j:k, :j].copy()
        ref = B @ R.T
        C = torch.zeros(ref.shape, dtype=torch.float64, device=DEV)
        native.mixed_gemm_debug(torch.tensor(B, device=DEV), torch.tensor(R, device=DEV), C, prec="fixed4")
        torch.cuda.synchronize()
        err = np.linalg.norm(C.cpu().numpy() - ref) / np.linalg.norm(ref)
        assert err <= 1e-8, (j, err)  # operands rounded to 2^-32 of their row maxima


@pytest.mark.parametrize("n", [8192, 16384])
def test_fixed4_matern_every_result_within_target(cd, n):
    S, Lb = W.mixed_matern_case(n)
    Sd = np.tril(W.sigma_dot(n, 3))
    S, Lb, Sd = (torch.tensor(a, device=DEV) for a in (S, Lb, Sd))
    L = S.clone()
    cd.chol_fwd(L)
    Ld = Sd.clone()
    cd.chol_fwd_sens(L, Ld)
    Sb = Lb.clone()
    cd.chol_rev(L, Sb)
    prec = "fixed4"
    Lm = S.clone()
    info = cd.chol_fwd(Lm, prec=prec)
    Ld_given = Sd.clone()
    cd.chol_fwd_sens(L, Ld_given, prec=prec)
    Ld_full = Sd.clone()
    cd.chol_fwd_sens(Lm, Ld_full, prec=prec)
    Sb_given = Lb.clone()
    cd.chol_rev(L, Sb_given, prec=prec)
    Sb_full = Lb.clone()
    cd.chol_rev(Lm, Sb_full, prec=prec)
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    errs = {"L": _rel(Lm, L), "L_dot given L": _rel(Ld_given, Ld), "L_dot full": _rel(Ld_full, Ld),
            "Sigma_bar given L": _rel(Sb_given, Sb), "Sigma_bar full": _rel(Sb_full, Sb)}
    if n == 8192:  # the one-loop pass gives the same two results
        A, Ad = S.clone(), Sd.clone()
        cd.chol_fwd_and_sens(A, Ad, prec=prec)
        torch.cuda.synchronize()
        errs["L (one loop)"] = _rel(A, L)
        errs["L_dot (one loop)"] = _rel(Ad, Ld)
    print(n, {k: f"{v:.2e}" for k, v in errs.items()})
    assert all(v <= TOL for v in errs.values()), errs
