"""The mixed-precision path: split-BF16 products on the tensor cores
(tcgen05), diagonal tiles in FP64.

Error model: x ~ t0 + t1 (+ t2) with BF16 terms; bf16x3 keeps the term
products down to 2^-8 of the leading one and bf16x6 down to 2^-16, so a
product is accurate to about 2^-16 (x3) or 2^-24 (x6) relative, plus FP32
accumulation over at most 2048 terms.  A dropped term product would raise the
error to 2^-8 (x3) or 2^-16 (x6), far above the tolerances below.
"""
import numpy as np
import pytest

import oracle
from paper_1602_07527_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
GEMM_TOL = {"bf16x3": 1e-4, "bf16x6": 2e-6}
# results of whole passes on well-conditioned (Wishart, condition ~5) inputs
OPS_TOL = {"bf16x3": 1e-3, "bf16x6": 1e-6}


@pytest.fixture(scope="module")
def cd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1602_07527_gb300 as m
    return m


@pytest.fixture(scope="module")
def nat(cd):
    from paper_1602_07527_gb300 import native
    return native


GEMM_CASES = [(1, 1, 1, False), (5, 7, 3, False), (128, 128, 64, False), (130, 70, 200, False),
              (257, 300, 1000, False), (64, 64, 5000, False), (300, 300, 777, True), (129, 129, 64, True)]


@pytest.mark.parametrize("prec", ["bf16x3", "bf16x6"])
@pytest.mark.parametrize("M,N,K,lower", GEMM_CASES)
def test_tensor_core_product(nat, prec, M, N, K, lower):
    rng = np.random.default_rng(M * 1000 + N * 10 + K)
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((N, K))
    ref = A @ B.T
    C = torch.full((M, N), float("nan"), dtype=torch.float64, device=DEV)
    nat.mixed_gemm_debug(torch.tensor(A, device=DEV), torch.tensor(B, device=DEV), C, prec=prec, lower=lower)
    torch.cuda.synchronize()
    out = C.cpu().numpy()
    if lower:
        assert np.all(np.isnan(out[np.triu_indices(M, 1)]))
        out, ref = np.tril(np.nan_to_num(out)), np.tril(ref)
    assert not np.any(np.isnan(out))
    err = np.linalg.norm(out - ref) / np.linalg.norm(ref)
    assert err <= GEMM_TOL[prec], err


def _case(n, seed):
    S = W.wishart(n, seed)
    L, info = oracle.chol_unblocked(S)
    assert info == 0
    return S, L, W.lbar(n, seed), W.sigma_dot(n, seed)


OPS_CASES = [(100, 64), (300, 64), (513, 128), (700, 128), (450, 96), (600, 256)]


@pytest.mark.parametrize("prec", ["bf16x3", "bf16x6"])
@pytest.mark.parametrize("n,nb", OPS_CASES)
def test_mixed_passes_vs_oracle(cd, prec, n, nb):
    S, L, Lb, Sd = _case(n, 1000 + n)
    A = torch.tensor(np.tril(S), device=DEV)
    assert int(cd.chol_fwd(A, nb=nb, prec=prec).item()) == 0
    Ld = torch.tensor(L, device=DEV)
    Ab = torch.tensor(Lb, device=DEV)
    cd.chol_rev(Ld, Ab, nb=nb, prec=prec)
    Ad = torch.tensor(np.tril(Sd), device=DEV)
    cd.chol_fwd_sens(Ld, Ad, nb=nb, prec=prec)
    torch.cuda.synchronize()
    e = [oracle.rel_fro(A.cpu().numpy(), L),
         oracle.rel_fro(Ab.cpu().numpy(), oracle.chol_unblocked_rev(L, Lb)),
         oracle.rel_fro(Ad.cpu().numpy(), oracle.chol_unblocked_fwd(L, Sd))]
    assert max(e) <= OPS_TOL[prec], e
    assert cd.device_error() == 0


def test_mixed_batched_ragged(cd):
    sizes = [0, 70, 200, 333, 64]
    cases = [_case(n, 1100 + i) if n else None for i, n in enumerate(sizes)]
    As = [torch.tensor(np.tril(c[0]), device=DEV) if c else torch.zeros((0, 0), dtype=torch.float64, device=DEV)
          for c in cases]
    info = cd.chol_fwd_batched(As, nb=64, prec="bf16x6")
    Ls = [torch.tensor(c[1], device=DEV) if c else As[i] for i, c in enumerate(cases)]
    Abs = [torch.tensor(c[2], device=DEV) if c else As[i].clone() for i, c in enumerate(cases)]
    cd.chol_rev_batched(Ls, Abs, nb=64, prec="bf16x6")
    torch.cuda.synchronize()
    assert np.all(info.cpu().numpy() == 0)
    for i, c in enumerate(cases):
        if c is None:
            continue
        a1 = torch.tensor(np.tril(c[0]), device=DEV)
        cd.chol_fwd(a1, nb=64, prec="bf16x6")
        r1 = torch.tensor(c[2], device=DEV)
        cd.chol_rev(Ls[i], r1, nb=64, prec="bf16x6")
        assert torch.equal(As[i], a1) and torch.equal(Abs[i], r1)   # batched == alone, bitwise
        assert oracle.rel_fro(As[i].cpu().numpy(), c[1]) <= OPS_TOL["bf16x6"]
        assert oracle.rel_fro(Abs[i].cpu().numpy(), oracle.chol_unblocked_rev(c[1], c[2])) <= OPS_TOL["bf16x6"]


def test_mixed_with_level2_diagonal(cd):
    n, nb = 333, 64
    S, L, Lb, Sd = _case(n, 1200)
    Ld = torch.tensor(L, device=DEV)
    Ab = torch.tensor(Lb, device=DEV)
    cd.chol_rev(Ld, Ab, nb=nb, prec="bf16x6", diag="level2")
    Ad = torch.tensor(np.tril(Sd), device=DEV)
    cd.chol_fwd_sens(Ld, Ad, nb=nb, prec="bf16x6", diag="level2")
    torch.cuda.synchronize()
    assert oracle.rel_fro(Ab.cpu().numpy(), oracle.chol_unblocked_rev(L, Lb)) <= OPS_TOL["bf16x6"]
    assert oracle.rel_fro(Ad.cpu().numpy(), oracle.chol_unblocked_fwd(L, Sd)) <= OPS_TOL["bf16x6"]
