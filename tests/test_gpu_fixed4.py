"""The fixed-point mixed mode (CD_MIXED_FIXED4) at small and ragged sizes.

The factorisation's products (Sec. 4.2 chol_blocked: Schur updates and the
panel solve) run on fixed-point slices: each operand rounded to 2^-32 of its
row maximum, the leading slice sums exact.  On well-conditioned inputs
(Wishart, condition ~5) L is then within ~1e-9 of the oracle; the derivative
passes of this mode use the three-term split (bf16x6), within ~1e-6.  Also:
ragged batches equal to the single calls bit for bit, the upper-triangle
convention, the one-loop pass, the factorisation's info word on non-positive
pivots, and upper triangles left untouched.
"""
import numpy as np
import pytest

import oracle
from paper_1602_07527_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
L_TOL = 1e-8      # the fixed-point factorisation
D_TOL = 1e-6      # derivative passes (three-term split)
PREC = "fixed4"


@pytest.fixture(scope="module")
def cd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1602_07527_gb300 as m
    return m


def _case(n, seed):
    S = W.wishart(n, seed)
    L, info = oracle.chol_unblocked(S)
    assert info == 0
    return S, L, W.lbar(n, seed), W.sigma_dot(n, seed)


def _dev(a):
    return torch.tensor(a, device=DEV)


@pytest.mark.parametrize("n,nb", [(1, 64), (65, 64), (100, 64), (300, 64), (513, 128), (700, 128), (450, 96),
                                  (600, 256)])
def test_fixed4_passes_vs_oracle(cd, n, nb):
    S, L, Lb, Sd = _case(n, 2000 + n)
    A = _dev(np.tril(S))
    assert int(cd.chol_fwd(A, nb=nb, prec=PREC).item()) == 0
    Ld, Ab, Ad = _dev(L), _dev(Lb), _dev(np.tril(Sd))
    cd.chol_rev(Ld, Ab, nb=nb, prec=PREC)
    cd.chol_fwd_sens(Ld, Ad, nb=nb, prec=PREC)
    A2, Ad2 = _dev(np.tril(S)), _dev(np.tril(Sd))
    cd.chol_fwd_and_sens(A2, Ad2, nb=nb, prec=PREC)
    torch.cuda.synchronize()
    e_fwd = oracle.rel_fro(A.cpu().numpy(), L)
    e_dual = oracle.rel_fro(A2.cpu().numpy(), L)
    e_rev = oracle.rel_fro(Ab.cpu().numpy(), oracle.chol_unblocked_rev(L, Lb))
    e_sens = oracle.rel_fro(Ad.cpu().numpy(), oracle.chol_unblocked_fwd(L, Sd))
    e_dsens = oracle.rel_fro(Ad2.cpu().numpy(), oracle.chol_unblocked_fwd(L, Sd))
    assert e_fwd <= L_TOL and e_dual <= L_TOL, (e_fwd, e_dual)
    assert max(e_rev, e_sens, e_dsens) <= D_TOL, (e_rev, e_sens, e_dsens)
    assert cd.device_error() == 0


def test_fixed4_product_shapes(cd):
    from paper_1602_07527_gb300 import native
    g = np.random.default_rng(5)
    for M, N, K, lower in [(1, 1, 1, False), (5, 7, 3, False), (130, 70, 200, False), (257, 300, 1000, False),
                           (64, 64, 5000, False), (300, 300, 777, True), (129, 129, 64, True)]:
        A = g.standard_normal((M, K))
        B = A if lower else g.standard_normal((N, K))
        ref = A @ B.T
        C = torch.zeros(ref.shape, dtype=torch.float64, device=DEV)
        native.mixed_gemm_debug(_dev(A), _dev(B), C, prec=PREC, lower=lower)
        torch.cuda.synchronize()
        got = C.cpu().numpy()
        if lower:
            assert np.count_nonzero(np.triu(got, 1)) == 0
            got, ref = np.tril(got), np.tril(ref)
        assert np.linalg.norm(got - ref) <= 1e-8 * np.linalg.norm(ref), (M, N, K, lower)


def test_fixed4_batched_equals_single(cd):
    sizes = [0, 70, 200, 333, 64, 129]
    cases = [_case(n, 2100 + i) if n else None for i, n in enumerate(sizes)]
    As = [_dev(np.tril(c[0])) if c else torch.zeros((0, 0), dtype=torch.float64, device=DEV) for c in cases]
    info = cd.chol_fwd_batched(As, nb=64, prec=PREC)
    torch.cuda.synchronize()
    assert np.all(info.cpu().numpy() == 0)
    for i, c in enumerate(cases):
        if c is None:
            continue
        a1 = _dev(np.tril(c[0]))
        cd.chol_fwd(a1, nb=64, prec=PREC)
        torch.cuda.synchronize()
        assert torch.equal(As[i], a1)
        assert oracle.rel_fro(As[i].cpu().numpy(), c[1]) <= L_TOL


def test_fixed4_upper_convention(cd):
    n, nb = 300, 64
    S, L, Lb, _ = _case(n, 2200)
    U = _dev(np.triu(S))
    assert int(cd.chol_fwd(U, nb=nb, prec=PREC, uplo="upper").item()) == 0
    torch.cuda.synchronize()
    assert oracle.rel_fro(U.cpu().numpy().T, L) <= L_TOL


@pytest.mark.parametrize("bad", [1, 70, 190])
def test_fixed4_info_first_bad_pivot(cd, bad):
    n = 256
    S = W.wishart(n, 2300 + bad)
    S[bad - 1, bad - 1] = -5.0 * n * n
    _, info_ref = oracle.chol_unblocked(S)
    assert info_ref == bad
    info = cd.chol_fwd(_dev(np.tril(S)), nb=64, prec=PREC)
    torch.cuda.synchronize()
    assert int(info.item()) == bad
    assert cd.device_error() == 0


def test_fixed4_leaves_upper_triangle(cd):
    n, nb = 257, 64
    S, L, _, Sd = _case(n, 2400)
    A = np.tril(S)
    A[np.triu_indices(n, 1)] = np.nan
    At = _dev(A)
    cd.chol_fwd(At, nb=nb, prec=PREC)
    Ad = np.tril(Sd)
    Ad[np.triu_indices(n, 1)] = np.nan
    A2, Ad2 = _dev(A), _dev(Ad)
    cd.chol_fwd_and_sens(A2, Ad2, nb=nb, prec=PREC)
    torch.cuda.synchronize()
    for X in (At, A2, Ad2):
        x = X.cpu().numpy()
        assert np.all(np.isnan(x[np.triu_indices(n, 1)]))
        assert not np.any(np.isnan(np.tril(x)))
    assert oracle.rel_fro(np.tril(At.cpu().numpy()), L) <= L_TOL
