"""The upper-triangle convention (CD_UPPER, LAPACK's uplo = 'U'): Sigma = U^T U
with U = L^T, every routine reading and writing upper triangles only.

Each case builds the upper-form inputs from the lower-form ones by
transposition, poisons the strictly lower triangle with NaN (it must not be
read or written), and compares the result, transposed back, with the oracle.
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


def upper_poisoned(lower_part, pad=3):
    """An n x (n + pad) buffer: the transpose of the given lower triangle in
    the upper triangle, NaN in the strict lower triangle and the padding."""
    n = lower_part.shape[0]
    buf = np.full((n, n + pad), np.nan)
    buf[:, :n] = np.where(np.triu(np.ones((n, n), dtype=bool)), np.tril(lower_part).T, np.nan)
    return torch.tensor(buf, device=DEV)


def upper_part(t, n):
    a = t.cpu().numpy()
    assert np.all(np.isnan(a[np.tril_indices(n, -1)])), "strict lower triangle was written"
    assert np.all(np.isnan(a[:, n:])), "padding was written"
    return np.triu(np.nan_to_num(a[:, :n])).T  # back to the lower form


def case(n, seed):
    S = W.wishart(n, seed)
    L, info = oracle.chol_unblocked(S)
    assert info == 0
    return S, L, W.lbar(n, seed), W.sigma_dot(n, seed)


@pytest.mark.parametrize("n,nb", [(1, 64), (70, 32), (200, 64), (333, 96)])
@pytest.mark.parametrize("prec,tol", [("fp64", TOL), ("bf16x6", 1e-6)])
def test_upper_fwd_rev_sens(nat, n, nb, prec, tol):
    S, L, Lb, Sd = case(n, 4000 + n)
    A = upper_poisoned(S)
    assert int(nat.chol_fwd(A[:, :n], nb=nb, prec=prec, uplo="upper").item()) == 0
    assert oracle.rel_fro(upper_part(A, n), L) <= tol
    U = upper_poisoned(L)
    Ab = upper_poisoned(Lb)
    nat.chol_rev(U[:, :n], Ab[:, :n], nb=nb, prec=prec, uplo="upper")
    assert oracle.rel_fro(upper_part(Ab, n), oracle.chol_unblocked_rev(L, Lb)) <= tol
    Ad = upper_poisoned(Sd)
    nat.chol_fwd_sens(U[:, :n], Ad[:, :n], nb=nb, prec=prec, uplo="upper")
    assert oracle.rel_fro(upper_part(Ad, n), oracle.chol_unblocked_fwd(L, Sd)) <= tol


def test_upper_fwd_and_sens_and_batched(nat):
    sizes = [5, 0, 130, 64]
    cases = [case(n, 4100 + i) if n else None for i, n in enumerate(sizes)]
    z = lambda: torch.zeros((0, 0), dtype=torch.float64, device=DEV)  # noqa: E731
    As = [upper_poisoned(c[0], pad=0) if c else z() for c in cases]
    Ads = [upper_poisoned(c[3], pad=0) if c else z() for c in cases]
    info = nat.chol_fwd_and_sens_batched(As, Ads, nb=64, uplo="upper")
    assert np.all(info.cpu().numpy() == 0)
    for i, c in enumerate(cases):
        if c is None:
            continue
        n = sizes[i]
        L, Ld, _ = oracle.chol_unblocked_and_fwd(c[0], c[3])
        assert oracle.rel_fro(upper_part(As[i], n), L) <= TOL
        assert oracle.rel_fro(upper_part(Ads[i], n), Ld) <= TOL


def test_upper_symmetric_output(nat):
    n = 150
    _, L, Lb, _ = case(n, 4200)
    U = upper_poisoned(L, pad=0)
    Ab = upper_poisoned(Lb, pad=0)
    nat.chol_rev(U, Ab, nb=64, out="sym", uplo="upper")
    got = Ab.cpu().numpy()
    ref = oracle.sym_from_tril(oracle.chol_unblocked_rev(L, Lb))
    assert np.linalg.norm(got - ref) <= TOL * np.linalg.norm(ref)


def test_upper_info(nat):
    n, bad = 200, 150
    S = W.wishart(n, 4300)
    S[bad - 1, bad - 1] = -5.0 * n * n
    info = nat.chol_fwd(upper_poisoned(S, pad=0), nb=64, uplo="upper")
    assert int(info.item()) == bad
