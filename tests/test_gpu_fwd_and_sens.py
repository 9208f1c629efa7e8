"""Parity of the one-loop factorisation and forward-sensitivity pass
(cd_chol_fwd_and_sens: Sec. 4.1-4.2 allow the forward-mode updates to be
accumulated in the factorisation's loop) with the oracle's one-loop routine.

Both outputs come from the same call, so L_dot is computed from the GPU's own
L.  On well-conditioned inputs (Wishart, condition ~5) both are compared
element by element at 1e-11; at N = 2048 the squared-exponential recipe is
taken with jitter 2e-3 (condition <= 1e6, where the 1e-11 FP64 bound is
stated); at N = 8192 (the benchmark's configuration) sampled columns are
checked against Sigma = L L^T and Sigma_dot = L_dot L^T + L L_dot^T.
"""
import numpy as np
import pytest

import oracle
from paper_1602_07527_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TOL = 1e-11
MIXED_TOL = {"bf16x3": 1e-3, "bf16x6": 1e-6}


@pytest.fixture(scope="module")
def nat():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_07527_gb300 import native
    return native


def dev(x):
    return torch.tensor(np.ascontiguousarray(x), device=DEV)


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def ref(n, seed):
    S = W.wishart(n, seed)
    Sd = W.sigma_dot(n, seed)
    L, Ld, info = oracle.chol_unblocked_and_fwd(S, Sd)
    assert info == 0
    return S, Sd, L, Ld


SHAPES = [(1, 64), (2, 64), (3, 2), (33, 16), (40, 1), (64, 64), (65, 64), (129, 128), (200, 64),
          (300, 128), (333, 96), (450, 192), (600, 256)]


@pytest.mark.parametrize("n,nb", SHAPES)
@pytest.mark.parametrize("diag", ["auto", "level2", "symbolic"])
def test_fwd_and_sens_parity(nat, n, nb, diag):
    S, Sd, L, Ld = ref(n, 1500 + n)
    A, Ad = dev(np.tril(S)), dev(np.tril(Sd))
    info = nat.chol_fwd_and_sens(A, Ad, nb=nb, diag=diag)
    assert int(info.item()) == 0
    assert oracle.rel_fro(host(A), L) <= TOL
    assert oracle.rel_fro(host(Ad), Ld) <= TOL


def test_fwd_and_sens_leaves_upper_and_padding(nat):
    n, nb, pad = 200, 64, 5
    S, Sd, L, Ld = ref(n, 1600)
    bufs = []
    for x in (S, Sd):
        b = np.full((n, n + pad), np.nan)
        b[:, :n] = np.where(np.tril(np.ones((n, n), dtype=bool)), x, np.nan)
        bufs.append(dev(b))
    A, Ad = bufs
    nat.chol_fwd_and_sens(A[:, :n], Ad[:, :n], nb=nb)
    a, ad = host(A), host(Ad)
    assert np.all(np.isnan(a[np.triu_indices(n, 1)])) and np.all(np.isnan(a[:, n:]))
    assert np.all(np.isnan(ad[np.triu_indices(n, 1)])) and np.all(np.isnan(ad[:, n:]))
    assert oracle.rel_fro(np.tril(a[:, :n]), L) <= TOL
    assert oracle.rel_fro(np.tril(ad[:, :n]), Ld) <= TOL


def test_fwd_and_sens_matches_the_two_calls(nat):
    """Same exact result as cd_chol_fwd followed by cd_chol_fwd_sens."""
    n, nb = 333, 64
    S, Sd, L, Ld = ref(n, 1700)
    A, Ad = dev(np.tril(S)), dev(np.tril(Sd))
    nat.chol_fwd_and_sens(A, Ad, nb=nb)
    A2, Ad2 = dev(np.tril(S)), dev(np.tril(Sd))
    nat.chol_fwd(A2, nb=nb)
    nat.chol_fwd_sens(A2, Ad2, nb=nb)
    assert oracle.rel_fro(host(A), host(A2)) <= TOL
    assert oracle.rel_fro(host(Ad), host(Ad2)) <= TOL


@pytest.mark.parametrize("n,nb,bad", [(200, 64, 150), (200, 64, 1), (130, 128, 129), (600, 256, 444)])
def test_fwd_and_sens_info(nat, n, nb, bad):
    S = W.wishart(n, 1800 + n)
    S[bad - 1, bad - 1] = -5.0 * n * n
    _, _, info_ref = oracle.chol_unblocked_and_fwd(S, W.sigma_dot(n, 1))
    assert info_ref == bad
    info = nat.chol_fwd_and_sens(dev(np.tril(S)), dev(np.tril(W.sigma_dot(n, 1))), nb=nb)
    assert int(info.item()) == bad


def test_fwd_and_sens_empty_and_invalid(nat):
    z = torch.zeros((0, 0), dtype=torch.float64, device=DEV)
    assert int(nat.chol_fwd_and_sens(z, z.clone()).item()) == 0
    A = torch.zeros((4, 4), dtype=torch.float64, device=DEV)
    with pytest.raises(nat.CholDiffError):
        nat.chol_fwd_and_sens(A, A)              # outputs must not be the same array
    with pytest.raises(ValueError):
        nat.chol_fwd_and_sens(A, torch.zeros((5, 5), dtype=torch.float64, device=DEV))


def test_fwd_and_sens_batched_equals_single(nat):
    sizes = [0, 1, 5, 64, 100, 257, 130, 33]
    nb = 64
    cases = [ref(n, 1900 + i) if n else None for i, n in enumerate(sizes)]
    z = lambda: torch.zeros((0, 0), dtype=torch.float64, device=DEV)  # noqa: E731
    As = [dev(np.tril(c[0])) if c else z() for c in cases]
    Ads = [dev(np.tril(c[1])) if c else z() for c in cases]
    info = nat.chol_fwd_and_sens_batched(As, Ads, nb=nb)
    assert np.all(host(info) == 0)
    for i, c in enumerate(cases):
        if c is None:
            continue
        a1, ad1 = dev(np.tril(c[0])), dev(np.tril(c[1]))
        nat.chol_fwd_and_sens(a1, ad1, nb=nb)
        torch.cuda.synchronize()
        assert torch.equal(As[i], a1) and torch.equal(Ads[i], ad1)   # batched == alone, bitwise
        assert oracle.rel_fro(host(As[i]), c[2]) <= TOL
        assert oracle.rel_fro(host(Ads[i]), c[3]) <= TOL


@pytest.mark.parametrize("prec", ["bf16x3", "bf16x6"])
@pytest.mark.parametrize("n,nb", [(100, 64), (300, 64), (513, 128), (600, 256)])
def test_fwd_and_sens_mixed(nat, prec, n, nb):
    S, Sd, L, Ld = ref(n, 2000 + n)
    A, Ad = dev(np.tril(S)), dev(np.tril(Sd))
    assert int(nat.chol_fwd_and_sens(A, Ad, nb=nb, prec=prec).item()) == 0
    e = [oracle.rel_fro(host(A), L), oracle.rel_fro(host(Ad), Ld)]
    assert max(e) <= MIXED_TOL[prec], e
    assert nat.device_error() == 0


def test_fwd_and_sens_mixed_batched_equals_single(nat):
    sizes = [70, 0, 200, 333]
    cases = [ref(n, 2100 + i) if n else None for i, n in enumerate(sizes)]
    z = lambda: torch.zeros((0, 0), dtype=torch.float64, device=DEV)  # noqa: E731
    As = [dev(np.tril(c[0])) if c else z() for c in cases]
    Ads = [dev(np.tril(c[1])) if c else z() for c in cases]
    nat.chol_fwd_and_sens_batched(As, Ads, nb=64, prec="bf16x6")
    for i, c in enumerate(cases):
        if c is None:
            continue
        a1, ad1 = dev(np.tril(c[0])), dev(np.tril(c[1]))
        nat.chol_fwd_and_sens(a1, ad1, nb=64, prec="bf16x6")
        torch.cuda.synchronize()
        assert torch.equal(As[i], a1) and torch.equal(Ads[i], ad1)
        assert oracle.rel_fro(host(Ads[i]), c[3]) <= MIXED_TOL["bf16x6"]


def test_n2048_se_against_full_oracle(nat):
    n = 2048
    S, _ = W.large_se_case(n, 2, jitter=2e-3)
    Sd = W.sigma_dot(n, 2)
    L, Ld, info = oracle.chol_unblocked_and_fwd(S, Sd)
    assert info == 0
    A, Ad = dev(np.tril(S)), dev(np.tril(Sd))
    assert int(nat.chol_fwd_and_sens(A, Ad).item()) == 0
    e_l, e_ld = oracle.rel_fro(host(A), L), oracle.rel_fro(host(Ad), Ld)
    print(f"N={n} SE jitter 2e-3: L {e_l:.2e} L_dot {e_ld:.2e}")
    assert e_l <= TOL and e_ld <= TOL


def test_n8192_column_residuals(nat):
    n = 8192
    S, _ = W.large_se_case(n, 2)
    Sd = W.sigma_dot(n, 2)
    A, Ad = dev(np.tril(S)), dev(np.tril(Sd))
    assert int(nat.chol_fwd_and_sens(A, Ad).item()) == 0
    L, Ld = host(A), host(Ad)
    cols = [0, 1, 127, 128, 4095, 6000, n - 129, n - 1]
    r_fwd = oracle.fwd_residual_columns(S, L, cols)
    r_sens = oracle.sens_residual_columns(Sd, L, Ld, cols)
    print(f"column residuals at N={n}: fwd {r_fwd:.2e} sens {r_sens:.2e}")
    assert r_fwd <= TOL and r_sens <= TOL
