"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerance: relative Frobenius error of the lower triangles <= 1e-11 for the
FP64 path (the stated FP64 target for condition numbers up to 1e6); integer
results (info) must match exactly.
"""
import numpy as np
import pytest

import oracle
from paper_1602_07527_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-11
DEV = "cuda:0"


@pytest.fixture(scope="module")
def cd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1602_07527_gb300 as m
    return m


def dev(x):
    return torch.tensor(np.ascontiguousarray(x), device=DEV)


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def case(n, seed):
    S = W.wishart(n, seed)
    L, info = oracle.chol_unblocked(S)
    assert info == 0
    return S, L, W.lbar(n, seed), W.sigma_dot(n, seed)


SHAPES = [(1, 64), (2, 64), (3, 2), (31, 16), (33, 16), (40, 1), (64, 64), (65, 64), (127, 64),
          (128, 128), (129, 128), (200, 64), (300, 128), (333, 96)]


@pytest.mark.parametrize("n,nb", SHAPES)
def test_fwd_parity(cd, n, nb):
    S, L, _, _ = case(n, 100 + n)
    A = dev(np.tril(S))
    info = cd.chol_fwd(A, nb=nb)
    assert int(info.item()) == 0
    assert oracle.rel_fro(host(A), L) <= TOL


@pytest.mark.parametrize("n,nb", SHAPES)
def test_rev_parity(cd, n, nb):
    _, L, Lb, _ = case(n, 200 + n)
    Ab = dev(Lb)
    cd.chol_rev(dev(L), Ab, nb=nb)
    ref = oracle.chol_unblocked_rev(L, Lb)
    assert oracle.rel_fro(host(Ab), ref) <= TOL


@pytest.mark.parametrize("n,nb", SHAPES)
def test_sens_parity(cd, n, nb):
    _, L, _, Sd = case(n, 300 + n)
    Ad = dev(np.tril(Sd))
    cd.chol_fwd_sens(dev(L), Ad, nb=nb)
    ref = oracle.chol_unblocked_fwd(L, Sd)
    assert oracle.rel_fro(host(Ad), ref) <= TOL


@pytest.mark.parametrize("n,nb", [(600, 256), (450, 192), (300, 160)])
def test_recursive_diagonal_blocks(cd, n, nb):
    """nb > 128: the diagonal step recurses into the blocked routine."""
    S, L, Lb, Sd = case(n, 400 + n)
    A = dev(np.tril(S))
    assert int(cd.chol_fwd(A, nb=nb).item()) == 0
    assert oracle.rel_fro(host(A), L) <= TOL
    Ab = dev(Lb)
    cd.chol_rev(dev(L), Ab, nb=nb)
    assert oracle.rel_fro(host(Ab), oracle.chol_unblocked_rev(L, Lb)) <= TOL
    Ad = dev(np.tril(Sd))
    cd.chol_fwd_sens(dev(L), Ad, nb=nb)
    assert oracle.rel_fro(host(Ad), oracle.chol_unblocked_fwd(L, Sd)) <= TOL


def test_empty_is_noop(cd):
    A = torch.zeros((0, 0), dtype=torch.float64, device=DEV)
    info = cd.chol_fwd(A)
    assert int(info.item()) == 0
    cd.chol_rev(A, A.clone())
    cd.chol_fwd_sens(A, A.clone())


def _poison_upper(x, pad):
    """Embed x in a wider row-major buffer; NaN in the strict upper triangle and the padding."""
    n = x.shape[0]
    buf = np.full((n, n + pad), np.nan)
    buf[:, :n] = np.where(np.tril(np.ones((n, n), dtype=bool)), x, np.nan)
    return buf


@pytest.mark.parametrize("n,nb", [(70, 32), (200, 64)])
def test_upper_triangle_and_padding_untouched(cd, n, nb):
    S, L, Lb, Sd = case(n, 500 + n)
    pad = 5
    upper = np.triu(np.ones((n, n + pad), dtype=bool), 1)
    Lp = dev(_poison_upper(L, pad))[:, :n]
    for kind in ("fwd", "rev", "sens"):
        src = {"fwd": S, "rev": Lb, "sens": Sd}[kind]
        buf = dev(_poison_upper(src, pad))
        view = buf[:, :n]
        if kind == "fwd":
            assert int(cd.chol_fwd(view, nb=nb).item()) == 0
            ref = L
        elif kind == "rev":
            cd.chol_rev(Lp, view, nb=nb)
            ref = oracle.chol_unblocked_rev(L, Lb)
        else:
            cd.chol_fwd_sens(Lp, view, nb=nb)
            ref = oracle.chol_unblocked_fwd(L, Sd)
        out = host(buf)
        assert np.all(np.isnan(out[upper])), kind
        assert oracle.rel_fro(np.tril(out[:, :n]), ref) <= TOL, kind


def test_rev_symmetric_output(cd):
    n = 150
    _, L, Lb, _ = case(n, 600)
    Ab = dev(Lb + np.triu(np.full((n, n), 7.0), 1))
    cd.chol_rev(dev(L), Ab, nb=64, out="sym")
    out = host(Ab)
    ref = oracle.sym_from_tril(oracle.chol_unblocked_rev(L, Lb))
    assert np.max(np.abs(out - ref)) <= TOL * np.linalg.norm(ref)
    assert np.array_equal(out, out.T)


@pytest.mark.parametrize("n,nb,bad", [(200, 64, 150), (200, 64, 1), (130, 128, 129), (90, 32, 64),
                                      (600, 256, 444)])
def test_fwd_info_first_bad_pivot(cd, n, nb, bad):
    S = W.wishart(n, 700 + n)
    S[bad - 1, bad - 1] = -5.0 * n * n
    _, info_ref = oracle.chol_unblocked(S)
    assert info_ref == bad
    A = dev(np.tril(S))
    info = cd.chol_fwd(A, nb=nb)
    assert int(info.item()) == bad
    S2 = W.wishart(n, 701)
    S2[bad - 1, bad - 1] = np.nan
    info = cd.chol_fwd(dev(np.tril(S2)), nb=nb)
    assert int(info.item()) == bad


BATCH_SIZES = [0, 1, 5, 64, 100, 257, 130, 33]


def test_batched_equals_single_and_oracle(cd):
    nb = 64
    cases = [case(n, 800 + i) if n > 0 else (np.zeros((0, 0)),) * 4 for i, n in enumerate(BATCH_SIZES)]
    # forward
    As = [dev(np.tril(c[0])) for c in cases]
    info = cd.chol_fwd_batched(As, nb=nb)
    assert np.all(host(info) == 0)
    # reverse and forward sensitivity
    Ls = [dev(c[1]) for c in cases]
    Abs = [dev(c[2]) for c in cases]
    Ads = [dev(np.tril(c[3])) for c in cases]
    cd.chol_rev_batched(Ls, Abs, nb=nb)
    cd.chol_fwd_sens_batched(Ls, Ads, nb=nb)
    torch.cuda.synchronize()
    for i, n in enumerate(BATCH_SIZES):
        if n == 0:
            continue
        S, L, Lb, Sd = cases[i]
        a1 = dev(np.tril(S))
        cd.chol_fwd(a1, nb=nb)
        r1 = dev(Lb)
        cd.chol_rev(Ls[i], r1, nb=nb)
        s1 = dev(np.tril(Sd))
        cd.chol_fwd_sens(Ls[i], s1, nb=nb)
        # every launch parameter of a problem depends on its own shape only:
        # a batched problem is computed exactly as it would be alone
        assert torch.equal(As[i], a1)
        assert torch.equal(Abs[i], r1)
        assert torch.equal(Ads[i], s1)
        assert oracle.rel_fro(host(As[i]), L) <= TOL
        assert oracle.rel_fro(host(Abs[i]), oracle.chol_unblocked_rev(L, Lb)) <= TOL
        assert oracle.rel_fro(host(Ads[i]), oracle.chol_unblocked_fwd(L, Sd)) <= TOL


def test_invalid_arguments_raise(cd):
    A = torch.zeros((4, 4), dtype=torch.float64, device=DEV)
    with pytest.raises(cd.CholDiffError):
        cd.chol_fwd(A, nb=-1)
    with pytest.raises(TypeError):
        cd.chol_fwd(A.float())
    with pytest.raises(ValueError):
        cd.chol_rev(A, torch.zeros((5, 5), dtype=torch.float64, device=DEV))


def test_launch_count_increases(cd):
    before = cd.launch_count()
    _, L, Lb, _ = case(96, 900)
    cd.chol_rev(dev(L), dev(Lb), nb=32)
    assert cd.launch_count() > before


@pytest.mark.parametrize("n,nb", [(1, 64), (2, 64), (33, 16), (129, 128), (300, 128), (333, 96), (600, 256)])
def test_symbolic_diagonal_step_matches_oracle(cd, n, nb):
    """The diagonal routine as the products of Eq. symrevtril / Eq. symfwd
    (the paper's alternative to the level-2 loop) gives the same result."""
    _, L, Lb, Sd = case(n, 950 + n)
    Ab = dev(Lb)
    cd.chol_rev(dev(L), Ab, nb=nb, diag="symbolic")
    assert oracle.rel_fro(host(Ab), oracle.chol_unblocked_rev(L, Lb)) <= TOL
    Ad = dev(np.tril(Sd))
    cd.chol_fwd_sens(dev(L), Ad, nb=nb, diag="symbolic")
    assert oracle.rel_fro(host(Ad), oracle.chol_unblocked_fwd(L, Sd)) <= TOL


def test_symbolic_diagonal_leaves_upper_untouched(cd):
    n, nb = 200, 64
    _, L, Lb, Sd = case(n, 990)
    pad = 3
    upper = np.triu(np.ones((n, n + pad), dtype=bool), 1)
    Lp = dev(_poison_upper(L, pad))[:, :n]
    for kind in ("rev", "sens"):
        buf = dev(_poison_upper(Lb if kind == "rev" else Sd, pad))
        if kind == "rev":
            cd.chol_rev(Lp, buf[:, :n], nb=nb, diag="symbolic")
            ref = oracle.chol_unblocked_rev(L, Lb)
        else:
            cd.chol_fwd_sens(Lp, buf[:, :n], nb=nb, diag="symbolic")
            ref = oracle.chol_unblocked_fwd(L, Sd)
        out = host(buf)
        assert np.all(np.isnan(out[upper])), kind
        assert oracle.rel_fro(np.tril(out[:, :n]), ref) <= TOL, kind


@pytest.mark.parametrize("diag", ["auto", "level2", "symbolic"])
def test_single_block_batches(cd, diag):
    """Batches where every problem is one block (the serving case for small n)."""
    sizes = [1, 7, 33, 64, 100, 128]
    cases = [case(n, 1300 + n) for n in sizes]
    Ls = [dev(c[1]) for c in cases]
    Abs = [dev(c[2]) for c in cases]
    Ads = [dev(np.tril(c[3])) for c in cases]
    cd.chol_rev_batched(Ls, Abs, nb=128, diag=diag)
    cd.chol_fwd_sens_batched(Ls, Ads, nb=128, diag=diag)
    torch.cuda.synchronize()
    for c, ab, ad in zip(cases, Abs, Ads):
        _, L, Lb, Sd = c
        assert oracle.rel_fro(host(ab), oracle.chol_unblocked_rev(L, Lb)) <= TOL
        assert oracle.rel_fro(host(ad), oracle.chol_unblocked_fwd(L, Sd)) <= TOL
