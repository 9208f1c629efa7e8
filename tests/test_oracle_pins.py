"""Pins for the CPU oracle: each check compares it with something other than
itself -- LAPACK, finite differences of a library Cholesky, the explicit
element formula (Eq. delements), closed forms, exact symbolic derivatives,
torch's own Cholesky gradient, the textbook Gaussian-process gradient and the
adjoint identity that links forward and reverse mode (Sec. 2).
"""
import numpy as np
import pytest

from paper_1602_07527_gb300 import workloads as W


def wishart(n, seed=1):
    return W.wishart(n, seed)


def lapack_chol(S):
    return np.linalg.cholesky(S)


def fd_jacobian(Sigma, h=1e-6):
    """Central-difference Jacobian dL_ij/dSigma_kl over tied pairs k >= l,
    using the library (LAPACK) Cholesky: each tied pair is perturbed by
    E = e_k e_l^T + e_l e_k^T (k != l) or e_k e_k^T."""
    n = Sigma.shape[0]
    J = np.zeros((n, n, n, n))
    for k in range(n):
        for l in range(k + 1):
            E = np.zeros((n, n))
            E[k, l] = 1.0
            E[l, k] = 1.0
            J[:, :, k, l] = (lapack_chol(Sigma + h * E) - lapack_chol(Sigma - h * E)) / (2 * h)
    return J


# -- forward factorisation ---------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 3, 5, 17, 64, 130])
def test_fwd_matches_lapack(oracle, n):
    S = wishart(n)
    L, info = oracle.chol_unblocked(S)
    assert info == 0
    Lref = lapack_chol(S)
    assert np.max(np.abs(L - Lref)) <= 1e-13 * np.max(np.abs(Lref))
    # invariant L L^T = Sigma (backward error of a few ulps times n)
    assert np.linalg.norm(L @ L.T - S) <= 4 * n * 2.2e-16 * np.linalg.norm(S)
    assert np.all(np.diag(L) > 0)


def test_fwd_n1_closed_form(oracle):
    L, info = oracle.chol_unblocked(np.array([[2.25]]))
    assert info == 0 and L[0, 0] == 1.5


def test_fwd_info_reports_first_bad_pivot(oracle):
    S = np.diag([4.0, 1.0, -1.0, 3.0])
    _, info = oracle.chol_unblocked(S)
    assert info == 3
    S = wishart(6)
    S[4, 4] = np.nan
    _, info = oracle.chol_unblocked(S)
    assert info == 5
    # semidefinite: rank-1 matrix fails at column 2
    v = np.arange(1.0, 5.0)
    _, info = oracle.chol_unblocked(np.outer(v, v))
    assert info == 2


# -- forward sensitivity ------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 5, 33, 96])
def test_sens_two_routes_agree(oracle, n):
    S = wishart(n)
    L, _ = oracle.chol_unblocked(S)
    Sd = W.sigma_dot(n, 1)
    a = oracle.chol_unblocked_fwd(L, Sd)
    b = oracle.chol_symbolic_fwd(L, Sd)
    assert oracle.rel_fro(a, b) <= 1e-13


@pytest.mark.parametrize("n", [2, 7, 40])
def test_sens_central_fd(oracle, n):
    """The paper's own check (Sec. code listing test): central differences of
    the library Cholesky with h = 1e-5, at rtol/atol far tighter than np.isclose."""
    S = wishart(n)
    Sd = W.sigma_dot(n, 1)
    L = lapack_chol(S)
    h = 1e-5
    fd = (lapack_chol(S + Sd * h / 2) - lapack_chol(S - Sd * h / 2)) / h
    a = oracle.chol_unblocked_fwd(L, Sd)
    assert oracle.rel_fro(a, fd) <= 1e-8


@pytest.mark.parametrize("n", [1, 2, 7, 40, 97])
def test_one_loop_fwd_and_sens(oracle, n):
    """Sec. 4.1's single loop: L against LAPACK, L_dot against central
    differences of LAPACK's Cholesky (h = 1e-5), and both bit for bit against
    the two routines run one after the other (same per-element arithmetic)."""
    S = wishart(n)
    Sd = W.sigma_dot(n, 1)
    L, Ld, info = oracle.chol_unblocked_and_fwd(S, Sd)
    assert info == 0
    Lref = lapack_chol(S)
    assert np.max(np.abs(L - Lref)) <= 1e-13 * np.max(np.abs(Lref))
    h = 1e-5
    fd = (lapack_chol(S + Sd * h / 2) - lapack_chol(S - Sd * h / 2)) / h
    assert oracle.rel_fro(Ld, fd) <= 1e-8
    L2, _ = oracle.chol_unblocked(S)
    assert np.array_equal(L, L2)
    assert np.array_equal(Ld, oracle.chol_unblocked_fwd(L2, Sd))


def test_one_loop_fwd_and_sens_reports_info(oracle):
    S = np.diag([4.0, 1.0, -1.0, 3.0])
    _, _, info = oracle.chol_unblocked_and_fwd(S, np.eye(4))
    assert info == 3


def test_sens_n1_closed_form(oracle):
    L = np.array([[3.0]])
    out = oracle.chol_unblocked_fwd(L, np.array([[1.5]]))
    assert out[0, 0] == 1.5 / (2 * 3.0)
    out = oracle.chol_symbolic_fwd(L, np.array([[1.5]]))
    assert out[0, 0] == 1.5 / (2 * 3.0)


# -- reverse mode ---------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 5, 33, 96, 150])
def test_rev_two_routes_agree(oracle, n):
    S = wishart(n)
    L, _ = oracle.chol_unblocked(S)
    Lb = W.lbar(n, 1)
    a = oracle.chol_unblocked_rev(L, Lb)
    b = oracle.chol_symbolic_rev(L, Lb)
    assert oracle.rel_fro(a, b) <= 1e-13


def test_rev_n1_closed_form(oracle):
    L = np.array([[3.0]])
    for f in (oracle.chol_unblocked_rev, oracle.chol_symbolic_rev):
        assert f(L, np.array([[1.5]]))[0, 0] == 1.5 / (2 * 3.0)


@pytest.mark.parametrize("n", [2, 3, 4, 6])
def test_rev_brute_force_fd_jacobian(oracle, n):
    S = wishart(n, seed=11)
    L = lapack_chol(S)
    Lb = W.lbar(n, 3)
    J = fd_jacobian(S)
    ref = np.einsum("ij,ijkl->kl", Lb, J)       # Sigma_bar_kl over tied pairs
    for f in (oracle.chol_unblocked_rev, oracle.chol_symbolic_rev):
        got = f(L, Lb)
        assert np.max(np.abs(got - np.tril(ref))) <= 1e-7 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("n", [3, 5])
def test_delements_matches_fd(oracle, n):
    """Eq. delements (explicit dL_ij/dSigma_kl) against brute-force FD."""
    S = wishart(n, seed=12)
    L = lapack_chol(S)
    J = oracle.dchol_jacobian(L)
    Jfd = fd_jacobian(S)
    mask = np.zeros_like(J, dtype=bool)
    for i in range(n):
        for j in range(i + 1):
            for k in range(n):
                for l in range(k + 1):
                    mask[i, j, k, l] = True
    assert np.max(np.abs(J[mask] - Jfd[mask])) <= 1e-8


@pytest.mark.parametrize("n", [4, 6])
def test_rev_and_sens_match_exact_jacobian(oracle, n):
    """Contracting Eq. delements with L_bar (reverse) or Sigma_dot (forward)
    must reproduce both oracle routes to rounding."""
    S = wishart(n, seed=13)
    L, _ = oracle.chol_unblocked(S)
    J = oracle.dchol_jacobian(L)
    Lb = W.lbar(n, 5)
    rev_ref = np.tril(np.einsum("ij,ijkl->kl", Lb, J))
    assert oracle.rel_fro(oracle.chol_unblocked_rev(L, Lb), rev_ref) <= 1e-13
    assert oracle.rel_fro(oracle.chol_symbolic_rev(L, Lb), rev_ref) <= 1e-13
    Sd = W.sigma_dot(n, 5)
    fwd_ref = np.einsum("ijkl,kl->ij", J, np.tril(Sd))
    assert oracle.rel_fro(oracle.chol_unblocked_fwd(L, Sd), fwd_ref) <= 1e-13
    assert oracle.rel_fro(oracle.chol_symbolic_fwd(L, Sd), fwd_ref) <= 1e-13


def test_rev_diagonal_sigma_closed_form(oracle):
    """Diagonal Sigma: Sigma_bar_ij = L_bar_ij / L_jj (i > j), L_bar_ii / (2 L_ii)."""
    n = 9
    d = np.linspace(0.5, 4.0, n)
    L = np.diag(np.sqrt(d))
    Lb = W.lbar(n, 2)
    ref = np.tril(Lb / np.sqrt(d)[None, :], -1) + np.diag(np.diag(Lb) / (2 * np.sqrt(d)))
    for f in (oracle.chol_unblocked_rev, oracle.chol_symbolic_rev):
        assert np.max(np.abs(f(L, Lb) - ref)) <= 1e-15 * np.max(np.abs(ref)) * 4


@pytest.mark.parametrize("n", [3, 50, 130])
def test_adjoint_identity(oracle, n):
    """<L_bar, L_dot> = sum_{i>=j} Sigma_bar_ij Sigma_dot_ij (Sec. 2 reverse vs forward)."""
    S = wishart(n, seed=4)
    L, _ = oracle.chol_unblocked(S)
    Lb = W.lbar(n, 4)
    Sd = W.sigma_dot(n, 4)
    lhs = float((Lb * oracle.chol_unblocked_fwd(L, Sd)).sum())
    for f in (oracle.chol_unblocked_rev, oracle.chol_symbolic_rev):
        rhs = float((f(L, Lb) * np.tril(Sd)).sum())
        assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


def test_sympy_exact_derivatives_3x3(oracle):
    """Exact derivatives of the closed-form 3x3 Cholesky, by computer algebra,
    at a rational SPD point."""
    sp = pytest.importorskip("sympy")
    a = sp.symbols("s00 s10 s11 s20 s21 s22")
    Sig = sp.Matrix([[a[0], a[1], a[3]], [a[1], a[2], a[4]], [a[3], a[4], a[5]]])
    l00 = sp.sqrt(Sig[0, 0])
    l10 = Sig[1, 0] / l00
    l20 = Sig[2, 0] / l00
    l11 = sp.sqrt(Sig[1, 1] - l10 ** 2)
    l21 = (Sig[2, 1] - l20 * l10) / l11
    l22 = sp.sqrt(Sig[2, 2] - l20 ** 2 - l21 ** 2)
    Lsym = {(0, 0): l00, (1, 0): l10, (1, 1): l11, (2, 0): l20, (2, 1): l21, (2, 2): l22}
    pairs = [(0, 0), (1, 0), (1, 1), (2, 0), (2, 1), (2, 2)]
    point = dict(zip(a, [sp.Rational(4), sp.Rational(1, 2), sp.Rational(3),
                         sp.Rational(-1, 3), sp.Rational(1, 4), sp.Rational(2)]))
    S = np.array(Sig.subs(point).evalf(30).tolist(), dtype=float)
    L, _ = oracle.chol_unblocked(S)
    Lb = np.tril(np.array([[0.7, 0, 0], [-1.1, 0.3, 0], [0.25, 2.0, -0.6]]))
    ref = np.zeros((3, 3))
    for (k, l), sym in zip(pairs, a):
        ref[k, l] = float(sum(Lb[i, j] * sp.diff(Lsym[(i, j)], sym).subs(point).evalf(30)
                              for (i, j) in pairs))
    for f in (oracle.chol_unblocked_rev, oracle.chol_symbolic_rev):
        assert np.max(np.abs(f(L, Lb) - ref)) <= 1e-14 * np.max(np.abs(ref)) * 8


def test_torch_cholesky_gradient_convention(oracle):
    """torch's symmetric gradient equals (tril Sigma_bar + tril Sigma_bar^T)/2."""
    torch = pytest.importorskip("torch")
    n = 12
    S = wishart(n, seed=6)
    Lb = W.lbar(n, 6)
    St = torch.tensor(S, dtype=torch.float64, requires_grad=True)
    Lt = torch.linalg.cholesky(St)
    Lt.backward(torch.tensor(Lb))
    L, _ = oracle.chol_unblocked(S)
    T = oracle.chol_unblocked_rev(L, Lb)
    ref = 0.5 * (T + T.T)
    assert np.max(np.abs(St.grad.numpy() - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_sym_output_matches_eq_symrev(oracle):
    """Eq. symrev: Sigma_bar = S + S^T - diag S, S = L^{-T} Phi(L^T L_bar) L^{-1}."""
    n = 10
    L, _ = oracle.chol_unblocked(wishart(n, seed=7))
    Lb = W.lbar(n, 7)
    Li = np.linalg.inv(L)
    Sm = Li.T @ oracle.phi(L.T @ Lb) @ Li
    ref = Sm + Sm.T - np.diag(np.diag(Sm))
    got = oracle.sym_from_tril(oracle.chol_symbolic_rev(L, Lb))
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_upper_triangle_is_not_read(oracle):
    n = 20
    S = wishart(n, seed=8)
    L, _ = oracle.chol_unblocked(S)
    Lb = W.lbar(n, 8)
    Sd = W.sigma_dot(n, 8)
    iu = np.triu_indices(n, 1)
    P = lambda M: (lambda X: (X.__setitem__(iu, np.nan), X)[1])(M.copy())
    Lp = P(L)
    assert np.array_equal(oracle.chol_unblocked(P(S))[0], L)
    assert np.array_equal(oracle.chol_unblocked_fwd(Lp, P(Sd)), oracle.chol_unblocked_fwd(L, Sd))
    assert np.array_equal(oracle.chol_unblocked_rev(Lp, P(Lb)), oracle.chol_unblocked_rev(L, Lb))
    assert np.array_equal(oracle.chol_symbolic_rev(Lp, P(Lb)), oracle.chol_symbolic_rev(L, Lb))
    assert np.array_equal(oracle.chol_symbolic_fwd(Lp, Sd), oracle.chol_symbolic_fwd(L, Sd))


# -- Gaussian-process likelihood gradient (differentiation demo) -------------

def test_gp_gradient_textbook_and_fd(oracle):
    n = 48
    X, y = W.gp_case(n)
    theta = np.array([1.0, 0.3, 0.1])
    g = oracle.gp_nlml_grad(theta, X, y)
    # textbook: dNLML/dt = 0.5 tr(Sigma^{-1} dSigma) - 0.5 alpha^T dSigma alpha
    S = oracle.gp_sigma(theta, X)
    alpha = np.linalg.solve(S, y)
    Si = np.linalg.inv(S)
    ref = np.array([0.5 * np.trace(Si @ dS) - 0.5 * alpha @ dS @ alpha
                    for dS in oracle.gp_dsigma(theta, X)])
    assert np.max(np.abs(g - ref)) <= 1e-9 * max(1.0, np.max(np.abs(ref)))
    # central differences, step 1e-6
    h = 1e-6
    fd = np.zeros(3)
    for t in range(3):
        e = np.zeros(3)
        e[t] = h
        fd[t] = (oracle.gp_nlml(theta + e, X, y) - oracle.gp_nlml(theta - e, X, y)) / (2 * h)
    assert np.max(np.abs(g - fd)) <= 1e-5 * max(1.0, np.max(np.abs(fd)))
    # the likelihood itself against a library log-determinant and solve
    sign, logdet = np.linalg.slogdet(S)
    assert abs(oracle.gp_nlml(theta, X, y) - (0.5 * y @ alpha + 0.5 * logdet)) <= 1e-10 * abs(logdet)


# -- column residuals used to check full-size results ------------------------

@pytest.mark.parametrize("n", [7, 90])
def test_column_residuals_accept_exact_and_reject_perturbed(oracle, n):
    S = wishart(n, seed=30)
    L, _ = oracle.chol_unblocked(S)
    Lb = W.lbar(n, 30)
    Sd = W.sigma_dot(n, 30)
    T = oracle.chol_unblocked_rev(L, Lb)
    Ld = oracle.chol_unblocked_fwd(L, Sd)
    cols = list(range(0, n, max(1, n // 6)))
    assert oracle.fwd_residual_columns(S, L, cols) <= 1e-14
    assert oracle.sens_residual_columns(Sd, L, Ld, cols) <= 1e-14
    assert oracle.rev_residual_columns(L, Lb, T, cols) <= 1e-14
    # a relative perturbation of 1e-9 anywhere in the checked columns' reach is visible
    E = np.zeros((n, n))
    E[n - 1, cols[-1]] = 1e-9 * np.max(np.abs(T))
    assert oracle.rev_residual_columns(L, Lb, T + E, cols) > 1e-12
    E = np.zeros((n, n))
    E[n - 1, cols[-1]] = 1e-9 * np.max(np.abs(Ld))
    assert oracle.sens_residual_columns(Sd, L, Ld + E, cols) > 1e-12
    E = np.zeros((n, n))
    E[n - 1, cols[-1]] = 1e-9 * np.max(np.abs(L))
    assert oracle.fwd_residual_columns(S, L + E, cols) > 1e-12
