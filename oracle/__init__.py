"""Plain FP64 CPU oracle for Murray, "Differentiation of the Cholesky
decomposition" (arXiv:1602.07527).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The CUDA library
and its Python binding never import it, and it imports nothing from them: the
two sides share no code.  The matrix routines live in ``cholref.c`` (plain C
loops, compiled by ``oracle/build.py``); this module adds ctypes marshalling,
the operator Phi, the explicit Jacobian of Eq. delements and the Gaussian-
process likelihood used by the differentiation demo.

Every routine takes and returns NumPy float64 arrays; only the lower triangle
of each input is read and every returned matrix is lower triangular.
"""
import ctypes

import numpy as np

from . import build as _build

_lib = None


def lib():
    """Load (compiling on first use) the C oracle library."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        L.or_chol_unblocked.argtypes = [ctypes.c_int, dp, ctypes.c_long]
        L.or_chol_unblocked.restype = ctypes.c_int
        for name in ("or_chol_unblocked_fwd", "or_chol_unblocked_rev"):
            f = getattr(L, name)
            f.argtypes = [ctypes.c_int, dp, ctypes.c_long, dp, ctypes.c_long]
            f.restype = None
        for name in ("or_chol_symbolic_fwd", "or_chol_symbolic_rev"):
            f = getattr(L, name)
            f.argtypes = [ctypes.c_int, dp, ctypes.c_long, dp, ctypes.c_long]
            f.restype = ctypes.c_int
        L.or_chol_unblocked_and_fwd.argtypes = [ctypes.c_int, dp, ctypes.c_long, dp, ctypes.c_long]
        L.or_chol_unblocked_and_fwd.restype = ctypes.c_int
        L.or_num_threads.restype = ctypes.c_int
        L.or_set_num_threads.argtypes = [ctypes.c_int]
        _lib = L
    return _lib


def num_threads() -> int:
    return int(lib().or_num_threads())


def set_num_threads(t: int) -> None:
    lib().or_set_num_threads(int(t))


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _square(a, name):
    if a.ndim != 2 or a.shape[0] != a.shape[1]:
        raise ValueError(f"{name} must be square, got shape {a.shape}")
    return a.shape[0]


# --------------------------------------------------------------------------
# Definitions (Sec. 3 and Sec. 4.1)
# --------------------------------------------------------------------------

def tril(a):
    """Eq. tril: keep i >= j."""
    return np.tril(a)


def phi(a):
    """Eq. phi: lower triangle with the diagonal halved."""
    out = np.tril(np.array(a, dtype=np.float64, copy=True))
    out[np.diag_indices_from(out)] *= 0.5
    return out


def chol_unblocked(sigma):
    """Sec. 4.1 chol_unblocked (DPOTF2) on tril(sigma).

    Returns (L, info): info = 0 on success, else the 1-based column of the
    first non-positive pivot (L is then only meaningful left of it).
    """
    a = _f64(sigma).copy()
    n = _square(a, "sigma")
    info = lib().or_chol_unblocked(n, _ptr(a), n)
    return np.tril(a), int(info)


def chol_unblocked_fwd(L, sigma_dot):
    """Sec. 4.1 chol_unblocked_fwd (Eqs. dub1, dub2): L_dot from tril(Sigma_dot)."""
    L = _f64(L)
    a = _f64(sigma_dot).copy()
    n = _square(a, "sigma_dot")
    lib().or_chol_unblocked_fwd(n, _ptr(L), L.shape[1], _ptr(a), n)
    return np.tril(a)


def chol_unblocked_and_fwd(sigma, sigma_dot):
    """Sec. 4.1: chol_unblocked with the updates of chol_unblocked_fwd placed
    in the same loop.  Returns (L, L_dot, info), info as chol_unblocked."""
    a = _f64(sigma).copy()
    ad = _f64(sigma_dot).copy()
    n = _square(a, "sigma")
    if ad.shape != a.shape:
        raise ValueError("sigma_dot must match sigma")
    info = lib().or_chol_unblocked_and_fwd(n, _ptr(a), n, _ptr(ad), n)
    return np.tril(a), np.tril(ad), int(info)


def chol_unblocked_rev(L, L_bar):
    """Sec. 4.1 chol_unblocked_rev: tril(Sigma_bar) from L_bar."""
    L = _f64(L)
    a = _f64(L_bar).copy()
    n = _square(a, "L_bar")
    lib().or_chol_unblocked_rev(n, _ptr(L), L.shape[1], _ptr(a), n)
    return np.tril(a)


def chol_symbolic_fwd(L, sigma_dot):
    """Eq. symfwd: L_dot = L Phi(L^{-1} Sigma_dot L^{-T}), by substitution."""
    L = _f64(L)
    a = _f64(sigma_dot).copy()
    n = _square(a, "sigma_dot")
    rc = lib().or_chol_symbolic_fwd(n, _ptr(L), L.shape[1], _ptr(a), n)
    if rc != 0:
        raise MemoryError("oracle work array")
    return np.tril(a)


def chol_symbolic_rev(L, L_bar):
    """Eq. symrevtril: tril(Sigma_bar) = Phi(L^{-T}(P + P^T)L^{-1}), P = Phi(L^T L_bar)."""
    L = _f64(L)
    a = _f64(L_bar).copy()
    n = _square(a, "L_bar")
    rc = lib().or_chol_symbolic_rev(n, _ptr(L), L.shape[1], _ptr(a), n)
    if rc != 0:
        raise MemoryError("oracle work array")
    return np.tril(a)


def sym_from_tril(t):
    """Eq. symrev's full symmetric Sigma_bar = S + S^T - diag(S) from tril(Sigma_bar).

    tril(Sigma_bar) holds the off-diagonal entries of S + S^T and, on the
    diagonal, S_ii; mirroring the strict lower triangle gives Eq. symrev.
    """
    t = np.tril(t)
    return t + np.tril(t, -1).T


# --------------------------------------------------------------------------
# Explicit derivatives (Eq. delements), for tiny n only: Theta(n^5) here.
# --------------------------------------------------------------------------

def dchol_jacobian(L):
    """J[i, j, k, l] = d L_ij / d Sigma_kl for i >= j, k >= l (Eq. delements).

    Sigma_kl and Sigma_lk are one tied input (k != l).  L^{-1} comes from a
    library inverse, a primitive step of the formula.
    """
    L = np.tril(_f64(L))
    n = L.shape[0]
    Li = np.linalg.inv(L)
    J = np.zeros((n, n, n, n))
    for i in range(n):
        for j in range(i + 1):
            for k in range(n):
                for l in range(k + 1):
                    t1 = sum(L[i, m] * Li[m, k] for m in range(j + 1, n)) + 0.5 * L[i, j] * Li[j, k]
                    val = t1 * Li[j, l]
                    if k != l:
                        t2 = sum(L[i, m] * Li[m, l] for m in range(j + 1, n)) + 0.5 * L[i, j] * Li[j, l]
                        val += t2 * Li[j, k]
                    J[i, j, k, l] = val
    return J


# --------------------------------------------------------------------------
# Error measure shared by tests and the benchmark report
# --------------------------------------------------------------------------

def rel_fro(x, ref):
    """||tril(x - ref)||_F / ||tril(ref)||_F (lower triangles only)."""
    x = np.tril(np.asarray(x, dtype=np.float64))
    ref = np.tril(np.asarray(ref, dtype=np.float64))
    den = np.linalg.norm(ref)
    num = np.linalg.norm(x - ref)
    return float(num / den) if den > 0 else float(num)


# --------------------------------------------------------------------------
# Gaussian-process negative log marginal likelihood (differentiation demo)
# --------------------------------------------------------------------------

def _forward_subst(L, b):
    """Solve L x = b for lower L (plain row loop)."""
    n = L.shape[0]
    x = np.zeros(n)
    for i in range(n):
        x[i] = (b[i] - L[i, :i] @ x[:i]) / L[i, i]
    return x


def _back_subst_t(L, b):
    """Solve L^T x = b for lower L (plain row loop, last row first)."""
    n = L.shape[0]
    x = np.zeros(n)
    for i in range(n - 1, -1, -1):
        x[i] = (b[i] - L[i + 1:, i] @ x[i + 1:]) / L[i, i]
    return x


def rbf_sqdist(X):
    X = _f64(X)
    sq = (X * X).sum(1)
    r2 = sq[:, None] + sq[None, :] - 2.0 * (X @ X.T)
    np.maximum(r2, 0.0, out=r2)
    r2[np.diag_indices_from(r2)] = 0.0
    return r2


def gp_sigma(theta, X):
    """Sigma(theta) = s^2 exp(-r^2 / (2 l^2)) + sigma^2 I, theta = (s, l, sigma)."""
    s, ell, sig = (float(t) for t in theta)
    r2 = rbf_sqdist(X)
    return s * s * np.exp(-r2 / (2.0 * ell * ell)) + sig * sig * np.eye(len(r2))


def gp_dsigma(theta, X):
    """Analytic dSigma/dtheta for theta = (s, l, sigma), three n x n matrices."""
    s, ell, sig = (float(t) for t in theta)
    r2 = rbf_sqdist(X)
    K = np.exp(-r2 / (2.0 * ell * ell))
    return [2.0 * s * K, s * s * K * r2 / ell ** 3, 2.0 * sig * np.eye(len(r2))]


def gp_nlml(theta, X, y):
    """0.5 y^T Sigma^{-1} y + sum_i log L_ii, built on the oracle Cholesky."""
    L, info = chol_unblocked(gp_sigma(theta, X))
    if info:
        raise np.linalg.LinAlgError(f"not positive definite at column {info}")
    v = _forward_subst(L, _f64(y))
    return 0.5 * float(v @ v) + float(np.log(np.diag(L)).sum())


def gp_nlml_grad(theta, X, y):
    """d NLML / d theta through reverse mode (Sec. 2):
    L_bar = -tril(beta v^T) + diag(1/L_ii) with v = L^{-1} y, beta = L^{-T} v;
    tril(Sigma_bar) = chol_unblocked_rev(L, L_bar);
    dNLML/dtheta_t = sum_{i >= j} Sigma_bar_ij (dSigma/dtheta_t)_ij.
    """
    L, info = chol_unblocked(gp_sigma(theta, X))
    if info:
        raise np.linalg.LinAlgError(f"not positive definite at column {info}")
    y = _f64(y)
    v = _forward_subst(L, y)
    beta = _back_subst_t(L, v)
    Lbar = -np.tril(np.outer(beta, v))
    Lbar[np.diag_indices_from(Lbar)] += 1.0 / np.diag(L)
    Sbar = chol_unblocked_rev(L, Lbar)
    return np.array([float((Sbar * np.tril(dS)).sum()) for dS in gp_dsigma(theta, X)])


# --------------------------------------------------------------------------
# Column residuals of the defining equations: O(n^2) per column, so they pin
# results at sizes where the full oracle would take minutes.
# --------------------------------------------------------------------------

def fwd_residual_columns(sigma, L, cols):
    """max_q ||(L L^T)[:, q] - Sigma[:, q]|| / ||Sigma[:, q]|| over the given columns (Sec. 1: Sigma = L L^T)."""
    L = np.tril(_f64(L))
    S = np.tril(_f64(sigma))
    S = S + np.tril(S, -1).T
    out = 0.0
    for q in cols:
        r = L @ L[q, :] - S[:, q]
        out = max(out, float(np.linalg.norm(r) / np.linalg.norm(S[:, q])))
    return out


def sens_residual_columns(sigma_dot, L, L_dot, cols):
    """Eq. symfwd implies L_dot L^T + L L_dot^T = Sigma_dot: max over columns of
    ||residual|| / (||L_dot|| ||L[q, :]|| + ||L|| ||L_dot[q, :]||)."""
    L = np.tril(_f64(L))
    Ld = np.tril(_f64(L_dot))
    Sd = np.tril(_f64(sigma_dot))
    Sd = Sd + np.tril(Sd, -1).T
    nL, nLd = np.linalg.norm(L), np.linalg.norm(Ld)
    out = 0.0
    for q in cols:
        r = Ld @ L[q, :] + L @ Ld[q, :] - Sd[:, q]
        scale = nLd * np.linalg.norm(L[q, :]) + nL * np.linalg.norm(Ld[q, :])
        out = max(out, float(np.linalg.norm(r) / scale))
    return out


def rev_residual_columns(L, L_bar, T, cols):
    """Eq. symrevtril implies L^T (T + T^T) L = P + P^T with P = Phi(L^T L_bar),
    T = tril(Sigma_bar): max over columns of ||residual|| / (||L|| ||(T + T^T) L[:, q]||)."""
    L = np.tril(_f64(L))
    Lb = np.tril(_f64(L_bar))
    T = np.tril(_f64(T))
    nL = np.linalg.norm(L)
    out = 0.0
    for q in cols:
        v = L[:, q]
        u = T @ v + T.T @ v
        lhs = L.T @ u
        colP = L.T @ Lb[:, q]            # column q of L^T L_bar
        colP[:q] = 0.0
        colP[q] *= 0.5
        rowP = L[:, q] @ Lb              # row q of L^T L_bar
        rowP[q + 1:] = 0.0
        rowP[q] *= 0.5
        rhs = colP + rowP
        out = max(out, float(np.linalg.norm(lhs - rhs) / (nL * np.linalg.norm(u))))
    return out


def flops_rev(n: int) -> float:
    """Nominal flop count of one reverse pass, 2 n^3 / 3 (leading term)."""
    return 2.0 * n ** 3 / 3.0


__all__ = [
    "lib", "num_threads", "set_num_threads", "tril", "phi",
    "chol_unblocked", "chol_unblocked_fwd", "chol_unblocked_rev",
    "chol_symbolic_fwd", "chol_symbolic_rev", "sym_from_tril",
    "dchol_jacobian", "rel_fro", "gp_sigma", "gp_dsigma", "gp_nlml",
    "gp_nlml_grad", "rbf_sqdist", "flops_rev", "fwd_residual_columns", "sens_residual_columns",
    "rev_residual_columns",
]
