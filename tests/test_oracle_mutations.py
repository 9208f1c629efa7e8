"""The oracle's pins must catch plausible mistakes.  Each case plants one
mistake in a temporary copy of the oracle's C source (never in the committed
file), compiles it, and checks that an independent pin -- the exact Jacobian
of Eq. delements, a library Cholesky, or the adjoint identity -- rejects it.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_1602_07527_gb300 import workloads as W

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "cholref.c")

# (routine, exact text in cholref.c, planted replacement)
MUTATIONS = [
    ("rev", "AT(Ab, lda, j, j) = db / 2.0;", "AT(Ab, lda, j, j) = db;"),                  # halving dropped
    ("rev", "double db = AT(Ab, lda, j, j) - ctc / d;", "double db = AT(Ab, lda, j, j) + ctc / d;"),  # sign
    ("rev", "rb -= AT(Ab, lda, i, j) * AT(L, ldl, i, k);", "rb -= AT(Ab, lda, i, j) * AT(L, ldl, i, j);"),  # index
    ("rev", "AT(Ab, lda, i, k) -= cb * AT(L, ldl, j, k);", "AT(Ab, lda, i, k) -= cb * AT(L, ldl, i, k);"),  # B_bar term
    ("rev", "double rb = AT(Ab, lda, j, k) - db * AT(L, ldl, j, k);", "double rb = AT(Ab, lda, j, k);"),  # d_bar r dropped
    ("fwd_sens", "c -= AT(L, ldl, i, j) * dd;", ""),                                       # c d_dot dropped
    ("fwd_sens", "double dd = AT(Ad, lda, j, j) / 2.0;", "double dd = AT(Ad, lda, j, j);"),  # halving dropped
    ("fwd_sens", "c -= AT(L, ldl, i, k) * AT(Ad, lda, j, k); /* B r_dot^T */", ""),          # B r_dot^T dropped
    ("chol", "c -= AT(A, lda, i, k) * AT(A, lda, j, k);", "c -= AT(A, lda, i, k) * AT(A, lda, i, k);"),
    ("fused", "cdi -= AT(A, lda, i, j) * dd;", ""),                                        # c d_dot dropped
    ("fused", "double dd = AT(Ad, ldad, j, j) / 2.0;", "double dd = AT(Ad, ldad, j, j);"),  # halving dropped
    ("fused", "ci -= AT(A, lda, i, k) * AT(A, lda, j, k); /* B r^T */",
              "ci -= AT(A, lda, i, k) * AT(A, lda, i, k); /* B r^T */"),                     # index in L part
    ("fused", "cdi -= AT(Ad, ldad, i, k) * AT(A, lda, j, k); /* B_dot r^T */",
              "cdi += AT(Ad, ldad, i, k) * AT(A, lda, j, k); /* B_dot r^T */"),              # sign
    ("symrev", "for (int i = 0; i < n; ++i) X[(long)i * n + i] *= 2.0;", ""),                # P + P^T diagonal
    ("symrev", "phi_inplace(n, X);\n  /* M = P + P^T (full symmetric). */", "/* M = P + P^T (full symmetric). */"),
    ("symfwd", "for (int k = j; k <= i; ++k) s += AT(L, ldl, i, k) * X[(long)k * n + j];",
               "for (int k = j; k < i; ++k) s += AT(L, ldl, i, k) * X[(long)k * n + j];"),
]


def _build_mutant(tmp_path, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor not unique/present: {old!r}"
    path = tmp_path / "mut.c"
    path.write_text(src.replace(old, new))
    lib = tmp_path / "libmut.so"
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11",
                    str(path), "-o", str(lib), "-lm"], check=True, capture_output=True)
    L = ctypes.CDLL(str(lib))
    dp = ctypes.POINTER(ctypes.c_double)
    for name in ("or_chol_unblocked_fwd", "or_chol_unblocked_rev",
                 "or_chol_symbolic_fwd", "or_chol_symbolic_rev"):
        getattr(L, name).argtypes = [ctypes.c_int, dp, ctypes.c_long, dp, ctypes.c_long]
    L.or_chol_unblocked.argtypes = [ctypes.c_int, dp, ctypes.c_long]
    L.or_chol_unblocked.restype = ctypes.c_int
    L.or_chol_unblocked_and_fwd.argtypes = [ctypes.c_int, dp, ctypes.c_long, dp, ctypes.c_long]
    L.or_chol_unblocked_and_fwd.restype = ctypes.c_int
    return L


def _call(lib, name, L, X):
    n = X.shape[0]
    a = np.ascontiguousarray(X, dtype=np.float64).copy()
    dp = ctypes.POINTER(ctypes.c_double)
    if L is None:
        getattr(lib, name)(n, a.ctypes.data_as(dp), n)
    else:
        Lc = np.ascontiguousarray(L)
        getattr(lib, name)(n, Lc.ctypes.data_as(dp), n, a.ctypes.data_as(dp), n)
    return np.tril(a)


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
@pytest.mark.parametrize("routine,old,new", MUTATIONS)
def test_pins_catch_planted_mistake(oracle, tmp_path, routine, old, new):
    n = 6
    S = W.wishart(n, 21)
    L = np.linalg.cholesky(S)
    J = oracle.dchol_jacobian(L)            # Eq. delements, independent of cholref.c
    Lb = W.lbar(n, 21)
    Sd = W.sigma_dot(n, 21)
    mut = _build_mutant(tmp_path, old, new)
    if routine == "fused":
        a = np.ascontiguousarray(S).copy()
        ad = np.ascontiguousarray(Sd).copy()
        dp = ctypes.POINTER(ctypes.c_double)
        mut.or_chol_unblocked_and_fwd(n, a.ctypes.data_as(dp), n, ad.ctypes.data_as(dp), n)
        ref = np.einsum("ijkl,kl->ij", J, np.tril(Sd))
        assert (not np.allclose(np.tril(a), L, rtol=1e-10, atol=1e-12)
                or oracle.rel_fro(np.tril(ad), ref) > 1e-6)
    elif routine == "chol":
        got = _call(mut, "or_chol_unblocked", None, S)
        assert not np.allclose(got, L, rtol=1e-10, atol=1e-12)
    elif routine in ("rev", "symrev"):
        name = "or_chol_unblocked_rev" if routine == "rev" else "or_chol_symbolic_rev"
        got = _call(mut, name, L, Lb)
        ref = np.tril(np.einsum("ij,ijkl->kl", Lb, J))
        lhs = float((Lb * np.einsum("ijkl,kl->ij", J, np.tril(Sd))).sum())
        rhs = float((got * np.tril(Sd)).sum())
        assert oracle.rel_fro(got, ref) > 1e-6 or abs(lhs - rhs) > 1e-9
    else:
        name = "or_chol_unblocked_fwd" if routine == "fwd_sens" else "or_chol_symbolic_fwd"
        got = _call(mut, name, L, Sd)
        ref = np.einsum("ijkl,kl->ij", J, np.tril(Sd))
        assert oracle.rel_fro(got, ref) > 1e-6
