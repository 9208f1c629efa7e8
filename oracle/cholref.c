/*
 * cholref.c -- plain FP64 CPU oracle for the Cholesky derivative routines of
 * Murray, "Differentiation of the Cholesky decomposition" (arXiv:1602.07527).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the tests, the smoke check and the benchmark's CPU
 * baseline leg use it.  It shares no code, header or constant with the CUDA
 * library; it is deliberately slow and written to be checked against the
 * paper by eye.
 *
 * Conventions (all functions):
 *   - matrices are dense, row-major, element (i, j) at M[i*ld + j], FP64;
 *   - only the lower triangle (i >= j) of every input is read, and only the
 *     lower triangle of every output is written (the paper's tril, Sec. 4.1);
 *   - indices are 0-based; the paper's 1-based loop "j = 1 to N" is j = 0..n-1.
 *
 * Compile with -O2 -ffp-contract=off (no fused multiply-add, no fast-math),
 * so that every operation is one IEEE-754 double rounding.  OpenMP, when
 * enabled, only splits independent rows or columns of one step across
 * threads; it never changes the order of any sum.
 *
 * Pins (see tests/test_oracle_pins.py): LAPACK agreement and L L^T = Sigma for
 * or_chol_unblocked; the one-loop factorisation-and-sensitivity routine
 * against finite differences of the factorisation and against the two
 * routines run one after the other; the two forward-sensitivity routes against each other and
 * against central finite differences; the two reverse routes against each
 * other, against brute-force finite-difference Jacobians (N <= 6), against the
 * explicit element formula (Eq. delements), against the diagonal-Sigma closed
 * form, and through the adjoint identity <Lbar, Ldot> = <tril Sigmabar, Sigmadot>.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define AT(M, ld, i, j) ((M)[(long)(i) * (long)(ld) + (long)(j)])

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void or_set_num_threads(int t) {
#ifdef _OPENMP
  if (t > 0) omp_set_num_threads(t);
#else
  (void)t;
#endif
}

/* ------------------------------------------------------------------------- */
/* Level-2 routines (Sec. 4.1).  For column j the paper's level2partition     */
/* names: r = A[j, 0:j], d = A[j, j], B = A[j+1:n, 0:j], c = A[j+1:n, j].     */
/* ------------------------------------------------------------------------- */

/*
 * chol_unblocked (Sec. 4.1, LAPACK DPOTF2): for j = 0..n-1,
 *     d <- sqrt(d - r r^T),   c <- (c - B r^T) / d.
 * In place on tril(A).  Returns 0, or j+1 (1-based, as LAPACK's info) for the
 * first column whose pivot d - r r^T is not positive; columns from j on are
 * then left unspecified.
 */
int or_chol_unblocked(int n, double *A, long lda) {
  for (int j = 0; j < n; ++j) {
    double piv = AT(A, lda, j, j);
    for (int k = 0; k < j; ++k) piv -= AT(A, lda, j, k) * AT(A, lda, j, k);
    if (!(piv > 0.0)) return j + 1;
    const double d = sqrt(piv);
    AT(A, lda, j, j) = d;
#pragma omp parallel for schedule(static)
    for (int i = j + 1; i < n; ++i) {
      double c = AT(A, lda, i, j);
      for (int k = 0; k < j; ++k) c -= AT(A, lda, i, k) * AT(A, lda, j, k);
      AT(A, lda, i, j) = c / d;
    }
  }
  return 0;
}

/*
 * chol_unblocked_fwd (Sec. 4.1, Eqs. dub1 and dub2): given L and
 * tril(Adot) = tril(Sigma_dot), for j = 0..n-1,
 *     d_dot <- (d_dot/2 - r r_dot^T) / d,
 *     c_dot <- (c_dot - B_dot r^T - B r_dot^T - c d_dot) / d,
 * leaving tril(Adot) = L_dot.  Columns left of j of Adot already hold L_dot.
 */
void or_chol_unblocked_fwd(int n, const double *L, long ldl, double *Ad, long lda) {
  for (int j = 0; j < n; ++j) {
    const double d = AT(L, ldl, j, j);
    double dd = AT(Ad, lda, j, j) / 2.0;
    for (int k = 0; k < j; ++k) dd -= AT(L, ldl, j, k) * AT(Ad, lda, j, k);
    dd = dd / d;
    AT(Ad, lda, j, j) = dd;
#pragma omp parallel for schedule(static)
    for (int i = j + 1; i < n; ++i) {
      double c = AT(Ad, lda, i, j);
      for (int k = 0; k < j; ++k) c -= AT(Ad, lda, i, k) * AT(L, ldl, j, k); /* B_dot r^T */
      for (int k = 0; k < j; ++k) c -= AT(L, ldl, i, k) * AT(Ad, lda, j, k); /* B r_dot^T */
      c -= AT(L, ldl, i, j) * dd;                                            /* c d_dot   */
      AT(Ad, lda, i, j) = c / d;
    }
  }
}

/*
 * chol_unblocked with its forward sensitivity accumulated in the same loop
 * (Sec. 4.1: the updates of chol_unblocked_fwd may follow the matching
 * updates of chol_unblocked).  For j = 0..n-1, column j of L is formed as in
 * or_chol_unblocked, then column j of L_dot as in or_chol_unblocked_fwd; the
 * latter reads only columns 0..j of L, all final by then.  tril(A) holds
 * tril(Sigma) on entry and L on exit; tril(Ad) holds tril(Sigma_dot) on entry
 * and L_dot on exit.  Returns 0 or, as or_chol_unblocked, the 1-based column
 * of the first non-positive pivot (both outputs unspecified from there on).
 */
int or_chol_unblocked_and_fwd(int n, double *A, long lda, double *Ad, long ldad) {
  for (int j = 0; j < n; ++j) {
    /* column j of L */
    double piv = AT(A, lda, j, j);
    for (int k = 0; k < j; ++k) piv -= AT(A, lda, j, k) * AT(A, lda, j, k);
    if (!(piv > 0.0)) return j + 1;
    const double d = sqrt(piv);
    AT(A, lda, j, j) = d;
#pragma omp parallel for schedule(static)
    for (int i = j + 1; i < n; ++i) {
      double ci = AT(A, lda, i, j);
      for (int k = 0; k < j; ++k) ci -= AT(A, lda, i, k) * AT(A, lda, j, k); /* B r^T */
      AT(A, lda, i, j) = ci / d;
    }
    /* column j of L_dot */
    double dd = AT(Ad, ldad, j, j) / 2.0;
    for (int k = 0; k < j; ++k) dd -= AT(A, lda, j, k) * AT(Ad, ldad, j, k);
    dd = dd / d;
    AT(Ad, ldad, j, j) = dd;
#pragma omp parallel for schedule(static)
    for (int i = j + 1; i < n; ++i) {
      double cdi = AT(Ad, ldad, i, j);
      for (int k = 0; k < j; ++k) cdi -= AT(Ad, ldad, i, k) * AT(A, lda, j, k); /* B_dot r^T */
      for (int k = 0; k < j; ++k) cdi -= AT(A, lda, i, k) * AT(Ad, ldad, j, k); /* B r_dot^T */
      cdi -= AT(A, lda, i, j) * dd;                                             /* c d_dot   */
      AT(Ad, ldad, i, j) = cdi / d;
    }
  }
  return 0;
}

/*
 * chol_unblocked_rev (Sec. 4.1, reverse-mode algorithm): given L and
 * tril(Abar) = L_bar, for j = n-1 down to 0,
 *     d_bar <- d_bar - c^T c_bar / d,
 *     [d_bar; c_bar] <- [d_bar; c_bar] / d,
 *     r_bar <- r_bar - [d_bar  c_bar^T] [r; B]   (= r_bar - d_bar r - c_bar^T B),
 *     B_bar <- B_bar - c_bar r,
 *     d_bar <- d_bar / 2,
 * leaving tril(Abar) = tril(Sigma_bar).
 */
void or_chol_unblocked_rev(int n, const double *L, long ldl, double *Ab, long lda) {
  for (int j = n - 1; j >= 0; --j) {
    const double d = AT(L, ldl, j, j);
    double ctc = 0.0;
    for (int i = j + 1; i < n; ++i) ctc += AT(L, ldl, i, j) * AT(Ab, lda, i, j);
    double db = AT(Ab, lda, j, j) - ctc / d;
    db = db / d;
    for (int i = j + 1; i < n; ++i) AT(Ab, lda, i, j) = AT(Ab, lda, i, j) / d;
    /* r_bar <- r_bar - d_bar r - c_bar^T B: each k is independent. */
#pragma omp parallel for schedule(static)
    for (int k = 0; k < j; ++k) {
      double rb = AT(Ab, lda, j, k) - db * AT(L, ldl, j, k);
      for (int i = j + 1; i < n; ++i) rb -= AT(Ab, lda, i, j) * AT(L, ldl, i, k);
      AT(Ab, lda, j, k) = rb;
    }
    /* B_bar <- B_bar - c_bar r: each row i is independent. */
#pragma omp parallel for schedule(static)
    for (int i = j + 1; i < n; ++i) {
      const double cb = AT(Ab, lda, i, j);
      for (int k = 0; k < j; ++k) AT(Ab, lda, i, k) -= cb * AT(L, ldl, j, k);
    }
    AT(Ab, lda, j, j) = db / 2.0;
  }
}

/* ------------------------------------------------------------------------- */
/* Symbolic routines (Sec. 3).  Inverses are never formed: L^{-1} X is found  */
/* by forward substitution and L^{-T} X by back substitution, column by       */
/* column, on full n x n work arrays.                                         */
/* ------------------------------------------------------------------------- */

/* X <- L^{-1} X (X full n x n, row-major, ld n): forward substitution per column. */
static void lower_solve_left(int n, const double *L, long ldl, double *X) {
#pragma omp parallel for schedule(static)
  for (int col = 0; col < n; ++col) {
    for (int i = 0; i < n; ++i) {
      double s = X[(long)i * n + col];
      for (int k = 0; k < i; ++k) s -= AT(L, ldl, i, k) * X[(long)k * n + col];
      X[(long)i * n + col] = s / AT(L, ldl, i, i);
    }
  }
}

/* X <- L^{-T} X (X full n x n): back substitution with the upper matrix L^T. */
static void lower_t_solve_left(int n, const double *L, long ldl, double *X) {
#pragma omp parallel for schedule(static)
  for (int col = 0; col < n; ++col) {
    for (int i = n - 1; i >= 0; --i) {
      double s = X[(long)i * n + col];
      for (int k = i + 1; k < n; ++k) s -= AT(L, ldl, k, i) * X[(long)k * n + col];
      X[(long)i * n + col] = s / AT(L, ldl, i, i);
    }
  }
}

static void transpose_inplace(int n, double *X) {
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) {
      double t = X[(long)i * n + j];
      X[(long)i * n + j] = X[(long)j * n + i];
      X[(long)j * n + i] = t;
    }
}

/* Phi (Eq. phi): keep the lower triangle, halve the diagonal, zero the rest. */
static void phi_inplace(int n, double *X) {
  for (int i = 0; i < n; ++i) {
    for (int j = i + 1; j < n; ++j) X[(long)i * n + j] = 0.0;
    X[(long)i * n + i] *= 0.5;
  }
}

/*
 * Symbolic forward mode (Eq. symfwd): L_dot = L Phi(L^{-1} Sigma_dot L^{-T}).
 * Sigma_dot is symmetric and given by its lower triangle in Ad; the result
 * overwrites tril(Ad).  Returns 0, or -2 if a work array cannot be allocated.
 */
int or_chol_symbolic_fwd(int n, const double *L, long ldl, double *Ad, long lda) {
  if (n <= 0) return 0;
  double *X = (double *)malloc(sizeof(double) * (size_t)n * (size_t)n);
  if (!X) return -2;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      X[(long)i * n + j] = (i >= j) ? AT(Ad, lda, i, j) : AT(Ad, lda, j, i);
  lower_solve_left(n, L, ldl, X);   /* L^{-1} Sigma_dot               */
  transpose_inplace(n, X);          /* (L^{-1} Sigma_dot)^T            */
  lower_solve_left(n, L, ldl, X);   /* L^{-1} Sigma_dot L^{-T} (symm.) */
  phi_inplace(n, X);
  /* L_dot = L Phi(.) : lower times lower is lower. */
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n; ++i)
    for (int j = 0; j <= i; ++j) {
      double s = 0.0;
      for (int k = j; k <= i; ++k) s += AT(L, ldl, i, k) * X[(long)k * n + j];
      AT(Ad, lda, i, j) = s;
    }
  free(X);
  return 0;
}

/*
 * Symbolic reverse mode, lower-triangular form (Eq. symrevtril):
 *     tril(Sigma_bar) = Phi(L^{-T} (P + P^T) L^{-1}),   P = Phi(L^T L_bar).
 * L_bar is tril(Ab); the result overwrites tril(Ab).
 * Returns 0, or -2 if a work array cannot be allocated.
 */
int or_chol_symbolic_rev(int n, const double *L, long ldl, double *Ab, long lda) {
  if (n <= 0) return 0;
  double *X = (double *)malloc(sizeof(double) * (size_t)n * (size_t)n);
  if (!X) return -2;
  /* P = Phi(L^T L_bar), both factors lower triangular. */
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int k = (i > j ? i : j); k < n; ++k) s += AT(L, ldl, k, i) * AT(Ab, lda, k, j);
      X[(long)i * n + j] = s;
    }
  phi_inplace(n, X);
  /* M = P + P^T (full symmetric). */
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < i; ++j) X[(long)j * n + i] = X[(long)i * n + j];
  for (int i = 0; i < n; ++i) X[(long)i * n + i] *= 2.0;
  lower_t_solve_left(n, L, ldl, X); /* L^{-T} M          */
  transpose_inplace(n, X);          /* (L^{-T} M)^T = M L^{-1}, M symmetric */
  lower_t_solve_left(n, L, ldl, X); /* L^{-T} M L^{-1}  */
  phi_inplace(n, X);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j <= i; ++j) AT(Ab, lda, i, j) = X[(long)i * n + j];
  free(X);
  return 0;
}
