// Mixed-precision (split-BF16, tcgen05) engine interface.
//
// FP64 operands are split into T = 2 or 3 BF16 terms, x ~ t0 + t1 (+ t2), each
// term the BF16 nearest to the remainder of the previous ones (formed in FP32
// from an exact two-piece FP32 form of x, so within 2^-24 of the exact
// remainder).  A product is formed as the sum of the term products whose
// order is at most 2^-8 (T = 2: t0 t0, t0 t1, t1 t0) or 2^-16 (T = 3: adds
// t0 t2, t2 t0, t1 t1) relative to the leading one, accumulated in FP32 in
// tensor memory (the leading product apart from the corrections), and added
// to the FP64 output in FP64 (an FP32 sum below 2^-126, subnormal, counts as
// zero).  Split-K partial sums are FP32.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace cd {

// A K-major BF16 term array: term t, row r, column c at
// base + (t * rows + r) * ld + c (elements).  A GEMM operand is the view with
// origin (y0 = row, x0 = column) of such an array; rows index M (or N), columns
// index K.  ld must be a multiple of 64 and x0 a multiple of 8.
struct MOp {
  const void *base;
  long long ld;    // elements per row (multiple of 64)
  long long rows;  // rows per term
  int T;           // terms (2 or 3; 4 fixed-point slices for cd_fixed.cu)
  int x0, y0;      // view origin
  const int *ex;   // fixed-point slices: exponent of each stored row (else unused)
};

// Cout = beta * Cin + alpha * op(A) op(B)^T over the views (M x K) and (N x K).
struct MProblem {
  MOp A, B;
  int M, N, K;
  const double *Cin;
  long long ldcin;
  double *Cout;
  long long ldcout;
  double alpha, beta;
  double *part;  // split-K partials (splits * M * N doubles) when splits > 1
  int splits;    // 1 = write Cout directly
  int kchunk;    // K range of one split, multiple of 64
};

int mixed_init();                                       // CD_OK or a CD_* error
bool mixed_available();                                 // engine built and usable
size_t mixed_workspace_bytes(int n, int nb, int prec);  // extra workspace for one problem
int mixed_ctas_per_sm();                                // resident GEMM CTAs per SM

// Launch one grouped tensor-core GEMM (and its split-K reduction) over
// `count` independent problems of the same term count and output mode.
// dev_err: device word set to CD_ETIMEOUT if a bounded wait runs out.
// tx_extra is a test hook (0 in production): the first load barrier of each
// CTA expects that many bytes more than its copy delivers, so the bounded
// wait of the MMA thread runs out and the kernel reports CD_ETIMEOUT.
// max_units bounds the output tiles one persistent CTA takes: a CTA holds its
// SM until its last tile, so products on the bulk stream take few tiles per
// CTA and hand SMs back to the diagonal chain's launches.
constexpr int kUnitsPerCtaChain = 4;
constexpr int kUnitsPerCtaBulk = 4;
cudaError_t mixed_gemm_launch(const MProblem *probs, int count, int T, bool lower, int *dev_err, cudaStream_t s,
                              int *launches, int tx_extra = 0, int max_units = kUnitsPerCtaChain);

// Split an FP64 view into T BF16 term arrays (see MOp).  The view is
// rows x cols of src (lower-triangle mode 1 keeps r >= c; mode 2 is the
// symmetric view of a lower-stored matrix with doubled diagonal); with
// transpose the destination holds the view's transpose.  The region
// rows [reg_r0, reg_r0 + dst_h) x cols [reg_c0, reg_c0 + dst_w) of every term
// of dst is written; the view's (0, 0) lands at (dst_r0, dst_c0) and region
// elements outside the view are set to zero.
struct SplitArgs {
  const double *src;
  long long lds;
  int rows, cols, mode, transpose;
  void *dst;
  long long ldd, dst_rows;  // term stride = dst_rows * ldd
  int reg_r0, reg_c0, dst_h, dst_w;
  int dst_r0, dst_c0;
  int T;
  int *ex;  // fixed-point splits: exponent of each destination row (cd_fixed.cu)
};
// Independent splits in one launch (count of them).
cudaError_t mixed_split_group_launch(const SplitArgs *a, int count, cudaStream_t s, int *launches);

// Fixed-point-slice products (cd_fixed.cu, CD_MIXED_FIXED4): operands are
// MOp views of 4-slice arrays with per-row exponents (MOp::ex); the leading
// slice products are exact over windows of 512 of K and every window is
// carried exactly in 64 bits, so each output has one FP64 rounding after
// the operands' rounding to 2^-32 of their row maxima (13 slice products).  Split-K
// partials are 64-bit totals (the region holds splits * M * N of them).
int fixed_init();
cudaError_t fixed_gemm_launch(const MProblem *probs, int count, bool lower, int *dev_err, cudaStream_t s,
                              int *launches, int max_units);
// Fixed-point splits (non-transposed views; SplitArgs::T = 4, ex = exponents
// of the destination rows): with compute_exponents each row's exponent is
// first taken from the maximum of its region, otherwise ex is read.
cudaError_t fixed_split_group_launch(const SplitArgs *a, int count, bool compute_exponents, cudaStream_t s,
                                     int *launches);
// ex[i] for the rows of the factor of Sigma (n x n, lds): an exponent E with
// |L_ik| < 2^E, from |L_ik| <= sqrt(Sigma_ii).  Must run before the
// factorisation overwrites Sigma.
cudaError_t fixed_diag_exponents(const double *S, long long lds, int n, int *ex, cudaStream_t s);

}  // namespace cd
