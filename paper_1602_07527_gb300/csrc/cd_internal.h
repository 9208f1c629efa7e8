// Internal declarations shared by the libcholdiff CUDA translation units.
// Not installed; the public interface is include/libcholdiff.h.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/libcholdiff.h"

namespace cd {

// ---------------------------------------------------------------------------
// Grouped FP64 GEMM: Cout = beta * Cin + alpha * op(A) op(B), for up to
// kMaxGemm independent problems per launch (batched work shares one grid).
// ---------------------------------------------------------------------------
enum AMode { A_N = 0, A_T = 1, A_SYM2 = 2, A_TL = 3, A_SYM1 = 4, A_NL = 5 };
// A_N   : a(i,k) = A[i*lda + k]
// A_T   : a(i,k) = A[k*lda + i]
// A_SYM2: a(i,k) = symmetric view of a lower-stored matrix with doubled
//         diagonal: A[i][k] (i > k), A[k][i] (i < k), 2 A[i][i] (i == k).
//         This is G = X + X^T for X = tril(A), used by the reverse pass.
// A_TL  : a(i,k) = A[k][i] if k >= i else 0   (transpose of a lower matrix)
// A_SYM1: a(i,k) = A[i][k] (i >= k), A[k][i] (i < k): symmetric view of a lower-stored matrix
// A_NL  : a(i,k) = A[i][k] if i >= k else 0   (lower matrix, upper storage ignored)
enum BMode { B_N = 0, B_T = 1, B_TL = 2, B_NL = 3 };
// B_N   : b(k,j) = B[k*ldb + j]
// B_T   : b(k,j) = B[j*ldb + k]
// B_TL  : b(k,j) = B[j*ldb + k] if j >= k else 0   (transpose of a lower matrix)
// B_NL  : b(k,j) = B[k*ldb + j] if k >= j else 0   (lower matrix, upper storage ignored)

struct GemmDesc {
  const double *A, *B, *Cin;
  double *Cout, *part;
  long long lda, ldb, ldcin, ldcout;
  double alpha, beta;
  int M, N, K, splits;
  int tiles_m, tiles_n, tile_begin, kchunk;
};

// Triangular operands (GemmGroup::tri): a product term a(i,k) b(k,j) known to
// be zero over part of K lets each output tile skip those K blocks exactly.
enum TriMask {
  TRI_A_UPPER = 1,  // a(i,k) = 0 for k < i
  TRI_A_LOWER = 2,  // a(i,k) = 0 for k > i
  TRI_B_LOWER = 4,  // b(k,j) = 0 for k < j
  TRI_B_UPPER = 8   // b(k,j) = 0 for k > j
};

constexpr int kMaxGemm = 32;
struct GemmGroup {
  int count, total_tiles;
  int amode, bmode, lower, phi;  // phi: halve the diagonal of a lower output (Eq. phi)
  int tri;                       // TriMask bits (0: general operands)
  int ts;                        // output tile size of the launch: 64, or 32 for small products
  GemmDesc d[kMaxGemm];
};
static_assert(sizeof(GemmGroup) <= 4096, "kernel parameter block too large");

// The work items of a 32 x 32-tile launch that contribute anything (tile
// indices of the group's tile list): with triangular operands many K splits
// of a tile are empty; launching only the others spreads the real work
// evenly over the SMs (the empty splits' partial sums are skipped by the
// reduction, which sums each tile's non-empty splits only).
constexpr int kMaxItems = 2048;
struct GemmItems {
  int count, pad_;
  int bid[kMaxItems];
};
// k_gemm_f64_items takes both blocks as __grid_constant__ parameters: above
// the classic 4 KB limit, within the 32764 bytes CUDA 12.1+ allows.
static_assert(sizeof(GemmGroup) + sizeof(GemmItems) <= 32764, "kernel parameter block too large");

// ---------------------------------------------------------------------------
// One-CTA diagonal-tile kernels (t <= kTileMax, tile in shared memory).
// ---------------------------------------------------------------------------
constexpr int kTileMax = 128;

struct TileDesc {
  const double *L;  // factor tile (rev / sens / inverse), lower
  double *X;        // in/out tile
  double *inv;      // output: inverse of the factor tile, t x t full (ld = ldinv)
  int *info;        // potf2: info word of the problem (may be null)
  long long ldl, ldx, ldinv;
  int t, col0;      // tile size; global column of the tile's first column
  // optional (T_POTRF with inv): the inverse also in a tensor-core operand format, slice or term s
  // of (r, c) at fsl + (s frows + r) ldf + c for r, c < frows: fterms = 0, fixed-point slices
  // (cd_fixed_digits.cuh) with the row exponents fex[0, frows); fterms = 2 or 3, that many BF16
  // terms of the split-BF16 products (cd_split_terms.cuh)
  void *fsl;
  int *fex;
  long long ldf;
  int frows, fterms;
};

constexpr int kMaxTile = 48;
struct TileGroup {
  int count, pad_;
  int *err;  // device error word: CD_ETIMEOUT if a bounded wait of the cluster kernel runs out
  TileDesc d[kMaxTile];
};
static_assert(sizeof(TileGroup) <= 32764, "kernel parameter block too large");

// T_REV / T_SENS: the level-2 derivative loops on one CTA.  T_POTRF: the
// diagonal tile on a cluster of CTAs: factorise X in place (info set at the
// first non-positive pivot) and, if inv != null, write the inverse of the
// factor.  T_TRTRI: the same kernel writing only the inverse of the given
// factor L.
enum TileOp { T_REV = 1, T_SENS = 2, T_TRTRI = 3, T_POTRF = 4 };

// Grouped 2-D copies (one launch for the panels of every problem of a step).
struct CopyDesc {
  const double *src;
  double *dst;
  long long lds, ldd;
  int rows, cols;
};
constexpr int kMaxCopy = 96;
struct CopyGroup {
  int count, pad_;
  CopyDesc d[kMaxCopy];
};

// ---------------------------------------------------------------------------
// Mixed-precision (split-BF16 tcgen05) engine: see cd_mixed.cu.
// ---------------------------------------------------------------------------
struct MixedGemm;  // opaque

}  // namespace cd

struct cd_handle {
  int device;
  int num_sms;
  size_t smem_optin;
  void *ws;
  size_t ws_bytes;
  int *dev_err;
  long long launches;
  int prof_on;  // cd_profile_enable
  void *prof;   // profiler state (cd_api.cu)
  int gemm_slots;              // resident FP64 GEMM CTAs on the whole GPU (64 x 64 tiles)
  int gemm_slots_small;        // the same for 32 x 32 tiles
  cudaStream_t side;           // second stream for work independent of the diagonal chain
  cudaStream_t crit;           // high-priority stream for the diagonal (critical) chain
  cudaEvent_t ev_fork, ev_join, ev_in, ev_out;
  cudaEvent_t ev_mid;          // a point inside the side stream's work of a step
  cudaEvent_t ev_look[2];      // lookahead factorisation: side-stream work issued one step early (by parity)
  cudaEvent_t ev_near;         // lookahead factorisation: the current step's side-stream update
  // One-loop mixed pass: the sensitivity steps run one block column behind the factorisation
  // on a chain and a bulk stream of their own, after events of the factorisation's two streams.
  cudaStream_t crit2, side2;
  cudaEvent_t ev_colA, ev_colB, ev_start2;
};

namespace cd {
// Launchers (cd_f64_kernels.cu).  All return cudaError_t of the launch.
cudaError_t launch_gemm_group(const GemmGroup &g, cudaStream_t s);
// A 32 x 32-tile group restricted to the listed work items.
cudaError_t launch_gemm_items(const GemmGroup &g, const GemmItems &it, cudaStream_t s);
cudaError_t launch_reduce_group(const GemmGroup &g, cudaStream_t s);
cudaError_t launch_tile_group(TileOp op, const TileGroup &g, cudaStream_t s);
cudaError_t launch_copy(const double *src, long long lds, double *dst, long long ldd, int rows,
                        int cols, cudaStream_t s);
cudaError_t launch_mirror_lower(double *A, long long lda, int n, cudaStream_t s);
// dst(i, j) = src(j, i): mode 0 lower of dst from upper of src, 1 upper from lower, 2 all.
cudaError_t launch_transpose(const double *src, long long lds, double *dst, long long ldd, int n, int mode,
                             cudaStream_t s);
cudaError_t launch_copy_group(const CopyGroup &g, cudaStream_t s);
// dst -= tril(src + src^T) for square blocks (rows == cols).
cudaError_t launch_subsym_group(const CopyGroup &g, cudaStream_t s);
cudaError_t tile_kernels_init();
// FP64 peak probes: kind 0 DFMA chains, 1 mma.sync m8n8k4 f64; *flops = work launched.
cudaError_t launch_fp64_probe(int kind, int blocks, long long iters, cudaStream_t st, double *flops);
// The diagonal factorisation's FP64 reciprocal and square-root helpers over an array.
cudaError_t launch_fp64_helpers(int n, const double *x, double *recip, double *sq, double *rsq, cudaStream_t st);
// Eq. delements: S (n^3 doubles) then J (n^4 doubles) from L and Linv = L^{-1}.
cudaError_t launch_jacobian(int n, const double *L, long long ldl, const double *Li, long long ldi, double *S,
                            double *J, cudaStream_t s);
int gemm_ctas_per_sm(int ts);  // resident CTAs of the FP64 GEMM per SM (tile size ts)
}  // namespace cd
