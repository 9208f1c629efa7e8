// FP64 kernels of libcholdiff: the grouped DFMA tile GEMM used for every
// off-diagonal block update of the blocked algorithms (Sec. 4.2), the
// one-CTA diagonal-tile kernels that run the level-2 derivative routines of
// Sec. 4.1 on a tile held in shared memory, and the diagonal-tile
// factorisation and inverse on a thread-block cluster.
//
// On GB300 the FP64 pipe issues about two DFMA per clock per SM (measured:
// 1.19 TFLOP/s for the whole GPU, 8 GFLOP/s on one SM), and DMMA
// (mma.sync f64) is slower still, so the FP64 engine is a register-blocked
// DFMA kernel: its only job is to keep the FP64 pipe of every SM busy.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "cd_internal.h"
#include "cd_fixed_digits.cuh"
#include "cd_split_terms.cuh"

namespace cd {

// ---------------------------------------------------------------------------
// Grouped GEMM
// ---------------------------------------------------------------------------

template <int AM>
__device__ __forceinline__ double load_a(const double *__restrict__ A, long long lda, int i, int k) {
  if (AM == A_N) return A[(long long)i * lda + k];
  if (AM == A_T) return A[(long long)k * lda + i];
  if (AM == A_TL) return k >= i ? A[(long long)k * lda + i] : 0.0;
  if (AM == A_NL) return i >= k ? A[(long long)i * lda + k] : 0.0;
  if (AM == A_SYM1) return i >= k ? A[(long long)i * lda + k] : A[(long long)k * lda + i];
  if (i > k) return A[(long long)i * lda + k];
  if (i < k) return A[(long long)k * lda + i];
  return 2.0 * A[(long long)i * lda + i];
}

template <int BM>
__device__ __forceinline__ double load_b(const double *__restrict__ B, long long ldb, int k, int j) {
  if (BM == B_N) return B[(long long)k * ldb + j];
  if (BM == B_T) return B[(long long)j * ldb + k];
  if (BM == B_NL) return k >= j ? B[(long long)k * ldb + j] : 0.0;
  return (j >= k) ? B[(long long)j * ldb + k] : 0.0;
}

// Threads of a CTA for output tile size TS: 256 for 64 x 64 tiles; 128 (four
// warps, one per sub-partition's FP64 unit) for the 32 x 32 tiles of small
// products.
template <int TS>
__host__ __device__ constexpr int gemm_threads() {
  return TS == 64 ? 256 : 128;
}
// K depth of a staged block: 16, or 8 for 32 x 32 tiles (4 KB of staging, so
// that two such CTAs fit beside a tensor-core product's CTA on one SM).
template <int TS>
__host__ __device__ constexpr int gemm_kblock() {
  return TS == 64 ? 16 : 8;
}

// One CTA computes a TS x TS output tile over its K range; each thread owns an
// RM x 4 micro-tile (rows ty + RT r, columns tx + CT c), so a warp reads few A
// values (broadcast) and consecutive B values per k.  TS = 64 (256 threads,
// 4 x 4) for ordinary products; TS = 32 (128 threads, 2 x 4) for small ones,
// where a 64 x 64 x 16 chunk alone would hold one SM's FP64 unit for ~16 us
// and too few CTAs would share the product's work.  Every FP64 instruction
// holds its sub-partition's FP64 unit for ~64 cycles, so a CTA's latency is
// set by the multiply-adds per warp: four warps halve it against two.
//
// gemm_tile is one such work item (output tile, K split): tile bid of the
// group's tile list, computed by the whole CTA with the given shared-memory
// staging, which is free again when it returns (every use of it ends with a
// CTA barrier).
template <int AM, int BM, bool LOWER, int TS>
__device__ __forceinline__ void gemm_tile(const GemmGroup &g, int bid, double (*As)[TS + 1], double (*Bs)[TS + 1]) {
  constexpr int KB = gemm_kblock<TS>();
  constexpr int NT = gemm_threads<TS>(), CT = TS / 4, RT = NT / CT, RM = TS / RT, LOADS = KB * TS / NT;
  static_assert(RT * RM == TS && LOADS * NT == KB * TS, "tile layout");
  int p = 0;
  while (p + 1 < g.count && bid >= g.d[p + 1].tile_begin) ++p;
  const GemmDesc &d = g.d[p];
  const int M = d.M, N = d.N;
  const int local = bid - d.tile_begin;
  // tril outputs (M == N) enumerate only the tm (tm + 1) / 2 tiles on or below the diagonal
  const int per_split = LOWER ? d.tiles_m * (d.tiles_m + 1) / 2 : d.tiles_m * d.tiles_n;
  const int z = local / per_split;
  const int rem = local - z * per_split;
  int m0, n0;
  if (LOWER) {
    int ti = (int)((sqrtf(8.0f * rem + 1.0f) - 1.0f) * 0.5f);
    while ((ti + 1) * (ti + 2) / 2 <= rem) ++ti;
    while (ti * (ti + 1) / 2 > rem) --ti;
    m0 = ti * TS;
    n0 = (rem - ti * (ti + 1) / 2) * TS;
  } else {
    m0 = (rem / d.tiles_n) * TS;
    n0 = (rem % d.tiles_n) * TS;
  }
  const int kbeg = z * d.kchunk;
  const int kend = min(d.K, kbeg + d.kchunk);
  // K range of this tile: triangular operands are zero outside [klo, khi)
  int klo = kbeg, khi = kend;
  if (g.tri & TRI_A_UPPER) klo = max(klo, m0);
  if (g.tri & TRI_B_LOWER) klo = max(klo, n0);
  if (g.tri & TRI_A_LOWER) khi = min(khi, m0 + TS);
  if (g.tri & TRI_B_UPPER) khi = min(khi, n0 + TS);
  const int kfirst = kbeg + (klo - kbeg) / KB * KB;  // K blocks stay aligned to the split's start
  const double *__restrict__ A = d.A;
  const double *__restrict__ B = d.B;
  const long long lda = d.lda, ldb = d.ldb;

  const int tid = threadIdx.x, tx = tid % CT, ty = tid / CT;
  double acc[RM][4];
#pragma unroll
  for (int r = 0; r < RM; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = 0.0;

  // one K block of the staged operands into the accumulators
  auto compute = [&](const double (*Ab)[TS + 1], const double (*Bb)[TS + 1]) {
#pragma unroll
    for (int kk = 0; kk < KB; ++kk) {
      double a[RM], b[4];
#pragma unroll
      for (int r = 0; r < RM; ++r) a[r] = Ab[kk][ty + RT * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = Bb[kk][tx + CT * c];
#pragma unroll
      for (int r = 0; r < RM; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
    }
  };
  // this thread's share of the K block at k0, from global memory
  double pa[LOADS], pb[LOADS];
  auto gload = [&](int k0) {
#pragma unroll
    for (int r = 0; r < LOADS; ++r) {
      const int e = tid + r * NT;
      int kk, ii;
      if (AM == A_T) { ii = e % TS; kk = e / TS; } else { kk = e % KB; ii = e / KB; }
      const int gi = m0 + ii, gk = k0 + kk;
      pa[r] = (gi < M && gk < khi) ? load_a<AM>(A, lda, gi, gk) : 0.0;
    }
#pragma unroll
    for (int r = 0; r < LOADS; ++r) {
      const int e = tid + r * NT;
      int kk, jj;
      if (BM == B_N) { jj = e % TS; kk = e / TS; } else { kk = e % KB; jj = e / KB; }
      const int gj = n0 + jj, gk = k0 + kk;
      pb[r] = (gj < N && gk < khi) ? load_b<BM>(B, ldb, gk, gj) : 0.0;
    }
  };
  auto sstore = [&](double (*Ab)[TS + 1], double (*Bb)[TS + 1]) {
#pragma unroll
    for (int r = 0; r < LOADS; ++r) {
      const int e = tid + r * NT;
      if (AM == A_T) Ab[e / TS][e % TS] = pa[r]; else Ab[e % KB][e / KB] = pa[r];
    }
#pragma unroll
    for (int r = 0; r < LOADS; ++r) {
      const int e = tid + r * NT;
      if (BM == B_N) Bb[e / TS][e % TS] = pb[r]; else Bb[e % KB][e / KB] = pb[r];
    }
  };
  if (TS == 64) {
    // two staging buffers (As and Bs hold 2 KB rows each): the next block's
    // global loads are in flight during this block's multiply-adds, and one
    // barrier a block separates the buffers' reuse
    int buf = 0;
    if (kfirst < khi) {
      gload(kfirst);
      sstore(As, Bs);
    }
    __syncthreads();
    for (int k0 = kfirst; k0 < khi; k0 += KB) {
      const bool more = k0 + KB < khi;
      if (more) gload(k0 + KB);
      compute(As + buf * KB, Bs + buf * KB);
      if (more) sstore(As + (buf ^ 1) * KB, Bs + (buf ^ 1) * KB);
      __syncthreads();
      buf ^= 1;
    }
  } else {
    for (int k0 = kfirst; k0 < khi; k0 += KB) {
      gload(k0);
      sstore(As, Bs);
      __syncthreads();
      compute(As, Bs);
      __syncthreads();
    }
  }

  const double alpha = d.alpha, beta = d.beta;
#pragma unroll
  for (int r = 0; r < RM; ++r) {
    const int i = m0 + ty + RT * r;
    if (i >= M) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int j = n0 + tx + CT * c;
      if (j >= N || (LOWER && j > i)) continue;
      if (d.splits == 1) {
        double v = alpha * acc[r][c];
        if (LOWER && g.phi && i == j) v *= 0.5;
        if (beta != 0.0) v = fma(beta, d.Cin[(long long)i * d.ldcin + j], v);
        d.Cout[(long long)i * d.ldcout + j] = v;
      } else {
        d.part[(long long)z * M * N + (long long)i * N + j] = alpha * acc[r][c];
      }
    }
  }
}

template <int AM, int BM, bool LOWER, int TS>
__global__ void __launch_bounds__(gemm_threads<TS>(), TS == 32 ? 8 : 1) k_gemm_f64(const __grid_constant__ GemmGroup g) {
  constexpr int kBufs = TS == 64 ? 2 : 1;  // 64 x 64 tiles stage the next K block during this one
  __shared__ double As[kBufs * gemm_kblock<TS>()][TS + 1];
  __shared__ double Bs[kBufs * gemm_kblock<TS>()][TS + 1];
  gemm_tile<AM, BM, LOWER, TS>(g, blockIdx.x, As, Bs);
}

// The same for the listed work items only (32 x 32 tiles).
template <int AM, int BM, bool LOWER>
__global__ void __launch_bounds__(gemm_threads<32>(), 8)
    k_gemm_f64_items(const __grid_constant__ GemmGroup g, const __grid_constant__ GemmItems it) {
  __shared__ double As[gemm_kblock<32>()][33];
  __shared__ double Bs[gemm_kblock<32>()][33];
  gemm_tile<AM, BM, LOWER, 32>(g, it.bid[blockIdx.x], As, Bs);
}

// Deterministic split-K reduction: Cout = beta Cin + sum_z part[z], z in order.
template <bool LOWER>
__device__ __forceinline__ void reduce_desc(const GemmGroup &g, const GemmDesc &d, long long first, long long stride) {
  const long long total = (long long)d.M * d.N;
  for (long long e = first; e < total; e += stride) {
    const int i = (int)(e / d.N), j = (int)(e - (long long)i * d.N);
    if (LOWER && j > i) continue;
    // The K splits that can contribute to this element's tile: with
    // triangular operands the others hold zeros (or were not launched).
    int zlo = 0, zhi = d.splits;
    if (g.tri && g.ts > 0) {
      const int m0 = i / g.ts * g.ts, n0 = j / g.ts * g.ts;
      int klo = 0, khi = d.K;
      if (g.tri & TRI_A_UPPER) klo = max(klo, m0);
      if (g.tri & TRI_B_LOWER) klo = max(klo, n0);
      if (g.tri & TRI_A_LOWER) khi = min(khi, m0 + g.ts);
      if (g.tri & TRI_B_UPPER) khi = min(khi, n0 + g.ts);
      zlo = klo / d.kchunk;
      zhi = klo < khi ? min(d.splits, (khi + d.kchunk - 1) / d.kchunk) : zlo;
    }
    // Partials loaded eight at a time (independent loads in flight), summed
    // in order.
    double s = 0.0;
    for (int z0 = zlo; z0 < zhi; z0 += 8) {
      double v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) v[q] = z0 + q < zhi ? __ldcg(d.part + (long long)(z0 + q) * total + e) : 0.0;
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (z0 + q < zhi) s += v[q];
    }
    if (LOWER && g.phi && i == j) s *= 0.5;
    if (d.beta != 0.0) s = fma(d.beta, d.Cin[(long long)i * d.ldcin + j], s);
    d.Cout[(long long)i * d.ldcout + j] = s;
  }
}

template <bool LOWER>
__global__ void k_reduce_f64(const __grid_constant__ GemmGroup g) {
  const GemmDesc &d = g.d[blockIdx.y];
  if (d.splits <= 1) return;
  reduce_desc<LOWER>(g, d, (long long)blockIdx.x * blockDim.x + threadIdx.x, (long long)gridDim.x * blockDim.x);
}

template <int AM, int BM>
static cudaError_t launch_gemm_ab(const GemmGroup &g, cudaStream_t s) {
  if (g.ts == 32) {
    if (g.lower)
      k_gemm_f64<AM, BM, true, 32><<<g.total_tiles, gemm_threads<32>(), 0, s>>>(g);
    else
      k_gemm_f64<AM, BM, false, 32><<<g.total_tiles, gemm_threads<32>(), 0, s>>>(g);
  } else {
    if (g.lower)
      k_gemm_f64<AM, BM, true, 64><<<g.total_tiles, gemm_threads<64>(), 0, s>>>(g);
    else
      k_gemm_f64<AM, BM, false, 64><<<g.total_tiles, gemm_threads<64>(), 0, s>>>(g);
  }
  return cudaGetLastError();
}

template <int AM, int BM>
static cudaError_t launch_items_ab(const GemmGroup &g, const GemmItems &it, cudaStream_t s) {
  if (g.lower)
    k_gemm_f64_items<AM, BM, true><<<it.count, gemm_threads<32>(), 0, s>>>(g, it);
  else
    k_gemm_f64_items<AM, BM, false><<<it.count, gemm_threads<32>(), 0, s>>>(g, it);
  return cudaGetLastError();
}

cudaError_t launch_gemm_items(const GemmGroup &g, const GemmItems &it, cudaStream_t s) {
  if (g.count <= 0 || it.count <= 0) return cudaSuccess;
  if (g.ts != 32 || it.count > kMaxItems) return cudaErrorInvalidValue;
  switch (g.amode * 8 + g.bmode) {
    case A_N * 8 + B_N: return launch_items_ab<A_N, B_N>(g, it, s);
    case A_N * 8 + B_T: return launch_items_ab<A_N, B_T>(g, it, s);
    case A_N * 8 + B_TL: return launch_items_ab<A_N, B_TL>(g, it, s);
    case A_T * 8 + B_N: return launch_items_ab<A_T, B_N>(g, it, s);
    case A_SYM2 * 8 + B_N: return launch_items_ab<A_SYM2, B_N>(g, it, s);
    case A_TL * 8 + B_NL: return launch_items_ab<A_TL, B_NL>(g, it, s);
    case A_SYM1 * 8 + B_T: return launch_items_ab<A_SYM1, B_T>(g, it, s);
    case A_NL * 8 + B_NL: return launch_items_ab<A_NL, B_NL>(g, it, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_gemm_group(const GemmGroup &g, cudaStream_t s) {
  if (g.count <= 0 || g.total_tiles <= 0) return cudaSuccess;
  switch (g.amode * 8 + g.bmode) {
    case A_N * 8 + B_N: return launch_gemm_ab<A_N, B_N>(g, s);
    case A_N * 8 + B_T: return launch_gemm_ab<A_N, B_T>(g, s);
    case A_N * 8 + B_TL: return launch_gemm_ab<A_N, B_TL>(g, s);
    case A_T * 8 + B_N: return launch_gemm_ab<A_T, B_N>(g, s);
    case A_SYM2 * 8 + B_N: return launch_gemm_ab<A_SYM2, B_N>(g, s);
    // symbolic diagonal steps (Eqs. symrevtril, symfwd)
    case A_TL * 8 + B_NL: return launch_gemm_ab<A_TL, B_NL>(g, s);
    case A_SYM1 * 8 + B_T: return launch_gemm_ab<A_SYM1, B_T>(g, s);
    case A_NL * 8 + B_NL: return launch_gemm_ab<A_NL, B_NL>(g, s);
    default: return cudaErrorInvalidValue;
  }
}

int gemm_ctas_per_sm(int ts) {
  int a = 0, b = 0;
  if (ts == 32) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_gemm_f64<A_N, B_N, false, 32>, gemm_threads<32>(), 0) !=
        cudaSuccess)
      a = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_gemm_f64<A_SYM2, B_N, false, 32>, gemm_threads<32>(), 0) !=
        cudaSuccess)
      b = 1;
  } else {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_gemm_f64<A_N, B_N, false, 64>, gemm_threads<64>(), 0) !=
        cudaSuccess)
      a = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_gemm_f64<A_SYM2, B_N, false, 64>, gemm_threads<64>(), 0) !=
        cudaSuccess)
      b = 1;
  }
  return std::max(1, std::min(a, b));
}

cudaError_t launch_reduce_group(const GemmGroup &g, cudaStream_t s) {
  bool any = false;
  long long biggest = 0;
  for (int p = 0; p < g.count; ++p)
    if (g.d[p].splits > 1) {
      any = true;
      biggest = (long long)g.d[p].M * g.d[p].N > biggest ? (long long)g.d[p].M * g.d[p].N : biggest;
    }
  if (!any) return cudaSuccess;
  long long blocks = (biggest + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  dim3 grid((unsigned)blocks, (unsigned)g.count);
  if (g.lower)
    k_reduce_f64<true><<<grid, 256, 0, s>>>(g);
  else
    k_reduce_f64<false><<<grid, 256, 0, s>>>(g);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Diagonal-tile kernels.  A t x t lower tile (t <= 128) is kept packed in
// shared memory, element (i, j <= i) at i (i + 1) / 2 + j.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int pk(int i, int j) { return (i * (i + 1) >> 1) + j; }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ void tile_load(double *S, const double *__restrict__ X, long long ldx, int t) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = warp; i < t; i += nw)
    for (int j = lane; j <= i; j += 32) S[pk(i, j)] = X[(long long)i * ldx + j];
}

__device__ void tile_store(const double *S, double *X, long long ldx, int t) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = warp; i < t; i += nw)
    for (int j = lane; j <= i; j += 32) X[(long long)i * ldx + j] = S[pk(i, j)];
}

// Row of flat index e in the packed lower triangle (row r holds r + 1 entries).
__device__ __forceinline__ int tri_row(int e) {
  int r = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
  while ((r + 1) * (r + 2) / 2 <= e) ++r;
  while (r * (r + 1) / 2 > e) --r;
  return r;
}

// chol_unblocked_rev (Sec. 4.1) on the tile: column j from t-1 down to 0,
//   d_bar <- (d_bar - c^T c_bar / d) / d,  c_bar <- c_bar / d,
//   r_bar <- r_bar - d_bar r - c_bar^T B,  B_bar <- B_bar - c_bar r,
//   d_bar <- d_bar / 2.
__device__ void dev_rev(const double *SL, double *SA, int t, double *red) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int j = t - 1; j >= 0; --j) {
    if (warp == 0) {
      double s = 0.0;
      for (int i = j + 1 + lane; i < t; i += 32) s = fma(SL[pk(i, j)], SA[pk(i, j)], s);
      s = warp_sum(s);
      if (lane == 0) red[0] = s;
    }
    __syncthreads();
    const double dj = SL[pk(j, j)];
    const double db = (SA[pk(j, j)] - red[0] / dj) / dj;
    for (int i = j + 1 + tid; i < t; i += blockDim.x) SA[pk(i, j)] /= dj;
    __syncthreads();
    const int len = t - j - 1;
    if (len > j) {
      // long dot products, few of them: one warp per k, lanes split the rows
      for (int k = warp; k < j; k += nw) {
        double s = 0.0;
        for (int i = j + 1 + lane; i < t; i += 32) s = fma(SA[pk(i, j)], SL[pk(i, k)], s);
        s = warp_sum(s);
        if (lane == 0) SA[pk(j, k)] = (SA[pk(j, k)] - db * SL[pk(j, k)]) - s;
      }
    } else {
      for (int k = tid; k < j; k += blockDim.x) {
        double s0 = 0.0, s1 = 0.0;
        int i = j + 1;
        for (; i + 1 < t; i += 2) {
          s0 = fma(SA[pk(i, j)], SL[pk(i, k)], s0);
          s1 = fma(SA[pk(i + 1, j)], SL[pk(i + 1, k)], s1);
        }
        if (i < t) s0 = fma(SA[pk(i, j)], SL[pk(i, k)], s0);
        SA[pk(j, k)] = (SA[pk(j, k)] - db * SL[pk(j, k)]) - (s0 + s1);
      }
    }
    for (int i = j + 1 + warp; i < t; i += nw) {
      const double cb = SA[pk(i, j)];
      for (int k = lane; k < j; k += 32) SA[pk(i, k)] -= cb * SL[pk(j, k)];
    }
    if (tid == 0) SA[pk(j, j)] = 0.5 * db;
    __syncthreads();
  }
}

// chol_unblocked_fwd (Sec. 4.1, Eqs. dub1-dub2) on the tile, right-looking:
// once column j of L_dot is final, its rank-2 contribution
// L_dot[:,j] L[k,j] + L[:,j] L_dot[k,j] is removed from every later column k.
__device__ void dev_sens(const double *SL, double *SD, int t) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int j = 0; j < t; ++j) {
    const double dj = SL[pk(j, j)];
    const double dd = 0.5 * SD[pk(j, j)] / dj;
    __syncthreads();
    for (int i = j + 1 + tid; i < t; i += blockDim.x)
      SD[pk(i, j)] = (SD[pk(i, j)] - SL[pk(i, j)] * dd) / dj;
    if (tid == 0) SD[pk(j, j)] = dd;
    __syncthreads();
    for (int i = j + 1 + warp; i < t; i += nw) {
      const double ldi = SD[pk(i, j)], li = SL[pk(i, j)];
      for (int k = j + 1 + lane; k <= i; k += 32)
        SD[pk(i, k)] -= ldi * SL[pk(k, j)] + li * SD[pk(k, j)];
    }
    __syncthreads();
  }
}

constexpr int kTileThreads = 256;
constexpr size_t kTileSmem = 2 * sizeof(double) * (kTileMax * (kTileMax + 1) / 2);

template <int OP>
__global__ void __launch_bounds__(kTileThreads) k_tile(const __grid_constant__ TileGroup g) {
  extern __shared__ double sm[];
  __shared__ double red[4];
  const TileDesc &d = g.d[blockIdx.x];
  const int t = d.t;
  if (t <= 0 || t > kTileMax) return;
  double *S0 = sm;
  double *S1 = sm + (kTileMax * (kTileMax + 1) / 2);
  tile_load(S0, d.L, d.ldl, t);
  tile_load(S1, d.X, d.ldx, t);
  __syncthreads();
  if (OP == T_REV)
    dev_rev(S0, S1, t, red);
  else
    dev_sens(S0, S1, t);
  __syncthreads();
  tile_store(S1, d.X, d.ldx, t);
}

// ---------------------------------------------------------------------------
// Diagonal tile on a thread-block cluster: chol_unblocked (Sec. 4.1) of a
// t x t tile (t <= 128) and the inverse of the factor, or the inverse alone.
//
// On GB300 every FP64 instruction holds its sub-partition's FP64 unit for
// about 64 cycles and a square root or division about 650, so a one-CTA
// factorisation of a 128 tile takes ~265 us: its 128 sequential pivots and
// the t^3/6 multiply-adds of its updates all run on one SM.  Here kCl CTAs
// (one SM each) share the tile through distributed shared memory: rows are
// dealt cyclically (row i to CTA i mod kCl); every CTA holds a full copy of
// L as it is finished.  The tile is factorised right-looking in 16-column
// panels (chol_blocked of Sec. 4.2 inside the tile):
//   (a) the owners of the panel's diagonal-block rows send them to all CTAs;
//   (b) every CTA factorises that block redundantly in its L D L^T form,
//       A = U diag(d) U^T with U unit lower, pipelined over four warps: warp
//       0 forms each pivot's reciprocal (an FP32 estimate and one cubic
//       correction: three FP64 operations instead of a division), U's column
//       u = a / d, publishes a and u and applies them to the next column at
//       once (lookahead of one), while warps 1-3 apply them to the later
//       columns -- the pivot chain costs five FP64 operations per column, and
//       all CTAs take the same pivot decisions; the block's square roots and
//       reciprocal square roots (Goldschmidt's iteration and two corrections)
//       are then taken for all its columns at once, one thread each;
//   (c) each CTA solves its own rows of the panel, C <- C L_D^{-T} with
//       L_D = U diag(sqrt(d)): forward substitution with U across the 16
//       lanes of a half-warp (each step a shuffle and one multiply-add), then
//       one multiply by 1/sqrt(d); it sends them to every CTA's copy of L;
//   (d) each CTA applies the rank-16 update to its own trailing rows.
// Two cluster barriers per panel.  The inverse then needs one exchange: CTA b
// inverts diagonal block b (a forward-substitution sweep per column, again
// across half-warps) and sends it to all; each CTA then forms its own columns
// of X = L^{-1} block row by block row, X_bi = D_bi^{-1} (E - L_{bi,<bi} X_{<bi}).
// On request (TileDesc::fsl) X is also written in the operand format of the
// tensor-core panel solve that consumes it: the split-BF16 terms of each
// element, or fixed-point slices, whose per-row exponents take the row's
// largest |X| over the cluster (each CTA's maximum over its own columns,
// gathered through distributed shared memory).  That saves the mixed
// factorisation a split launch on its diagonal chain at every block step.
// ---------------------------------------------------------------------------
constexpr int kCl = 16;                    // CTAs per tile (a non-portable cluster size)
constexpr int kPb = 16;                    // panel width
constexpr int kOwn = kTileMax / kCl;       // rows (and inverse columns) per CTA
constexpr int kNpMax = kTileMax / kPb;     // panels per tile
constexpr int kPotrfThreads = 256;
constexpr int kLfN = kTileMax * (kTileMax + 1) / 2;
constexpr int kDgLd = kPb + 1;
// (a) sends each CTA's kPb / kCl rows of a diagonal block with one thread per (row, column, CTA);
// (c) takes a half-warp per own row on warps 4-7, (d) kPotrfThreads / kOwn threads per row; the inverse takes
// own-column pairs on warps 0 .. kOwn/2 - 1 (and their K ranges' second halves on the next
// kOwn/2 warps); CTA b inverts diagonal block b.
static_assert(kPotrfThreads == 256 && kPb * kPb == kPotrfThreads && kCl <= kPb && kPb <= 2 * kCl &&
                  2 * kOwn * kPb <= kPotrfThreads && kOwn % 2 == 0 && kOwn <= 16 && kNpMax <= kCl,
              "thread layout");
constexpr int kYt = kPb * (kOwn > kPb ? kOwn : kPb);  // Yt: kPb x kOwn, and the kPb x kPb block-inverse scratch
// With few own columns (kOwn = 8), two warps share a column pair in the inverse, one per half of
// its K range; Yt2 holds the second halves' sums.
constexpr bool kSplitK = 2 * kOwn * kPb <= kPotrfThreads;
constexpr size_t kPotrfSmem = sizeof(double) * (kLfN + kOwn * kTileMax + kPb * kDgLd + kTileMax +
                                                kNpMax * kPb * kPb + kTileMax * kOwn + kYt + (kSplitK ? kPb * kOwn : 0));

// mbarrier helpers for the pipelined panel factorisation (shared memory, one CTA).
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mb_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mb_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mb_test(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Waits for the phase of the given parity; gives up after 2 s, or at once
// once *abort is set (a wait of the same CTA gave up), setting *abort.
__device__ __forceinline__ void mb_wait(uint64_t *bar, uint32_t parity, volatile int *abort) {
  if (mb_test(bar, parity)) return;
  const unsigned long long t0 = now_ns();
  while (!mb_test(bar, parity)) {
    if (*abort) return;
    if (now_ns() - t0 > 2000000000ULL) {
      *abort = 1;
      return;
    }
  }
}

// Exact binary32 -> binary64 of a normal positive float, with integer operations.
__device__ __forceinline__ double pos_f32_to_f64(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t e = b >> 23;
  return __hiloint2double((int)(((e + 896u) << 20) | ((b & 0x7FFFFFu) >> 3)), (int)(b << 29));
}

// v * 2^k by the exponent field (v normal, result normal).
__device__ __forceinline__ double scale_pow2(double v, int k) {
  return __longlong_as_double(__double_as_longlong(v) + ((long long)k << 52));
}

// 1/sqrt(x) and sqrt(x) for a positive FP64 x by Goldschmidt's iteration
// (g -> sqrt(m), h -> 1/(2 sqrt(m)); r = 1/2 - g h, g += g r, h += h r),
// started from the FP32 hardware estimate of 1/sqrt(m), m = x 2^(-2k) in
// [1, 4).  Two iterations take the 2^-23 start near FP64 rounding; a final
// correction of the root from its residual m - g^2 and a Newton step of the
// reciprocal root from the exact residual 1 - m y^2 bring both within one
// unit in the last place (measured: the root correctly rounded).  Subnormal and infinite x
// take the library square root.
__device__ __forceinline__ void rsqrt_sqrt(double x, double &rs, double &sq) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)(b >> 52) & 0x7FF;
  if (e == 0 || e == 0x7FF) {
    sq = sqrt(x);
    rs = 1.0 / sq;
    return;
  }
  const int k = (e - 1023) >> 1;
  const unsigned long long em = (unsigned long long)(e - 2 * k);  // 1023 or 1024
  const double m = __longlong_as_double((long long)((b & 0x000FFFFFFFFFFFFFull) | (em << 52)));
  const float mf = __uint_as_float((unsigned)((em - 896ull) << 23) | (unsigned)((b >> 29) & 0x7FFFFFull));
  const double y0 = pos_f32_to_f64(rsqrtf(mf));
  double g = m * y0, h = scale_pow2(y0, -1);
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const double r = fma(-g, h, 0.5);
    g = fma(g, r, g);
    h = fma(h, r, h);
  }
  // final corrections (Goldschmidt's iteration alone leaves up to about 1.5
  // ulp): the root from its residual m - g^2 (exact through the FMA)
  g = fma(h, fma(-g, g, m), g);
  // y = 2 h ~ 1/sqrt(m): the residual 1 - m y^2 from the exact square
  // y^2 = p + q (q by FMA), then y += (y / 2) residual
  const double y = h + h;
  const double p = y * y, q = fma(y, y, -p);
  const double res = fma(-m, q, fma(-m, p, 1.0));
  sq = scale_pow2(g, k);
  rs = scale_pow2(fma(h, res, y), -k);
}

// 1/x for a positive normal FP64 x in three FP64 operations: the FP32
// approximate reciprocal (rcp.approx, relative error ~2^-23) of x's
// significand m, truncated to 24 bits, moved to x's exponent with integer
// operations, starts one step of the cubic iteration y <- y + y (e + e^2),
// e = 1 - x y (Householder's method of order two), which takes the ~2^-22
// start error e to ~e^3, below FP64 rounding.  Subnormal, infinite and very
// large x (whose reciprocal would be subnormal) divide.
__device__ __forceinline__ double recip_pos(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)(b >> 52) & 0x7FF;
  if (e == 0 || e >= 2045) return 1.0 / x;
  const float mf = __uint_as_float((127u << 23) | (unsigned)((b >> 29) & 0x7FFFFFull));  // [1, 2)
  float rf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(mf));  // in [0.5, 1]
  const double y0 = scale_pow2(pos_f32_to_f64(rf), 1023 - e);
  const double em = fma(-x, y0, 1.0);
  return fma(y0, fma(em, em, em), y0);
}

// Inverse of the lower kPb x kPb block of Lf at (c0, c0) (w x w used, rest
// zero) into Li (row major), given the reciprocals rd of its diagonal.  All
// 256 threads: half-warp q (16 lanes = rows) sweeps column q forward.
__device__ void block_inverse_sweep(const double *Lf, const double *rd, int c0, int w, double *Li) {
  const int lane16 = threadIdx.x & 15, col = threadIdx.x >> 4;  // 16 half-warps = 16 columns
  const int r = lane16;
  double x = (r == col && r < w) ? rd[c0 + r] : 0.0, acc = 0.0;
  for (int s = 0; s < kPb; ++s) {
    if (s > col && r == s && r < w) x = -acc * rd[c0 + r];
    const double xs = __shfl_sync(0xffffffffu, x, s, 16);
    if (r > s && s >= col && r < w) acc = fma(Lf[pk(c0 + r, c0 + s)], xs, acc);
  }
  Li[r * kPb + col] = (r >= col && r < w && col < w) ? x : 0.0;
}

__global__ void __cluster_dims__(kCl, 1, 1) __launch_bounds__(kPotrfThreads, 1)
    k_potrf_cluster(const __grid_constant__ TileGroup g) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ double sm[];
  __shared__ int s_bad;
  __shared__ volatile int s_tmo;
  __shared__ __align__(8) uint64_t pub_bar, done_bar;
  __shared__ double acol[2 * kPb], ucol[2 * kPb];
  __shared__ double Ut[kPb * kDgLd];  // the panel's unit-lower factor a / d (below the diagonal)
  __shared__ unsigned long long s_rmax[kTileMax];  // fixed-point output: row maxima of |X| (bits)
  __shared__ int s_fex[kTileMax];                   // and the rows' exponents
  const TileDesc &d = g.d[blockIdx.y];
  const int t = d.t;
  // Both exits below are taken by every CTA of the cluster alike (same
  // descriptor; info is written only by earlier launches), before any barrier.
  if (t <= 0 || t > kTileMax) return;
  const bool factor = d.X != nullptr;
  if (factor && d.info != nullptr && *(volatile int *)d.info != 0) return;  // an earlier column failed
  const int rank = (int)cluster.block_rank();
  const int tid = threadIdx.x;
  double *Lf = sm;                          // packed L, every row (each CTA holds a full copy)
  double *R = Lf + kLfN;                    // own rows i = rank + kCl * li, R[li * kTileMax + k]
  double *Dg = R + kOwn * kTileMax;         // the panel's diagonal block, kPb x kDgLd
  double *rd = Dg + kPb * kDgLd;            // reciprocals of L's diagonal
  double *Li = rd + kTileMax;               // inverses of the diagonal blocks, [block][kPb][kPb]
  double *Xc = Li + kNpMax * kPb * kPb;     // own inverse columns c = rank + kCl * q: Xc[r * kOwn + q]
  double *Yt = Xc + kTileMax * kOwn;        // kPb x kOwn temporary (kYt doubles: also a kPb x kPb scratch)
  double *Yt2 = Yt + kYt;                   // kPb x kOwn: the second halves of the K ranges (kSplitK)
  const int nown = rank < t ? (t - 1 - rank) / kCl + 1 : 0;
  const int np = (t + kPb - 1) / kPb;
  if (tid == 0) {
    s_bad = -1;
    s_tmo = 0;
    mb_init(&pub_bar, 1);
    mb_init(&done_bar, 3);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (factor) {
    for (int e = tid; e < nown * kTileMax; e += blockDim.x) {
      const int li = e / kTileMax, k = e - li * kTileMax, i = rank + kCl * li;
      if (k <= i) R[e] = d.X[(long long)i * d.ldx + k];
    }
    cluster.sync();  // every CTA resident (its shared memory exists) before any remote store
    for (int p = 0; p < np; ++p) {
      const int c0 = p * kPb, w = min(kPb, t - c0);
      {  // (a) own rows of the diagonal block (c0 + rank, and c0 + rank + kCl if kCl < kPb) to every CTA
        const int slot = tid / (kPb * kCl), c = (tid / kCl) % kPb, dst = tid % kCl;
        const int i = c0 + rank + kCl * slot;
        if (slot < 2 && i < c0 + w && c0 + c <= i) {
          double *rem = cluster.map_shared_rank(Dg, dst);
          rem[(i - c0) * kDgLd + c] = R[((i - rank) / kCl) * kTileMax + c0 + c];
        }
      }
      cluster.sync();
      if (tid < 128) {  // (b) chol_unblocked of the block in its L D L^T form, redundantly in
        // every CTA, A = U diag(d) U^T, pipelined: warp 0 (lanes = rows) forms
        // pivot d's reciprocal (three FP64 operations), the column a scaled by it,
        // u = a / d, publishes a and u, and applies them to the next column
        // at once; warps 1-3 apply them to the columns after that,
        // A(r, k) -= a(r) u(k).  The pivot chain is five FP64 operations a
        // column; the unscaled columns stay in Dg and become L's columns
        // a / sqrt(d) below, all at once.  g numbers the columns over all
        // panels: the phases of the two mbarriers.
        if (tid < 32) {
          const int r = tid;
          for (int c = 0; c < w; ++c) {
            const int g = c0 + c;
            const double piv = Dg[c * kDgLd + c];
            const long long pb = __double_as_longlong(piv);
            const bool ok = pb > 0 && pb <= 0x7FF0000000000000ll;  // piv > 0 (false for NaN)
            const double inv = ok ? recip_pos(piv) : 0.0;
            const double a = (r > c && r < w) ? Dg[r * kDgLd + c] : 0.0;
            const double u = a * inv;
            if (c >= 1) mb_wait(&done_bar, (uint32_t)(g - 1) & 1u, &s_tmo);  // workers' step g-1
            if (r > c && r < w) {
              acol[(g & 1) * kPb + r] = a;
              ucol[(g & 1) * kPb + r] = u;
              Ut[r * kDgLd + c] = u;  // U = a / d below the diagonal, for (c)
            }
            if (r == 0 && !ok && s_bad < 0) s_bad = c0 + c;
            __syncwarp();
            if (r == 0) mb_arrive(&pub_bar);
            const double unext = __shfl_sync(0xffffffffu, u, c + 1 < 32 ? c + 1 : 0);
            if (c + 1 < w && r >= c + 1 && r < w)  // column c+1 gets column c's update now
              Dg[r * kDgLd + c + 1] = fma(-a, unext, Dg[r * kDgLd + c + 1]);
            __syncwarp();
          }
        } else {
          const int e0 = tid - 32;
          for (int c = 0; c < w; ++c) {
            const int g = c0 + c;
            mb_wait(&pub_bar, (uint32_t)g & 1u, &s_tmo);
            const double *ac = acol + (g & 1) * kPb, *uc = ucol + (g & 1) * kPb;
            const int m = w - c - 2;  // columns c+2 .. w-1
            for (int e = e0; e < m * (m + 1) / 2; e += 96) {
              const int rr = tri_row(e), kk = e - rr * (rr + 1) / 2;
              const int r = c + 2 + rr, k = c + 2 + kk;
              Dg[r * kDgLd + k] = fma(-ac[r], uc[k], Dg[r * kDgLd + k]);
            }
            __syncwarp();
            if ((tid & 31) == 0) mb_arrive(&done_bar);
          }
        }
      }
      __syncthreads();
      // The panel rows' substitution (c) needs 1/sqrt(d) only for its last multiply, so it runs on
      // warps 4-7 while warp 0 takes the square roots.
      const int li = (tid - kPotrfThreads / 2) / kPb, cs = tid % kPb, irow = rank + kCl * li;
      const bool act = tid >= kPotrfThreads / 2 && li < nown && irow >= c0 + w;
      double acc = act && cs < w ? R[li * kTileMax + c0 + cs] : 0.0;
      if (tid >= kPotrfThreads / 2) {
        // (c) own rows below the block: y = C U^{-T} with the unit-lower factor U = a / d by forward
        // substitution across each half-warp (one FMA a step); L = y / sqrt(d) below.  A warp
        // whose two rows are both above the panel or absent has nothing to solve.
        if (__any_sync(0xffffffffu, act))
          for (int s2 = 0; s2 + 1 < w; ++s2) {
            const double ys = __shfl_sync(0xffffffffu, acc, s2, 16);
            if (cs > s2 && cs < w) acc = fma(-ys, Ut[cs * kDgLd + s2], acc);
          }
      } else if (tid < w) {  // pivots: sqrt(d) on L's diagonal, 1/sqrt(d) for the scaling and (c)
        const double piv = Dg[tid * kDgLd + tid];
        const long long pb = __double_as_longlong(piv);
        const bool ok = pb > 0 && pb <= 0x7FF0000000000000ll;
        double rs = 0.0, sq = piv;
        if (ok) rsqrt_sqrt(piv, rs, sq);
        Lf[pk(c0 + tid, c0 + tid)] = ok ? sq : piv;
        rd[c0 + tid] = rs;
      }
      __syncthreads();
      for (int e = tid; e < w * w; e += blockDim.x) {  // L's columns below the diagonal: a / sqrt(d)
        const int r = e / w, c = e - r * w;
        if (r > c) Lf[pk(c0 + r, c0 + c)] = Dg[r * kDgLd + c] * rd[c0 + c];
      }
      if (s_bad >= 0) break;  // the same in every CTA: all factorised the same block
      if (act && cs < w) {  // (c), finished: scale and send to every CTA's copy of L
        const double lic = acc * rd[c0 + cs];
        R[li * kTileMax + c0 + cs] = lic;
#pragma unroll
        for (int dst = 0; dst < kCl; ++dst) cluster.map_shared_rank(Lf, dst)[pk(irow, c0 + cs)] = lic;
      }
      cluster.sync();  // every CTA's Lf holds the panel's columns of L
      {  // (d) rank-kPb update of own trailing rows, kPotrfThreads / kOwn threads per row (a
        // warp's FP64 issue rate bounds the longest row, so every warp takes part)
        constexpr int kTpr = kPotrfThreads / kOwn;
        const int li = tid / kTpr, i = rank + kCl * li;
        if (li < nown && i >= c0 + w) {
          double lrow[kPb];
#pragma unroll
          for (int c = 0; c < kPb; ++c) lrow[c] = R[li * kTileMax + c0 + c];
          for (int k = c0 + w + (tid % kTpr); k <= i; k += kTpr) {
            const double *lk = Lf + pk(k, c0);
            double v = R[li * kTileMax + k];
#pragma unroll
            for (int c = 0; c < kPb; ++c) v = fma(-lrow[c], lk[c], v);
            R[li * kTileMax + k] = v;
          }
        }
      }
      __syncthreads();
    }
    cluster.sync();
    if (tid == 0 && s_tmo && g.err != nullptr) atomicExch(g.err, CD_ETIMEOUT);
    if (s_bad >= 0) {
      if (rank == 0 && tid == 0 && d.info != nullptr) *d.info = d.col0 + s_bad + 1;
      return;  // no remote store follows: each CTA may finish on its own
    }
    for (int e = tid; e < nown * kTileMax; e += blockDim.x) {
      const int li = e / kTileMax, k = e - li * kTileMax, i = rank + kCl * li;
      if (k <= i) d.X[(long long)i * d.ldx + k] = Lf[pk(i, k)];
    }
    if (d.inv == nullptr) return;  // no remote store follows
  } else {
    tile_load(Lf, d.L, d.ldl, t);
    __syncthreads();
    for (int i = tid; i < t; i += blockDim.x) rd[i] = 1.0 / Lf[pk(i, i)];
    cluster.sync();  // every CTA resident before the block inverses are exchanged
  }
  // Inverse.  CTA b inverts diagonal block b and sends it to every CTA.
  if (rank < np) {
    const int c0 = rank * kPb;
    __syncthreads();
    block_inverse_sweep(Lf, rd, c0, min(kPb, t - c0), Yt);  // Yt: kPb x kPb scratch here
    __syncthreads();
    for (int e = tid; e < kPb * kPb * kCl; e += blockDim.x) {
      const int dst = e / (kPb * kPb), o = e - dst * kPb * kPb;
      cluster.map_shared_rank(Li, dst)[rank * kPb * kPb + o] = Yt[o];
    }
  }
  cluster.sync();  // every CTA holds every block inverse; no remote store follows
  // Thread -> (row rr of a block row, own column q).  A warp takes two
  // adjacent columns (one per half-warp), so its lanes share the K range of
  // the substitution below instead of running to the longest of sixteen; the
  // column pairs are dealt so that the two warps of a sub-partition (w and
  // w + 4) hold one long and one short column pair between them.
  const int warp = tid >> 5, lane = tid & 31;
  // kSplitK: warps w and w + kOwn/2 take column pair w, the first and the second half of its K range
  const int khalf = kSplitK ? warp / (kOwn / 2) : 0;
  const int q0 = kSplitK ? 2 * (warp % (kOwn / 2)) : (warp < 4 ? 2 * warp : 22 - 2 * warp);
  const int rr = lane & 15, q = q0 + (lane >> 4), c = rank + kCl * q;
  const bool qok = q < kOwn;
  for (int bi = 0; bi < np; ++bi) {
    const int r0 = bi * kPb, wb = min(kPb, t - r0), r = r0 + rr;
    double y = 0.0;
    if (qok && rr < wb && c < t && c <= r) {
      const int kmid = kSplitK ? (c + r0 + 1) / 2 : r0;  // [c, kmid) and [kmid, r0)
      const int ka = khalf ? kmid : c, kb = khalf ? r0 : kmid;
      y = (!khalf && r == c) ? 1.0 : 0.0;
      for (int k = ka; k < kb; ++k) y = fma(-Lf[pk(r, k)], Xc[k * kOwn + q], y);
    }
    if (qok) (khalf ? Yt2 : Yt)[rr * kOwn + q] = y;
    __syncthreads();
    if (kSplitK) {
      if (qok && !khalf) Yt[rr * kOwn + q] += Yt2[rr * kOwn + q];
      __syncthreads();
    }
    if (qok && !khalf && rr < wb) {
      double x = 0.0;
      if (c <= r) {  // X(r, c) = 0 above the diagonal; never read there
        const double *Lb = Li + bi * kPb * kPb + rr * kPb;
        for (int r2 = 0; r2 <= rr; ++r2) x = fma(Lb[r2], Yt[r2 * kOwn + q], x);
      }
      Xc[r * kOwn + q] = x;
    }
    __syncthreads();
  }
  if (d.fsl != nullptr && d.fterms > 0) {  // the inverse also as the split-BF16 terms of the panel solve
    __nv_bfloat16 *tsl = (__nv_bfloat16 *)d.fsl;
    const long long ts = (long long)d.frows * d.ldf;
    for (int e = tid; e < d.frows * kOwn; e += blockDim.x) {
      const int r = e / kOwn, qq = e - r * kOwn, cc = rank + kCl * qq;
      if (cc >= d.frows) continue;
      float hi, lo;
      f64_to_f32x2((r < t && cc <= r) ? Xc[r * kOwn + qq] : 0.0, hi, lo);
      write_split_terms(tsl, ts, (long long)r * d.ldf + cc, hi, lo, d.fterms);
    }
  } else if (d.fsl != nullptr) {
    // The inverse also in the fixed-point format of the tensor-core panel solve: row r's exponent
    // from its largest |X(r, c)| over the cluster (each CTA's maximum over its own columns,
    // gathered through distributed shared memory), then each CTA writes its own columns' slices
    // (zero outside the tile's lower triangle, up to frows <= kTileMax rows and columns).
    for (int r = tid; r < kTileMax; r += blockDim.x) {
      unsigned long long m = 0;  // |x| as bits: ordered like the values
      if (r < t)
        for (int qq = 0; qq < kOwn; ++qq) {
          const int cc = rank + kCl * qq;
          if (cc <= r) m = max(m, (unsigned long long)__double_as_longlong(fabs(Xc[r * kOwn + qq])));
        }
      s_rmax[r] = m;
    }
    cluster.sync();
    for (int r = tid; r < kTileMax; r += blockDim.x) {
      unsigned long long m = 0;
      for (int b = 0; b < kCl; ++b) m = max(m, cluster.map_shared_rank(s_rmax, b)[r]);
      const int E = exp_above(__longlong_as_double((long long)m));
      s_fex[r] = E;
      if (rank == 0 && r < d.frows) d.fex[r] = E;
    }
    cluster.sync();  // every CTA has read every maximum; none is read after this
    __nv_bfloat16 *fsl = (__nv_bfloat16 *)d.fsl;
    const long long ts = (long long)d.frows * d.ldf;
    for (int e = tid; e < d.frows * kOwn; e += blockDim.x) {
      const int r = e / kOwn, qq = e - r * kOwn, cc = rank + kCl * qq;
      if (cc >= d.frows) continue;
      const double x = (r < t && cc <= r) ? Xc[r * kOwn + qq] : 0.0;
      write_fixed_slices(fsl, ts, (long long)r * d.ldf + cc, fixed_q(x, s_fex[r]));
    }
  }
  for (int e = tid; e < t * kOwn; e += blockDim.x) {
    const int r2 = e / kOwn, qq = e - r2 * kOwn, cc = rank + kCl * qq;
    if (cc < t) d.inv[(long long)r2 * d.ldinv + cc] = (cc <= r2) ? Xc[e] : 0.0;
  }
}

cudaError_t launch_potrf_cluster_group(const TileGroup &g, cudaStream_t s) {
  if (g.count <= 0) return cudaSuccess;
  k_potrf_cluster<<<dim3(kCl, (unsigned)g.count), kPotrfThreads, kPotrfSmem, s>>>(g);
  return cudaGetLastError();
}

cudaError_t launch_tile_group(TileOp op, const TileGroup &g, cudaStream_t s) {
  if (g.count <= 0) return cudaSuccess;
  switch (op) {
    case T_REV: k_tile<T_REV><<<g.count, kTileThreads, kTileSmem, s>>>(g); break;
    case T_SENS: k_tile<T_SENS><<<g.count, kTileThreads, kTileSmem, s>>>(g); break;
    case T_TRTRI:  // the inverse of a given factor: the cluster kernel without its factorisation
    case T_POTRF: return launch_potrf_cluster_group(g, s);
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Explicit Jacobian (Eq. delements), for analysis: Theta(n^4) time and memory.
//   dL_ij / dSigma_kl = S_ijk Linv_jl + (1 - delta_kl) S_ijl Linv_jk,
//   S_ijk = sum_{m > j} L_im Linv_mk + L_ij Linv_jk / 2,   i >= j, k >= l,
// with Sigma_kl and Sigma_lk one tied input.  Linv is lower triangular, so
// the sum runs over max(j + 1, k) <= m <= i.
// ---------------------------------------------------------------------------
__global__ void k_jac_s(int n, const double *__restrict__ L, long long ldl, const double *__restrict__ Li,
                        long long ldi, double *__restrict__ S) {
  const long long total = (long long)n * n * n;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(e % n);
    const long long r = e / n;
    const int j = (int)(r % n), i = (int)(r / n);
    double v = 0.0;
    if (j <= i && k <= i) {
      for (int m = max(j + 1, k); m <= i; ++m) v = fma(L[(long long)i * ldl + m], Li[(long long)m * ldi + k], v);
      if (k <= j) v = fma(0.5 * L[(long long)i * ldl + j], Li[(long long)j * ldi + k], v);
    }
    S[e] = v;
  }
}

__global__ void k_jac(int n, const double *__restrict__ Li, long long ldi, const double *__restrict__ S,
                      double *__restrict__ J) {
  const long long n2 = (long long)n * n, total = n2 * n2;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int l = (int)(e % n), k = (int)((e / n) % n);
    const long long ij = e / n2;
    const int j = (int)(ij % n), i = (int)(ij / n);
    double v = 0.0;
    if (j <= i && l <= k) {
      const double *Sij = S + ij * n;
      v = Sij[k] * Li[(long long)j * ldi + l];
      if (k != l) v = fma(Sij[l], Li[(long long)j * ldi + k], v);
    }
    J[e] = v;
  }
}

cudaError_t launch_jacobian(int n, const double *L, long long ldl, const double *Li, long long ldi, double *S,
                            double *J, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const long long n3 = (long long)n * n * n, n4 = n3 * n;
  k_jac_s<<<(unsigned)std::min<long long>(8192, (n3 + 255) / 256), 256, 0, s>>>(n, L, ldl, Li, ldi, S);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_jac<<<(unsigned)std::min<long long>(65536, (n4 + 255) / 256), 256, 0, s>>>(n, Li, ldi, S, J);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Small helpers
// ---------------------------------------------------------------------------
__global__ void k_copy(const double *__restrict__ src, long long lds, double *__restrict__ dst, long long ldd,
                       int rows, int cols) {
  const long long total = (long long)rows * cols;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / cols), j = (int)(e - (long long)i * cols);
    dst[(long long)i * ldd + j] = src[(long long)i * lds + j];
  }
}

cudaError_t launch_copy(const double *src, long long lds, double *dst, long long ldd, int rows, int cols,
                        cudaStream_t s) {
  const long long total = (long long)rows * cols;
  if (total <= 0) return cudaSuccess;
  long long blocks = (total + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  k_copy<<<(unsigned)blocks, 256, 0, s>>>(src, lds, dst, ldd, rows, cols);
  return cudaGetLastError();
}

__global__ void k_copy_group(const __grid_constant__ CopyGroup g) {
  const CopyDesc &d = g.d[blockIdx.y];
  const long long total = (long long)d.rows * d.cols;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / d.cols), j = (int)(e - (long long)i * d.cols);
    d.dst[(long long)i * d.ldd + j] = d.src[(long long)i * d.lds + j];
  }
}

cudaError_t launch_copy_group(const CopyGroup &g, cudaStream_t s) {
  if (g.count <= 0) return cudaSuccess;
  long long biggest = 0;
  for (int p = 0; p < g.count; ++p) biggest = std::max(biggest, (long long)g.d[p].rows * g.d[p].cols);
  if (biggest <= 0) return cudaSuccess;
  const long long blocks = std::min<long long>(1024, (biggest + 255) / 256);
  k_copy_group<<<dim3((unsigned)blocks, (unsigned)g.count), 256, 0, s>>>(g);
  return cudaGetLastError();
}

// dst(i, j) -= src(i, j) + src(j, i) on and below the diagonal of a square
// block: D_dot <- D_dot - tril(P + P^T) with P = R_dot R^T, which is the
// forward-sensitivity update g1 (R R_dot^T = P^T) from one product.
__global__ void k_subsym_group(const __grid_constant__ CopyGroup g) {
  const CopyDesc &d = g.d[blockIdx.y];
  const long long total = (long long)d.rows * d.cols;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / d.cols), j = (int)(e - (long long)i * d.cols);
    if (j > i) continue;
    double *o = d.dst + (long long)i * d.ldd + j;
    *o -= d.src[(long long)i * d.lds + j] + d.src[(long long)j * d.lds + i];
  }
}

cudaError_t launch_subsym_group(const CopyGroup &g, cudaStream_t s) {
  if (g.count <= 0) return cudaSuccess;
  long long biggest = 0;
  for (int p = 0; p < g.count; ++p) biggest = std::max(biggest, (long long)g.d[p].rows * g.d[p].cols);
  if (biggest <= 0) return cudaSuccess;
  const long long blocks = std::min<long long>(1024, (biggest + 255) / 256);
  k_subsym_group<<<dim3((unsigned)blocks, (unsigned)g.count), 256, 0, s>>>(g);
  return cudaGetLastError();
}

// Strict upper triangle <- mirror of the strict lower one, through a 32 x 32
// shared tile so that both the reads and the writes are coalesced.
__global__ void k_mirror(double *A, long long lda, int n) {
  __shared__ double tile[32][33];
  const int bi = blockIdx.y, bj = blockIdx.x;  // source tile (rows bi, cols bj), bi >= bj
  if (bj > bi) return;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int r = ty; r < 32; r += 8) {
    const int i = bi * 32 + r, j = bj * 32 + tx;
    tile[r][tx] = (i < n && j < n) ? A[(long long)i * lda + j] : 0.0;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int i = bj * 32 + r, j = bi * 32 + tx;  // destination (i, j), upper: j > i
    if (i < n && j < n && j > i) A[(long long)i * lda + j] = tile[tx][r];
  }
}

// dst(i, j) = src(j, i) through 32 x 32 shared tiles, both sides coalesced.
// mode 0: the lower triangle of dst from the upper triangle of src (the
// lower one of src is not read); mode 1: the upper triangle of dst from the
// lower triangle of src; mode 2: every element.
__global__ void k_transpose(const double *src, long long lds, double *dst, long long ldd, int n, int mode) {
  __shared__ double tile[32][33];
  const int bi = blockIdx.y, bj = blockIdx.x;  // destination tile: rows bi, columns bj
  if ((mode == 0 && bj > bi) || (mode == 1 && bj < bi)) return;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int r = ty; r < 32; r += 8) {
    const int si = bj * 32 + r, sj = bi * 32 + tx;  // src(si, sj) = dst(sj, si)
    const bool want = mode == 2 || (mode == 0 ? sj >= si : sj <= si);
    tile[r][tx] = (si < n && sj < n && want) ? src[(long long)si * lds + sj] : 0.0;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int i = bi * 32 + r, j = bj * 32 + tx;
    const bool want = mode == 2 || (mode == 0 ? j <= i : j >= i);
    if (i < n && j < n && want) dst[(long long)i * ldd + j] = tile[tx][r];
  }
}

cudaError_t launch_transpose(const double *src, long long lds, double *dst, long long ldd, int n, int mode,
                             cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int nt = (n + 31) / 32;
  k_transpose<<<dim3(nt, nt), dim3(32, 8), 0, s>>>(src, lds, dst, ldd, n, mode);
  return cudaGetLastError();
}

cudaError_t launch_mirror_lower(double *A, long long lda, int n, cudaStream_t s) {
  if (n <= 1) return cudaSuccess;
  const int nt = (n + 31) / 32;
  k_mirror<<<dim3(nt, nt), dim3(32, 8), 0, s>>>(A, lda, n);
  return cudaGetLastError();
}

// The small kernels of the diagonal chain (32 x 32 GEMM tiles, split-K
// reductions, copies) ask for the largest shared-memory carveout: an SM
// configured for a tensor-core product's 211 KB then still takes their CTAs
// beside it.  With the default preference a kernel without shared memory
// (a split-K reduction) was held until the SM's other work drained.
template <class K>
static cudaError_t carve(K *k) {
  return cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
}
template <int AM, int BM>
static cudaError_t carve_ab() {
  cudaError_t e;
  if ((e = carve(k_gemm_f64<AM, BM, true, 32>)) || (e = carve(k_gemm_f64<AM, BM, false, 32>)) ||
      (e = carve(k_gemm_f64_items<AM, BM, true>)) || (e = carve(k_gemm_f64_items<AM, BM, false>)))
    return e;
  return cudaSuccess;
}

cudaError_t tile_kernels_init() {
  cudaError_t e;
  if ((e = carve_ab<A_N, B_N>()) || (e = carve_ab<A_N, B_T>()) || (e = carve_ab<A_N, B_TL>()) ||
      (e = carve_ab<A_T, B_N>()) || (e = carve_ab<A_SYM2, B_N>()) || (e = carve_ab<A_TL, B_NL>()) ||
      (e = carve_ab<A_SYM1, B_T>()) || (e = carve_ab<A_NL, B_NL>()) || (e = carve(k_reduce_f64<true>)) ||
      (e = carve(k_reduce_f64<false>)) || (e = carve(k_copy)) || (e = carve(k_copy_group)) ||
      (e = carve(k_subsym_group)))
    return e;
  if ((e = cudaFuncSetAttribute(k_tile<T_REV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTileSmem)))
    return e;
  if ((e = cudaFuncSetAttribute(k_tile<T_SENS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTileSmem)))
    return e;
  if ((e = cudaFuncSetAttribute(k_potrf_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPotrfSmem)))
    return e;
  if (kCl > 8 && (e = cudaFuncSetAttribute(k_potrf_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1)))
    return e;
  return cudaSuccess;
}

// The factorisation's FP64 reciprocal and square-root helpers applied to an
// array, so that they can be checked against correctly rounded references.
__global__ void k_fp64_helpers(int n, const double *x, double *recip, double *sq, double *rsq) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = x[i];
  recip[i] = recip_pos(v);
  double rs, s2;
  rsqrt_sqrt(v, rs, s2);
  sq[i] = s2;
  rsq[i] = rs;
}

cudaError_t launch_fp64_helpers(int n, const double *x, double *recip, double *sq, double *rsq, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_fp64_helpers<<<(n + 255) / 256, 256, 0, st>>>(n, x, recip, sq, rsq);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FP64 peak probes (measurement support): the rate of the FP64 pipe as the
// products above use it (DFMA) and of the FP64 matrix instruction
// (mma.sync m8n8k4), on register operands only.  Eight independent chains a
// thread hide the pipe's latency; the sink store never happens for the
// values reached, but the compiler cannot know that.
__device__ double g_fp64_sink;

// DFMA: a 4 x 2 register outer product per thread, acc += a b^T, with a
// rotated between rounds (register moves, off the FP64 pipe).  Measured on
// GB300: small outer products (4 x 2, 2 x 2, 8 x 1) reach the same rate,
// while shapes with more accumulators per operand (4 x 4, 3 x 4) lose about
// a sixth to operand-register conflicts.
template <int R, int C>
__global__ void k_dfma_probe(long long iters, double seed) {
  double acc[R][C], a[R], b[C];
#pragma unroll
  for (int i = 0; i < R; ++i) a[i] = seed * (threadIdx.x + i + 1);
#pragma unroll
  for (int j = 0; j < C; ++j) b[j] = 1.0 - seed * (j + 1);
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < C; ++j) acc[i][j] = 0.0;
  for (long long it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
      for (int j = 0; j < C; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    const double t = a[0];
#pragma unroll
    for (int i = 0; i + 1 < R; ++i) a[i] = a[i + 1];
    a[R - 1] = t;
  }
  double sum = 0.0;
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < C; ++j) sum += acc[i][j];
  if (sum == 1234.5678) g_fp64_sink = sum;
}

__global__ void __launch_bounds__(256) k_dmma_probe(long long iters, double seed) {
  double d[4][2];
#pragma unroll
  for (int c = 0; c < 4; ++c) d[c][0] = d[c][1] = seed * (threadIdx.x + c);
  const double a = 1.0 - 1e-12, b = 1e-3;
  for (long long i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < 4; ++c)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                   : "+d"(d[c][0]), "+d"(d[c][1])
                   : "d"(a), "d"(b));
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < 4; ++c) s += d[c][0] + d[c][1];
  if (s == 1234.5678) g_fp64_sink = s;
}

cudaError_t launch_fp64_probe(int kind, int blocks, long long iters, cudaStream_t st, double *flops) {
  const int threads = 256;
  if (kind == 0) {
    k_dfma_probe<4, 2><<<blocks, threads, 0, st>>>(iters, 1e-3);
    *flops = 2.0 * 8.0 * (double)iters * threads * blocks;  // 4 x 2 multiply-adds a round
  } else {
    k_dmma_probe<<<blocks, threads, 0, st>>>(iters, 1e-3);
    *flops = 2.0 * 256.0 * 4.0 * (double)iters * (threads / 32) * blocks;  // 8 x 8 x 4 per warp instruction
  }
  return cudaGetLastError();
}

}  // namespace cd
