// FP64 kernels of libcholdiff: the grouped DFMA tile GEMM used for every
// off-diagonal block update of the blocked algorithms (Sec. 4.2), and the
// one-CTA diagonal-tile kernels that run the level-2 routines of Sec. 4.1 on
// a tile held in shared memory.
//
// On GB300 the FP64 pipe issues about two DFMA per clock per SM (measured:
// 1.19 TFLOP/s for the whole GPU, 8 GFLOP/s on one SM), and DMMA
// (mma.sync f64) is slower still, so the FP64 engine is a register-blocked
// DFMA kernel: its only job is to keep the FP64 pipe of every SM busy.
#include <cuda_runtime.h>

#include <algorithm>

#include "cd_internal.h"

namespace cd {

// ---------------------------------------------------------------------------
// Grouped GEMM
// ---------------------------------------------------------------------------
constexpr int GBM = 64, GBN = 64, GBK = 16, GT = 256;

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

// One CTA computes a 64 x 64 output tile over its K range; each thread owns a
// 4 x 4 micro-tile (rows ty + 16 r, columns tx + 16 c), so a warp reads two
// A values (broadcast) and sixteen consecutive B values per k.
template <int AM, int BM, bool LOWER>
__global__ void __launch_bounds__(GT) k_gemm_f64(const __grid_constant__ GemmGroup g) {
  const int bid = blockIdx.x;
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
    m0 = ti * GBM;
    n0 = (rem - ti * (ti + 1) / 2) * GBN;
  } else {
    m0 = (rem / d.tiles_n) * GBM;
    n0 = (rem % d.tiles_n) * GBN;
  }
  const int kbeg = z * d.kchunk;
  const int kend = min(d.K, kbeg + d.kchunk);
  const double *__restrict__ A = d.A;
  const double *__restrict__ B = d.B;
  const long long lda = d.lda, ldb = d.ldb;

  __shared__ double As[GBK][GBM + 1];
  __shared__ double Bs[GBK][GBN + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = 0.0;

  for (int k0 = kbeg; k0 < kend; k0 += GBK) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int e = tid + r * GT;
      int kk, ii;
      if (AM == A_T) { ii = e & 63; kk = e >> 6; } else { kk = e & 15; ii = e >> 4; }
      const int gi = m0 + ii, gk = k0 + kk;
      As[kk][ii] = (gi < M && gk < kend) ? load_a<AM>(A, lda, gi, gk) : 0.0;
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int e = tid + r * GT;
      int kk, jj;
      if (BM == B_N) { jj = e & 63; kk = e >> 6; } else { kk = e & 15; jj = e >> 4; }
      const int gj = n0 + jj, gk = k0 + kk;
      Bs[kk][jj] = (gj < N && gk < kend) ? load_b<BM>(B, ldb, gk, gj) : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GBK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[kk][ty + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = Bs[kk][tx + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
    }
    __syncthreads();
  }

  const double alpha = d.alpha, beta = d.beta;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int i = m0 + ty + 16 * r;
    if (i >= M) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int j = n0 + tx + 16 * c;
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

// Deterministic split-K reduction: Cout = beta Cin + sum_z part[z], z in order.
template <bool LOWER>
__global__ void k_reduce_f64(const __grid_constant__ GemmGroup g) {
  const GemmDesc &d = g.d[blockIdx.y];
  if (d.splits <= 1) return;
  const long long total = (long long)d.M * d.N;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / d.N), j = (int)(e - (long long)i * d.N);
    if (LOWER && j > i) continue;
    double s = 0.0;
    for (int z = 0; z < d.splits; ++z) s += d.part[(long long)z * total + e];
    if (LOWER && g.phi && i == j) s *= 0.5;
    if (d.beta != 0.0) s = fma(d.beta, d.Cin[(long long)i * d.ldcin + j], s);
    d.Cout[(long long)i * d.ldcout + j] = s;
  }
}

template <int AM, int BM>
static cudaError_t launch_gemm_ab(const GemmGroup &g, cudaStream_t s) {
  if (g.lower)
    k_gemm_f64<AM, BM, true><<<g.total_tiles, GT, 0, s>>>(g);
  else
    k_gemm_f64<AM, BM, false><<<g.total_tiles, GT, 0, s>>>(g);
  return cudaGetLastError();
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

int gemm_ctas_per_sm() {
  int a = 0, b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_gemm_f64<A_N, B_N, false>, GT, 0) != cudaSuccess) a = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_gemm_f64<A_SYM2, B_N, false>, GT, 0) != cudaSuccess) b = 1;
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

// chol_unblocked (Sec. 4.1) on the tile, in right-looking order (the same
// arithmetic as the paper's column loop, with each column's update applied
// as soon as the column is final).  Per column: one thread forms the pivot's
// square root and reciprocal; all threads scale the column by it; then the
// rank-1 update of the trailing triangle is spread flat over all threads,
// one FMA per element, so every warp is full.  cj holds the unscaled column
// (double-buffered: the update writes the next column's values into cn).
// Returns the first 0-based column whose pivot is not positive (or NaN), else -1.
__device__ int dev_potf2(double *T, int t, double *cbuf, double *red) {
  const int tid = threadIdx.x;
  double *sc = cbuf + 2 * kTileMax;  // scaled column j
  // flat index -> (row, column) of a trailing triangle, the same for every column
  short2 *rc = reinterpret_cast<short2 *>(cbuf + 3 * kTileMax);
  const int Emax = t * (t - 1) / 2;
  for (int e = tid; e < Emax; e += blockDim.x) {
    const int r = tri_row(e);
    rc[e] = make_short2((short)r, (short)(e - r * (r + 1) / 2));
  }
  for (int i = tid; i < t; i += blockDim.x) cbuf[i] = T[pk(i, 0)];
  __syncthreads();
  for (int j = 0; j < t; ++j) {
    double *cj = cbuf + (j & 1) * kTileMax;
    double *cn = cbuf + ((j + 1) & 1) * kTileMax;
    if (tid == 0) {
      const double piv = cj[j];
      const bool ok = piv > 0.0;
      const double dj = ok ? sqrt(piv) : 0.0;
      red[0] = ok ? 1.0 / dj : 0.0;
      red[1] = ok ? 1.0 : 0.0;
      T[pk(j, j)] = ok ? dj : piv;
    }
    __syncthreads();
    if (red[1] == 0.0) return j;
    const double rd = red[0];
    for (int i = j + 1 + tid; i < t; i += blockDim.x) {
      const double v = cj[i] * rd;
      sc[i] = v;
      T[pk(i, j)] = v;
    }
    __syncthreads();
    const int m = t - j - 1;
    const int E = m * (m + 1) / 2;
    for (int e = tid; e < E; e += blockDim.x) {
      const short2 q = rc[e];
      const int cc = q.y, i = j + 1 + q.x, k = j + 1 + cc;
      const double v = fma(-sc[i], sc[k], T[pk(i, k)]);
      T[pk(i, k)] = v;
      if (cc == 0) cn[i] = v;
    }
    __syncthreads();
  }
  return -1;
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
  if (OP == T_POTF2) {
    if (d.info != nullptr && *(volatile int *)d.info != 0) return;  // an earlier column failed
    tile_load(S0, d.X, d.ldx, t);
    __syncthreads();
    const int bad = dev_potf2(S0, t, S1, red);
    __syncthreads();
    tile_store(S0, d.X, d.ldx, t);
    if (bad >= 0 && threadIdx.x == 0 && d.info != nullptr) *d.info = d.col0 + bad + 1;
  } else {
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
}

// X = T^{-1} for a lower tile T (t <= 128): every column of X is an
// independent forward substitution T x = e_c, so each warp computes one
// column (lanes split the dot products, a shuffle tree sums them) and a tile
// spreads over t / 8 CTAs.  Writes the full t x t inverse, zeros above.
constexpr int kInvCols = 8;  // columns (warps) per CTA
constexpr size_t kInvSmem = sizeof(double) * (kTileMax * (kTileMax + 1) / 2 + kTileMax + kInvCols * kTileMax);

__global__ void __launch_bounds__(32 * kInvCols) k_trtri_cols(const __grid_constant__ TileGroup g) {
  extern __shared__ double sm[];
  const TileDesc &d = g.d[blockIdx.y];
  const int t = d.t;
  const int c0 = blockIdx.x * kInvCols;
  if (t <= 0 || t > kTileMax || c0 >= t) return;
  double *S = sm;                                       // packed tile
  double *rdiag = sm + kTileMax * (kTileMax + 1) / 2;   // 1 / T_ii
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double *x = rdiag + kTileMax + warp * kTileMax;       // this warp's column
  tile_load(S, d.L, d.ldl, t);
  __syncthreads();
  for (int i = threadIdx.x; i < t; i += blockDim.x) rdiag[i] = 1.0 / S[pk(i, i)];
  __syncthreads();
  const int c = c0 + warp;
  if (c < t) {
    for (int i = lane; i < c; i += 32) x[i] = 0.0;
    if (lane == 0) x[c] = rdiag[c];
    __syncwarp();
    for (int i = c + 1; i < t; ++i) {
      double s0 = 0.0;
      for (int k = c + lane; k < i; k += 32) s0 = fma(S[pk(i, k)], x[k], s0);
      s0 = warp_sum(s0);
      if (lane == 0) x[i] = -s0 * rdiag[i];
      __syncwarp();
    }
    for (int i = lane; i < t; i += 32) d.inv[(long long)i * d.ldinv + c] = x[i];
  }
}

cudaError_t launch_trtri_group(const TileGroup &g, cudaStream_t s) {
  if (g.count <= 0) return cudaSuccess;
  int tmax = 0;
  for (int p = 0; p < g.count; ++p) tmax = std::max(tmax, g.d[p].t);
  if (tmax <= 0) return cudaSuccess;
  const dim3 grid((unsigned)((tmax + kInvCols - 1) / kInvCols), (unsigned)g.count);
  k_trtri_cols<<<grid, 32 * kInvCols, kInvSmem, s>>>(g);
  return cudaGetLastError();
}

cudaError_t tile_kernels_init() {
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_tile<T_POTF2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTileSmem)))
    return e;
  if ((e = cudaFuncSetAttribute(k_tile<T_REV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTileSmem)))
    return e;
  if ((e = cudaFuncSetAttribute(k_tile<T_SENS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTileSmem)))
    return e;
  if ((e = cudaFuncSetAttribute(k_trtri_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kInvSmem))) return e;
  return cudaSuccess;
}

cudaError_t launch_tile_group(TileOp op, const TileGroup &g, cudaStream_t s) {
  if (g.count <= 0) return cudaSuccess;
  switch (op) {
    case T_POTF2: k_tile<T_POTF2><<<g.count, kTileThreads, kTileSmem, s>>>(g); break;
    case T_REV: k_tile<T_REV><<<g.count, kTileThreads, kTileSmem, s>>>(g); break;
    case T_SENS: k_tile<T_SENS><<<g.count, kTileThreads, kTileSmem, s>>>(g); break;
    case T_TRTRI: return launch_trtri_group(g, s);
    default: return cudaErrorInvalidValue;
  }
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

cudaError_t launch_mirror_lower(double *A, long long lda, int n, cudaStream_t s) {
  if (n <= 1) return cudaSuccess;
  const int nt = (n + 31) / 32;
  k_mirror<<<dim3(nt, nt), dim3(32, 8), 0, s>>>(A, lda, n);
  return cudaGetLastError();
}

}  // namespace cd
