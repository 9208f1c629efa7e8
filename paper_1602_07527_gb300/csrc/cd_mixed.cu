// Mixed-precision engine of libcholdiff: split-BF16 products on the sm_103a
// tensor cores (tcgen05.mma, accumulator in tensor memory), operands staged by
// TMA (cp.async.bulk.tensor) through a multi-stage mbarrier pipeline.
//
// Used for the large off-diagonal products of the blocked algorithms
// (Sec. 4.2: the panel solves as products with the FP64 inverse of the
// diagonal block, and the GEMM / SYRK trailing updates); the diagonal-tile
// work stays in FP64 (cd_f64_kernels.cu).
//
// One CTA computes a 128 x 128 output tile over its K range:
//   warp 0, lane 0   issues the TMA loads of all terms of A and B per 64-wide K block;
//   warp 1, lane 0   issues tcgen05.mma for every term product of the block
//                    (leading product and corrections in two accumulators);
//   warps 0-3        drain the FP32 accumulator from tensor memory (tcgen05.ld),
//                    stage it in shared memory as FP64, and write
//                    beta * Cin + alpha * acc (or a split-K partial) with
//                    coalesced FP64 stores.
// Every wait on an mbarrier gives up after 2 s of %globaltimer, sets the
// caller's device error word to CD_ETIMEOUT and lets the CTA finish.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>

#include "cd_internal.h"
#include "cd_mixed.h"
#include "cd_tc.cuh"
#include "cd_split_terms.cuh"

namespace cd {
namespace {

using namespace tc;

constexpr int BM = 128, BN = 128, BK = 64;
constexpr int kEpiWarps = 8;                  // epilogue warps: two per tensor-memory lane quarter
constexpr int kThreads = 64 + 32 * kEpiWarps;  // warp 0 TMA, warp 1 MMA, warps 2-9 epilogue
constexpr uint32_t kTileBytes = BM * BK * 2;  // one term of one operand per K block (BM == BN)
constexpr int kMaxM = 10;

struct MDesc {  // 64-byte aligned through CUtensorMap
  CUtensorMap ta, tb;
  const double *Cin;
  double *Cout;
  float *part;  // split-K partial sums (FP32, as accumulated)
  long long ldcin, ldcout;
  double alpha, beta;
  int M, N, K, splits, kchunk;
  int tiles_m, tiles_n, tile_begin;
  int ax, ay, bx, by;
  int comb;     // a Comb value
  int vec;      // Cout (and Cin if read) 16-byte aligned with even leading dimensions: 16-byte accesses
};

struct MGroup {
  int count, total_tiles, lower;
  int tx_extra;  // test hook: bytes the first load barrier expects beyond the copy (0 in production)
  int *err;
  MDesc d[kMaxM];
};
static_assert(sizeof(MGroup) <= 4096, "kernel parameter block too large");

// Instruction descriptor, kind::f16: D = F32 (bits 4-5 = 1), A = B = BF16
// (bits 7-9 = 1, 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                            ((uint32_t)(BM >> 4) << 24);


// The epilogue stages each warp's accumulators 32 rows x kEpiCols columns at
// a time (lane = row on the way in), so that the output can be written with
// consecutive lanes on consecutive columns.  16 columns keep the staging at
// 17 KB per CTA, which leaves room on the SM for an FP64 CTA of the diagonal
// chain to run beside a tensor-core product.
constexpr int kEpiCols = 16;
constexpr int kEpiLd = kEpiCols + 1;

// Writes the staged rows rr = r0 + 2 k (k < 16, rr < nrows) of one output
// column j (rows rbase + rr) from the FP32 staging column stw[rr * ld],
// forming each value under mode COMB.
template <int COMB, bool LOWER>
__device__ __forceinline__ void write_column(const MDesc &d, const float *stw, int ld, int rbase, int nrows, int j,
                                             int r0) {
  constexpr bool kUseCin = COMB >= kAdd;
  double cin[16];
  const double *ci = d.Cin + (long long)(rbase + r0) * d.ldcin + j;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int rr = r0 + 2 * k;
    cin[k] = (kUseCin && rr < nrows && !(LOWER && j > rbase + rr)) ? ci[0] : 0.0;
    ci += 2 * d.ldcin;
  }
  double *co = d.Cout + (long long)(rbase + r0) * d.ldcout + j;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int rr = r0 + 2 * k;
    if (rr < nrows && !(LOWER && j > rbase + rr)) *co = combine<COMB>(f32_to_f64(stw[rr * ld]), cin[k], d.alpha, d.beta);
    co += 2 * d.ldcout;
  }
}

// The same for the staged 32 x 16 block in 16-byte accesses: lane l covers
// columns j0 + 2 (l % 8) + {0, 1} of rows l / 8 + 4 k (Cout, Cin 16-byte
// aligned, even leading dimensions, j0 even).  Non-LOWER tiles only.
template <int COMB>
__device__ __forceinline__ void write_block_v2(const MDesc &d, const float *stw, int ld, int rbase, int nrows, int j0,
                                               int ncols, int lane) {
  constexpr bool kUseCin = COMB >= kAdd;
  const int c = 2 * (lane & 7), h = lane >> 3;
  const bool col_ok = c < ncols;  // ncols even here
  double2 cin[8];
  const double *ci = d.Cin + (long long)(rbase + h) * d.ldcin + j0 + c;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    cin[k] = make_double2(0.0, 0.0);
    if (kUseCin && col_ok && 4 * k + h < nrows) cin[k] = *reinterpret_cast<const double2 *>(ci);
    ci += 4 * d.ldcin;
  }
  double *co = d.Cout + (long long)(rbase + h) * d.ldcout + j0 + c;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int rr = 4 * k + h;
    if (col_ok && rr < nrows) {
      double2 v;
      v.x = combine<COMB>(f32_to_f64(stw[rr * ld + c]), cin[k].x, d.alpha, d.beta);
      v.y = combine<COMB>(f32_to_f64(stw[rr * ld + c + 1]), cin[k].y, d.alpha, d.beta);
      *reinterpret_cast<double2 *>(co) = v;
    }
    co += 4 * d.ldcout;
  }
}

__device__ __forceinline__ void write_block_v2_any(int comb, const MDesc &d, const float *stw, int ld, int rbase,
                                                   int nrows, int j0, int ncols, int lane) {
  switch (comb) {
    case kCopy: write_block_v2<kCopy>(d, stw, ld, rbase, nrows, j0, ncols, lane); break;
    case kNeg: write_block_v2<kNeg>(d, stw, ld, rbase, nrows, j0, ncols, lane); break;
    case kScale: write_block_v2<kScale>(d, stw, ld, rbase, nrows, j0, ncols, lane); break;
    case kAdd: write_block_v2<kAdd>(d, stw, ld, rbase, nrows, j0, ncols, lane); break;
    case kSub: write_block_v2<kSub>(d, stw, ld, rbase, nrows, j0, ncols, lane); break;
    case kAxpy: write_block_v2<kAxpy>(d, stw, ld, rbase, nrows, j0, ncols, lane); break;
    default: write_block_v2<kGeneral>(d, stw, ld, rbase, nrows, j0, ncols, lane); break;
  }
}

template <bool LOWER>
__device__ __forceinline__ void write_column_any(int comb, const MDesc &d, const float *stw, int ld, int rbase,
                                                 int nrows, int j, int r0) {
  switch (comb) {
    case kCopy: write_column<kCopy, LOWER>(d, stw, ld, rbase, nrows, j, r0); break;
    case kNeg: write_column<kNeg, LOWER>(d, stw, ld, rbase, nrows, j, r0); break;
    case kScale: write_column<kScale, LOWER>(d, stw, ld, rbase, nrows, j, r0); break;
    case kAdd: write_column<kAdd, LOWER>(d, stw, ld, rbase, nrows, j, r0); break;
    case kSub: write_column<kSub, LOWER>(d, stw, ld, rbase, nrows, j, r0); break;
    case kAxpy: write_column<kAxpy, LOWER>(d, stw, ld, rbase, nrows, j, r0); break;
    default: write_column<kGeneral, LOWER>(d, stw, ld, rbase, nrows, j, r0); break;
  }
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t acc) {
  mma_bf16_id(tmem_d, adesc, bdesc, kIdesc, acc);
}

template <int T>
struct Terms;
// Term products kept, smallest first: T = 2 keeps t1 t0, t0 t1, t0 t0.
template <>
struct Terms<2> {
  static constexpr int n = 3;
  __device__ static int a(int q) { return q == 0 ? 1 : 0; }
  __device__ static int b(int q) { return q == 1 ? 1 : 0; }
};
// T = 3 keeps t1 t1, t2 t0, t0 t2, t1 t0, t0 t1, t0 t0.
template <>
struct Terms<3> {
  static constexpr int n = 6;
  __device__ static int a(int q) {
    const int v[6] = {1, 2, 0, 1, 0, 0};
    return v[q];
  }
  __device__ static int b(int q) {
    const int v[6] = {1, 0, 2, 0, 1, 0};
    return v[q];
  }
};

template <int T>
__host__ __device__ constexpr int stages() {
  return T == 2 ? 3 : 2;
}
template <int T>
__host__ __device__ constexpr uint32_t stage_bytes() {
  return 2u * T * kTileBytes;
}
// Epilogue staging: one 32 x kEpiCols FP32 block per epilogue warp (padded rows).
constexpr size_t kEpiBytes = (size_t)kEpiWarps * 32 * kEpiLd * sizeof(float);
template <int T>
constexpr size_t dyn_smem() {
  return (size_t)stages<T>() * stage_bytes<T>() + kEpiBytes + 1024;
}
static_assert(dyn_smem<2>() <= 232448 && dyn_smem<3>() <= 232448, "shared memory per CTA");

// One output tile of one problem: the work of a CTA for a while.
struct Unit {
  int p, z, m0, n0, kbeg, nkb;
};

template <bool LOWER>
__device__ __forceinline__ Unit decode_unit(const MGroup &g, int u) {
  Unit x;
  int p = 0;
  while (p + 1 < g.count && u >= g.d[p + 1].tile_begin) ++p;
  const MDesc &d = g.d[p];
  const int local = u - d.tile_begin;
  const int per_split = LOWER ? d.tiles_m * (d.tiles_m + 1) / 2 : d.tiles_m * d.tiles_n;
  x.p = p;
  x.z = local / per_split;
  const int rem = local - x.z * per_split;
  if (LOWER) {
    int ti = (int)((sqrtf(8.0f * rem + 1.0f) - 1.0f) * 0.5f);
    while ((ti + 1) * (ti + 2) / 2 <= rem) ++ti;
    while (ti * (ti + 1) / 2 > rem) --ti;
    x.m0 = ti * BM;
    x.n0 = (rem - ti * (ti + 1) / 2) * BN;
  } else {
    x.m0 = (rem / d.tiles_n) * BM;
    x.n0 = (rem % d.tiles_n) * BN;
  }
  x.kbeg = x.z * d.kchunk;
  const int kend = min(d.K, x.kbeg + d.kchunk);
  x.nkb = kend > x.kbeg ? (kend - x.kbeg + BK - 1) / BK : 0;
  return x;
}

// Persistent, warp-specialised product.  A CTA takes the units
// blockIdx.x, blockIdx.x + gridDim.x, ... of the group:
//   warp 0        lane 0 streams every unit's K blocks through the stage ring
//                 with TMA; the whole warp first pulls the unit's Cin rows
//                 into L2 for the epilogue;
//   warp 1        lane 0 issues the tcgen05.mma of each unit into one of two
//                 tensor-memory accumulator sets (256 columns each: leading
//                 product and corrections), alternating between units;
//   warps 2-9     drain a finished accumulator set (each warp 32 tensor
//                 memory lanes, i.e. rows, and half of the columns, loaded
//                 32 at a time and staged 16 at a time through shared
//                 memory) and write the FP64 output or
//                 FP32 split-K partials, while the MMA warp already fills the
//                 other set.  Two warps per sub-partition hide each other's
//                 load and store latency.
//
// At most 128 registers a thread (no spills): a sub-partition that holds
// three of the ten warps then keeps 4K registers free, room for a warp of an
// FP64 chain kernel or a reduction beside the product.
template <int T, bool LOWER>
__global__ void __maxnreg__(128) k_mgemm(const __grid_constant__ MGroup g) {
  constexpr int S = stages<T>();
  constexpr uint32_t SB = stage_bytes<T>();
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  float *epi = (float *)(smem + (size_t)S * SB);
  __shared__ __align__(8) uint64_t full_bar[S];
  __shared__ __align__(8) uint64_t empty_bar[S];
  __shared__ __align__(8) uint64_t tfull_bar[2];
  __shared__ __align__(8) uint64_t tempty_bar[2];
  __shared__ __align__(8) uint64_t drain_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int s_err;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int units = g.total_tiles;
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull_bar[b], 1);
      mbar_init(&tempty_bar[b], kEpiWarps);
    }
    mbar_init(&drain_bar, 1);
    s_err = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {  // all of tensor memory: two accumulator sets of 2 x BN columns
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(4 * BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp == 0) {
    uint32_t it = 0;  // K blocks issued by this CTA, over all its units
    bool ok = true;
    uint32_t last_it[S];
#pragma unroll
    for (int s = 0; s < S; ++s) last_it[s] = 0xFFFFFFFFu;
    for (int u = blockIdx.x; u < units && ok; u += gridDim.x) {
      const Unit x = decode_unit<LOWER>(g, u);
      const MDesc &d = g.d[x.p];
      if (d.splits == 1 && d.comb >= kAdd) {
        const int rows = min(BM, d.M - x.m0), cols = min(BN, d.N - x.n0);
        for (int r = lane; r < rows; r += 32) {
          const char *p0 = (const char *)(d.Cin + (long long)(x.m0 + r) * d.ldcin + x.n0);
          for (int o = 0; o < cols * 8; o += 128) asm volatile("prefetch.global.L2 [%0];" ::"l"(p0 + o));
          asm volatile("prefetch.global.L2 [%0];" ::"l"(p0 + cols * 8 - 8));
        }
      }
      if (lane == 0) {
        for (int kb = 0; kb < x.nkb; ++kb, ++it) {
          const int s = (int)(it % S);
          if (it >= (uint32_t)S && !mbar_wait_or_abort(&empty_bar[s], ((it / S) - 1) & 1u, &s_err)) {
            s_err = 1;
            ok = false;
            break;
          }
          uint8_t *sa = smem + s * SB;
          uint8_t *sb = sa + T * kTileBytes;
          mbar_expect_tx(&full_bar[s], SB + (it == 0 ? (uint32_t)g.tx_extra : 0u));
          const int kx = x.kbeg + kb * BK;
          tma_load_3d(sa, &d.ta, d.ax + kx, d.ay + x.m0, 0, &full_bar[s]);
          tma_load_3d(sb, &d.tb, d.bx + kx, d.by + x.n0, 0, &full_bar[s]);
          last_it[s] = it;
        }
      }
      ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
    }
    if (lane == 0 && !ok) {
      // failure: let copies still in flight land before the CTA exits (bounded)
      for (int s = 0; s < S; ++s)
        if (last_it[s] != 0xFFFFFFFFu) {
          const unsigned long long t0 = globaltimer();
          while (!mbar_try_wait(&full_bar[s], (last_it[s] / S) & 1u) && globaltimer() - t0 < kTimeoutNs / 8) {
          }
        }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      uint32_t it = 0;
      int t = 0;
      bool issued = false;
      for (int u = blockIdx.x; u < units; u += gridDim.x, ++t) {
        const Unit x = decode_unit<LOWER>(g, u);
        const int b = t & 1;
        if (t >= 2 && !mbar_wait_or_abort(&tempty_bar[b], (uint32_t)((t >> 1) - 1) & 1u, &s_err)) {
          s_err = 1;
          break;
        }
        tc_fence_after();
        const uint32_t acc = tmem + (uint32_t)(b * 2 * BN);
        int issued_main = 0, issued_corr = 0;
        bool ok = true;
        for (int kb = 0; kb < x.nkb; ++kb, ++it) {
          const int s = (int)(it % S);
          if (!mbar_wait_or_abort(&full_bar[s], (it / S) & 1u, &s_err)) {
            s_err = 1;
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = smem_u32(smem + s * SB);
          const uint32_t sb = sa + T * kTileBytes;
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk) {
#pragma unroll
            for (int q = 0; q < Terms<T>::n; ++q) {
              const int ta = Terms<T>::a(q), tb = Terms<T>::b(q);
              const uint64_t ad = sw128_desc(sa + ta * kTileBytes + kk * 32);
              const uint64_t bd = sw128_desc(sb + tb * kTileBytes + kk * 32);
              if (ta == 0 && tb == 0) {
                mma_bf16(acc, ad, bd, issued_main ? 1u : 0u);
                issued_main = 1;
              } else {
                mma_bf16(acc + BN, ad, bd, issued_corr ? 1u : 0u);
                issued_corr = 1;
              }
            }
          }
          issued = true;
          mma_commit(&empty_bar[s]);
        }
        if (!ok) break;
        mma_commit(&tfull_bar[b]);
      }
      if (s_err && issued) {  // failure: products already issued finish before tensor memory is freed
        mma_commit(&drain_bar);
        mbar_wait(&drain_bar, 0);
      }
    }
    __syncwarp();
  } else {
    // Epilogue.  Tensor-memory lanes are reachable from warp w in quarter w % 4.
    const int qd = warp & 3;
    const int half = (warp - 2) / 4;  // columns [64 half, 64 half + 64)
    float *stw = epi + (size_t)(warp - 2) * 32 * kEpiLd;
    int t = 0;
    for (int u = blockIdx.x; u < units; u += gridDim.x, ++t) {
      const Unit x = decode_unit<LOWER>(g, u);
      const MDesc &d = g.d[x.p];
      const int b = t & 1;
      const bool got = mbar_wait_or_abort(&tfull_bar[b], (uint32_t)(t >> 1) & 1u, &s_err);
      if (!__all_sync(0xffffffffu, got)) {
        s_err = 1;
        break;
      }
      tc_fence_after();
      const uint32_t acc = tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)(b * 2 * BN);
      const int rbase = x.m0 + qd * 32;  // this warp's 32 rows
      const int nrows = max(0, min(32, d.M - rbase));
      const int comb = d.comb;
#pragma unroll 1
      for (int c0 = half * (BN / 2); c0 < (half + 1) * (BN / 2); c0 += 32) {
        uint32_t r[32], q[32];
        tmem_ld32(acc + (uint32_t)c0, r);
        tmem_ld32(acc + (uint32_t)(BN + c0), q);
#pragma unroll
        for (int hh = 0; hh < 32 / kEpiCols; ++hh) {
#pragma unroll
          for (int i = 0; i < kEpiCols; ++i)
            stw[lane * kEpiLd + i] =
                x.nkb > 0 ? __uint_as_float(r[hh * kEpiCols + i]) + __uint_as_float(q[hh * kEpiCols + i]) : 0.0f;
          __syncwarp();
          // lane % 16 = output column, lane / 16 = row parity: coalesced row segments
          const int j0 = x.n0 + c0 + hh * kEpiCols, col = lane & 15, r0 = lane >> 4, j = j0 + col;
          const int ncols = min(kEpiCols, d.N - j0);
          if (d.splits > 1) {
            if (j < d.N)
              for (int rr = r0; rr < nrows; rr += 2) {
                const int i = rbase + rr;
                if (!(LOWER && j > i)) d.part[((long long)x.z * d.M + i) * d.N + j] = stw[rr * kEpiLd + col];
              }
          } else if (d.vec && !(LOWER && x.m0 == x.n0) && (ncols & 1) == 0) {
            if (ncols > 0) write_block_v2_any(comb, d, stw, kEpiLd, rbase, nrows, j0, ncols, lane);
          } else if (j < d.N) {
            write_column_any<LOWER>(comb, d, stw + col, kEpiLd, rbase, nrows, j, r0);
          }
          __syncwarp();
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty_bar[b]);
    }
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(4 * BN) : "memory");
  }
  if (threadIdx.x == 0 && s_err && g.err) atomicExch(g.err, CD_ETIMEOUT);
}

// Split-K reduction: the FP32 partials, in order, by compensated summation
// in FP32 (Neumaier's variant of Kahan summation: the rounding error of each
// addition, obtained exactly, is carried in c), then s + c to FP64 and the
// output formed as in the product's epilogue (mode fixed per loop, as there).
template <int COMB, bool LOWER>
__device__ __forceinline__ void reduce_loop(const MDesc &d) {
  const long long total = (long long)d.M * d.N;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / d.N), j = (int)(e - (long long)i * d.N);
    if (LOWER && j > i) continue;
    float s = 0.0f, c = 0.0f;
    for (int z = 0; z < d.splits; ++z) {
      const float x = d.part[(long long)z * total + e];
      const float t = s + x;
      c += fabsf(s) >= fabsf(x) ? (s - t) + x : (x - t) + s;
      s = t;
    }
    const double a = f32_to_f64(s) + f32_to_f64(c);
    const double cin = COMB >= kAdd ? d.Cin[(long long)i * d.ldcin + j] : 0.0;
    d.Cout[(long long)i * d.ldcout + j] = combine<COMB>(a, cin, d.alpha, d.beta);
  }
}

template <bool LOWER>
__global__ void k_mreduce(const __grid_constant__ MGroup g) {
  const MDesc &d = g.d[blockIdx.y];
  if (d.splits <= 1) return;
  switch (d.comb) {
    case kCopy: reduce_loop<kCopy, LOWER>(d); break;
    case kNeg: reduce_loop<kNeg, LOWER>(d); break;
    case kScale: reduce_loop<kScale, LOWER>(d); break;
    case kAdd: reduce_loop<kAdd, LOWER>(d); break;
    case kSub: reduce_loop<kSub, LOWER>(d); break;
    case kAxpy: reduce_loop<kAxpy, LOWER>(d); break;
    default: reduce_loop<kGeneral, LOWER>(d); break;
  }
}

// FP64 -> T BF16 terms.  x is first cut exactly into FP32 pieces hi + lo
// (integer operations, no FP64 instruction); t0 is the BF16 nearest to hi,
// and each further term the BF16 nearest to the remainder so far,
// (hi - t0 - ...) + lo, formed in FP32: hi - t0 is exact, and adding lo
// rounds at 2^-24 of the remainder, far below the last term kept.
//
// split_load: the FP32 pieces hi + lo of destination element (rr, cc) of a
// split, the source value it views or zero outside the view (padding).
__device__ __forceinline__ void split_load(const SplitArgs &a, int rr, int cc, float &hi, float &lo) {
  const int vr_n = a.transpose ? a.cols : a.rows;  // view extent in destination coordinates
  const int vc_n = a.transpose ? a.rows : a.cols;
  const int vr = a.reg_r0 + rr - a.dst_r0, vc = a.reg_c0 + cc - a.dst_c0;
  hi = 0.0f;
  lo = 0.0f;
  if (vr >= 0 && vc >= 0 && vr < vr_n && vc < vc_n) {
    const int r = a.transpose ? vc : vr, c = a.transpose ? vr : vc;
    const bool upper = r < c;
    if (a.mode == 0 || !upper || a.mode == 2) {
      const long long off = upper && a.mode == 2 ? (long long)c * a.lds + r : (long long)r * a.lds + c;
      f64_to_f32x2(a.src[off], hi, lo);
      if (a.mode == 2 && r == c) {  // doubled diagonal: exact in FP32
        hi *= 2.0f;
        lo *= 2.0f;
      }
    }
  }
}

// The T BF16 terms of one element from its FP32 pieces.
__device__ __forceinline__ void split_store(const SplitArgs &a, int rr, int cc, float hi, float lo) {
  write_split_terms((__nv_bfloat16 *)a.dst, a.dst_rows * a.ldd, (long long)(a.reg_r0 + rr) * a.ldd + a.reg_c0 + cc,
                    hi, lo, a.T);
}

// cuTensorMapEncodeTiled is a driver entry point; it is looked up through the
// runtime (no link-time dependency on the driver library).
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn g_encode = nullptr;

constexpr int kMaxSplit = 36;
struct SplitGroup {
  int count, pad_;
  SplitArgs a[kMaxSplit];
};
static_assert(sizeof(SplitGroup) <= 4096, "kernel parameter block too large");

// Several splits, in 32 x 32 destination tiles (one split per blockIdx.y).
// A transposed split reads its source tile row by row (coalesced: consecutive
// threads take consecutive source columns) into shared memory and writes the
// destination rows from there, so that both sides are contiguous.  The 8 KB
// tile fits beside a tensor-core product's CTA on one SM.
constexpr int kSplitTR = 32, kSplitTC = 32, kSplitThreads = 256;
__global__ void __launch_bounds__(kSplitThreads) k_split_group(const __grid_constant__ SplitGroup g) {
  const SplitArgs &a = g.a[blockIdx.y];
  __shared__ float sh[2][kSplitTC][kSplitTR + 1];
  const int tiles_c = (a.dst_w + kSplitTC - 1) / kSplitTC;
  const int tiles = ((a.dst_h + kSplitTR - 1) / kSplitTR) * tiles_c;
  for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
    const int rr0 = (t / tiles_c) * kSplitTR, cc0 = (t % tiles_c) * kSplitTC;
    const int h = min(kSplitTR, a.dst_h - rr0), w = min(kSplitTC, a.dst_w - cc0);
    if (a.transpose) {
      for (int e = threadIdx.x; e < kSplitTR * kSplitTC; e += kSplitThreads) {
        const int cc = e / kSplitTR, rr = e - cc * kSplitTR;
        float hi = 0.0f, lo = 0.0f;
        if (rr < h && cc < w) split_load(a, rr0 + rr, cc0 + cc, hi, lo);
        sh[0][cc][rr] = hi;
        sh[1][cc][rr] = lo;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < kSplitTR * kSplitTC; e += kSplitThreads) {
        const int rr = e / kSplitTC, cc = e - rr * kSplitTC;
        if (rr < h && cc < w) split_store(a, rr0 + rr, cc0 + cc, sh[0][cc][rr], sh[1][cc][rr]);
      }
      __syncthreads();
    } else {
      for (int e = threadIdx.x; e < kSplitTR * kSplitTC; e += kSplitThreads) {
        const int rr = e / kSplitTC, cc = e - rr * kSplitTC;
        if (rr < h && cc < w) {
          float hi, lo;
          split_load(a, rr0 + rr, cc0 + cc, hi, lo);
          split_store(a, rr0 + rr, cc0 + cc, hi, lo);
        }
      }
    }
  }
}

bool encode_map(CUtensorMap *m, const MOp &op) {
  if (!g_encode) return false;
  if (!op.base || (op.ld % 64) != 0 || ((uintptr_t)op.base % 16) != 0 || op.rows <= 0 || op.T < 2 || op.T > 3)
    return false;
  cuuint64_t dims[3] = {(cuuint64_t)op.ld, (cuuint64_t)op.rows, (cuuint64_t)op.T};
  cuuint64_t strides[2] = {(cuuint64_t)op.ld * 2, (cuuint64_t)op.ld * 2 * (cuuint64_t)op.rows};
  cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)BM, (cuuint32_t)op.T};
  cuuint32_t estr[3] = {1, 1, 1};
  return g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(op.base), dims, strides,
                                box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}


int sm_count() {
  static int cached[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
  if (cached[dev] == 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
    cached[dev] = n;
  }
  return cached[dev];
}

template <int T, bool LOWER>
cudaError_t launch_one(const MGroup &g, cudaStream_t s, int max_units) {
  const int units = g.total_tiles;
  const int grid = std::min(units, std::max(sm_count(), (units + max_units - 1) / max_units));
  k_mgemm<T, LOWER><<<grid, kThreads, dyn_smem<T>(), s>>>(g);
  return cudaGetLastError();
}

// Per device: function attributes (the dynamic shared-memory limit) are set
// on the current device.
constexpr int kMaxDev = 64;
bool g_ready[kMaxDev];

int current_device() {
  int dev = -1;
  return cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < kMaxDev ? dev : -1;
}

}  // namespace

int mixed_init() {
  const int dev = current_device();
  if (dev < 0) return CD_ECUDA;
  if (g_ready[dev]) return CD_OK;
  void *fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || fn == nullptr) {
    cudaGetLastError();
    return CD_ECUDA;
  }
  g_encode = (EncodeTiledFn)fn;
  cudaError_t e = cudaSuccess;
  e = cudaFuncSetAttribute(k_mgemm<2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_smem<2>());
  if (!e) e = cudaFuncSetAttribute(k_mgemm<2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_smem<2>());
  if (!e) e = cudaFuncSetAttribute(k_mgemm<3, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_smem<3>());
  if (!e) e = cudaFuncSetAttribute(k_mgemm<3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_smem<3>());
  // the reductions and splits run beside the products: same (largest) shared-memory carveout
  const int carve = cudaSharedmemCarveoutMaxShared;
  if (!e) e = cudaFuncSetAttribute(k_mreduce<true>, cudaFuncAttributePreferredSharedMemoryCarveout, carve);
  if (!e) e = cudaFuncSetAttribute(k_mreduce<false>, cudaFuncAttributePreferredSharedMemoryCarveout, carve);
  if (!e) e = cudaFuncSetAttribute(k_split_group, cudaFuncAttributePreferredSharedMemoryCarveout, carve);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return CD_ECUDA;
  }
  g_ready[dev] = true;
  return CD_OK;
}

bool mixed_available() {
  const int dev = current_device();
  return dev >= 0 && g_ready[dev];
}

int mixed_ctas_per_sm() { return 1; }

size_t mixed_workspace_bytes(int n, int nb, int prec) {
  if (prec == CD_FP64 || n <= 0) return 0;
  const int T = prec == CD_MIXED_BF16X6 ? 3 : 2;
  const size_t nbp = (size_t)((std::max(nb, 64) + 63) / 64 * 64);
  const size_t ldb = (size_t)((n + 8 + 63) / 64 * 64), ldn = (size_t)((n + 63) / 64 * 64 + 64);
  const size_t e = 2 * (size_t)n * ldb + (size_t)n * nbp + 2 * nbp * ldn + nbp * nbp;
  return 2 * T * e + 16 * 256;
}

cudaError_t mixed_gemm_launch(const MProblem *probs, int count, int T, bool lower, int *dev_err, cudaStream_t s,
                              int *launches, int tx_extra, int max_units) {
  max_units = std::max(1, max_units);
  if (T != 2 && T != 3) return cudaErrorInvalidValue;
  int i = 0;
  while (i < count) {
    MGroup g;
    memset(&g, 0, sizeof(g));
    g.lower = lower ? 1 : 0;
    g.err = dev_err;
    g.tx_extra = tx_extra;
    bool any_split = false;
    long long biggest = 0;
    for (; i < count && g.count < kMaxM; ++i) {
      const MProblem &P = probs[i];
      if (P.M <= 0 || P.N <= 0 || P.K <= 0) continue;
      if ((P.A.x0 % 8) || (P.B.x0 % 8) || P.A.x0 < 0 || P.B.x0 < 0 || P.A.y0 < 0 || P.B.y0 < 0 ||
          (P.kchunk % BK) || P.kchunk <= 0 || P.A.T != T || P.B.T != T || (lower && P.M != P.N))
        return cudaErrorInvalidValue;
      MDesc &d = g.d[g.count];
      if (!encode_map(&d.ta, P.A) || !encode_map(&d.tb, P.B)) return cudaErrorInvalidValue;
      d.Cin = P.Cin;
      d.Cout = P.Cout;
      d.part = reinterpret_cast<float *>(P.part);  // the region holds splits * M * N doubles: ample for floats
      d.comb = P.beta == 0.0 ? (P.alpha == 1.0 ? kCopy : P.alpha == -1.0 ? kNeg : kScale)
               : P.beta == 1.0 ? (P.alpha == 1.0 ? kAdd : P.alpha == -1.0 ? kSub : kAxpy)
                               : kGeneral;
      d.vec = ((uintptr_t)P.Cout % 16 == 0) && (P.ldcout % 2 == 0) &&
              (d.comb < kAdd || (((uintptr_t)P.Cin % 16 == 0) && (P.ldcin % 2 == 0)));
      d.ldcin = P.ldcin;
      d.ldcout = P.ldcout;
      d.alpha = P.alpha;
      d.beta = P.beta;
      d.M = P.M;
      d.N = P.N;
      d.K = P.K;
      d.splits = P.splits;
      d.kchunk = P.kchunk;
      d.tiles_m = (P.M + BM - 1) / BM;
      d.tiles_n = (P.N + BN - 1) / BN;
      d.tile_begin = g.total_tiles;
      d.ax = P.A.x0;
      d.ay = P.A.y0;
      d.bx = P.B.x0;
      d.by = P.B.y0;
      const int per = lower ? d.tiles_m * (d.tiles_m + 1) / 2 : d.tiles_m * d.tiles_n;
      g.total_tiles += per * P.splits;
      if (P.splits > 1) {
        any_split = true;
        biggest = std::max(biggest, (long long)P.M * P.N);
      }
      ++g.count;
    }
    if (g.count == 0) continue;
    cudaError_t e;
    if (T == 2)
      e = lower ? launch_one<2, true>(g, s, max_units) : launch_one<2, false>(g, s, max_units);
    else
      e = lower ? launch_one<3, true>(g, s, max_units) : launch_one<3, false>(g, s, max_units);
    if (launches) ++*launches;
    if (e != cudaSuccess) return e;
    if (any_split) {
      long long blocks = std::min<long long>(1024, (biggest + 255) / 256);
      dim3 grid((unsigned)blocks, (unsigned)g.count);
      if (lower)
        k_mreduce<true><<<grid, 256, 0, s>>>(g);
      else
        k_mreduce<false><<<grid, 256, 0, s>>>(g);
      if (launches) ++*launches;
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

cudaError_t mixed_split_group_launch(const SplitArgs *a, int count, cudaStream_t s, int *launches) {
  int i = 0;
  while (i < count) {
    SplitGroup g;
    memset(&g, 0, sizeof(g));
    long long biggest = 0;
    for (; i < count && g.count < kMaxSplit; ++i) {
      if ((long long)a[i].dst_h * a[i].dst_w <= 0) continue;
      if (a[i].T < 2 || a[i].T > 3 || !a[i].dst) return cudaErrorInvalidValue;
      g.a[g.count++] = a[i];
      biggest = std::max(biggest, (long long)((a[i].dst_h + kSplitTR - 1) / kSplitTR) *
                                      ((a[i].dst_w + kSplitTC - 1) / kSplitTC));
    }
    if (g.count == 0) continue;
    const long long blocks = std::max<long long>(1, std::min<long long>(4096, biggest));  // biggest: tiles
    k_split_group<<<dim3((unsigned)blocks, (unsigned)g.count), kSplitThreads, 0, s>>>(g);
    if (launches) ++*launches;
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}


}  // namespace cd
