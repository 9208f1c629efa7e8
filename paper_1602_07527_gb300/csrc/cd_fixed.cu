// Fixed-point-slice products on the sm_103a tensor cores: the accurate mode
// of libcholdiff's mixed precision (CD_MIXED_FIXED4).
//
// The split-BF16 products of cd_mixed.cu keep every operand element as its
// own floating BF16 terms and accumulate in FP32: about FP32 accuracy.  The
// blocked factorisation (Sec. 4.2, chol_blocked: the Schur updates of the
// diagonal block and the panel, and the panel solve) amplifies that error by
// the conditioning of Sigma.  Here the operands are cut instead into
// fixed-point slices that share one exponent per row (the splitting of
// Ozaki and co-workers), so that the leading partial sums are exact:
//
//   row r of an operand has an exponent E_r with |x| < 2^E_r for each of its
//   elements; x = 2^(E_r - 7) (b_0 + b_1 + b_2 + b_3) up to 2^(E_r - 32),
//   with b_s = a_s 2^(-8 s) and each a_s an integer in [-128, 128] (exact in
//   BF16).  Then for C = A B^T (row exponents E_i of A, F_j of B):
//
//     C_ij = 2^(E_i + F_j - 14) (acc0 + acc1 + acc2 + acc3),
//     acc0 = sum_k b_0 c_0                 integers, |acc0| <= 2^22 per window
//     acc1 = sum_k (b_0 c_1 + b_1 c_0)     multiples of 2^-8, below 2^23 of them
//     acc2 = sum_k over s + t = 2          multiples of 2^-16, below 3 2^22 of them
//     acc3 = sum_k over s + t in {3, 4}    FP32, below 2^-24 of acc0's scale
//
//   over windows of 256 of K, so acc0-acc2 are exact in FP32 whatever
//   the order and rounding of the tensor core's additions (every partial sum
//   is an integer multiple of the last place below 2^24 units).  Each window
//   ends with the four accumulators added (acc3 floored at 2^-32) into a
//   64-bit integer in units of 2^-32 held in the epilogue's registers; the
//   last window converts it to FP64 (one rounding) and forms the output.
//   Thirteen slice products per multiply-add (s + t <= 4); error about
//   2^-32 |A_ik| max|B_j.| + 2^-32 max|A_i.| |B_jk| per term from the
//   operands' rounding, and below 2^-40 max|A_i.| max|B_j.| from the
//   products left out.
//
// One CTA per SM, persistent and warp-specialised as the split-BF16 product:
//   warp 0   TMA loads of the four slices of A (128 x 64) and B (64 x 64) per
//            64-wide K block through a two-stage mbarrier ring;
//   warp 1   tcgen05.mma of the thirteen slice products into one of two
//            tensor-memory accumulator sets (4 x 64 columns each);
//   warps 2-9 add a finished window into their 64-bit totals (registers),
//            hand the set back and, after the last window, write the output
//            (or a 64-bit split-K partial).
// Every wait gives up after 2 s of %globaltimer and reports CD_ETIMEOUT.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>

#include "cd_internal.h"
#include "cd_mixed.h"
#include "cd_tc.cuh"
#include "cd_fixed_digits.cuh"

namespace cd {
namespace {

using namespace tc;

constexpr int FBM = 128, FBN = 64, FBK = 64;
constexpr int kSlices = 4;
constexpr int kWinKb = 4;  // K blocks of one exact window (256 of K)
constexpr int kStages = 2;
constexpr int kEpiWarps = 8;
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr uint32_t kATile = FBM * FBK * 2;  // one slice of A per K block
constexpr uint32_t kBTile = FBN * FBK * 2;  // one slice of B per K block
constexpr uint32_t kStageBytes = kSlices * (kATile + kBTile);
constexpr int kAccs = 4;                // accumulators: s + t = 0, 1, 2 (exact) and 3-4
constexpr int kAccCols = kAccs * FBN;   // one accumulator set (two sets in tensor memory)
constexpr int kStageLd = 9;            // FP64 output staging: 32 rows x 8 columns (+1)
constexpr size_t kEpiBytes = (size_t)kEpiWarps * 32 * kStageLd * sizeof(double);
constexpr size_t kDynSmem = (size_t)kStages * kStageBytes + kEpiBytes + 1024;
static_assert(kDynSmem <= 232448 - 1024, "shared memory per CTA");
static_assert(2 * kAccCols <= 512, "tensor memory columns");
// Exact windows: in units of its last place, accumulator d sums (d + 1)
// products of two integers in [-128, 128] per K: (d + 1) 256 2^14 <= 2^24.
static_assert((2 + 1) * kWinKb * FBK * (1 << 14) <= (1 << 24), "exact window");
constexpr int kMaxF = 8;

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major,
// N = 64 (N >> 3 at bit 17), M = 128 (M >> 4 at bit 24).
constexpr uint32_t kFIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(FBN >> 3) << 17) |
                             ((uint32_t)(FBM >> 4) << 24);

struct FDesc {  // 64-byte aligned through CUtensorMap
  CUtensorMap ta, tb;
  const double *Cin;
  double *Cout;
  long long *part;       // split-K partials: 64-bit totals, [split][M][N]
  const int *exa, *exb;  // row exponents of the stored operands, indexed by stored row
  long long ldcin, ldcout;
  double alpha, beta;
  int M, N, K, splits, kchunk;
  int tiles_m, tiles_n, tile_begin;
  int ax, ay, bx, by;
  int comb;
};

struct FGroup {
  int count, total_tiles, lower, pad_;
  int *err;
  FDesc d[kMaxF];
};
static_assert(sizeof(FGroup) <= 4096, "kernel parameter block too large");

// floor(f 2^32) as a 64-bit integer, from the bits of the binary32 f, in a
// few integer operations: the signed significand placed in the high word and
// shifted right arithmetically by 150 - exponent.  Exact when f is a
// multiple of 2^-32, which acc0, acc1 and acc2 are; acc3 (below 2^-24 of
// acc0's scale) is floored at 2^-32 of acc0's unit, 2^-46 of the product of
// the row maxima.  Zeros give 0; every reachable accumulator has |f| < 2^23,
// so the shift is at least 1.
__device__ __forceinline__ long long f32_to_fix(float f) {
  const int b = __float_as_int(f);
  const int e = (b >> 23) & 0xFF;
  const int s = b >> 31;  // 0 or -1
  const int m = (b & 0x7FFFFF) | (e ? 0x800000 : 0);
  const int sm = (m ^ s) - s;
  const int sh = max(1, min(150 - e, 63));
  return ((long long)sm << 32) >> sh;
}

// v 2^e2 as the nearest binary64 (ties to even), integer operations only.
// Results below the normal range flush to zero, above it give infinity.
__device__ __forceinline__ double fix_to_f64(long long v, int e2) {
  if (v == 0) return 0.0;
  const unsigned long long sg = v < 0 ? 0x8000000000000000ull : 0ull;
  unsigned long long u = v < 0 ? (unsigned long long)(-v) : (unsigned long long)v;
  const int lz = __clzll((long long)u);
  u <<= lz;  // leading one at bit 63
  unsigned long long mant = (u >> 11) & 0xFFFFFFFFFFFFFull;
  const unsigned long long rest = u & 0x7FFull;
  if (rest > 0x400ull || (rest == 0x400ull && (mant & 1ull))) ++mant;
  int ex = 63 - lz + e2 + 1023;
  if (mant >> 52) {
    mant = 0;
    ++ex;
  }
  if (ex <= 0) return __longlong_as_double((long long)sg);
  if (ex >= 2047) return __longlong_as_double((long long)(sg | 0x7FF0000000000000ull));
  return __longlong_as_double((long long)(sg | ((unsigned long long)ex << 52) | mant));
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// The slice products of one 16-deep K step (s + t <= 4), with their
// accumulator (0, 1, 2).  Dropping s + t = 4 as well would leave an error of
// about 2^-32 max|A_i.| max|B_j.| per multiply-add whatever the size of the
// elements (the last slices of every element are full digits), which rows
// that decay away from their maximum (rows of a Cholesky factor) feel as a
// large relative error; with them the dropped terms are below 2^-40.
constexpr int kProds = 13;
__device__ __forceinline__ int prod_a(int q) {
  const int v[kProds] = {0, 0, 1, 0, 1, 2, 0, 1, 2, 3, 1, 2, 3};
  return v[q];
}
__device__ __forceinline__ int prod_b(int q) {
  const int v[kProds] = {0, 1, 0, 2, 1, 0, 3, 2, 1, 0, 3, 2, 1};
  return v[q];
}
__device__ __forceinline__ int prod_acc(int q) { return q == 0 ? 0 : q < 3 ? 1 : q < 6 ? 2 : 3; }

struct Unit {
  int p, z, m0, n0, kbeg, nkb;
};

// Output tiles of a lower (i >= j) product: tile row ti holds column tiles
// tj < min(tiles_n, 2 ti + 2) (128-row by 64-column tiles).
__device__ __forceinline__ int lower_row_tiles(const FDesc &d, int ti) { return min(d.tiles_n, 2 * ti + 2); }

__device__ __forceinline__ int tiles_per_split(const FDesc &d, bool lower) {
  if (!lower) return d.tiles_m * d.tiles_n;
  int t = 0;
  for (int ti = 0; ti < d.tiles_m; ++ti) t += lower_row_tiles(d, ti);
  return t;
}

template <bool LOWER>
__device__ __forceinline__ Unit decode_unit(const FGroup &g, int u) {
  Unit x;
  int p = 0;
  while (p + 1 < g.count && u >= g.d[p + 1].tile_begin) ++p;
  const FDesc &d = g.d[p];
  const int local = u - d.tile_begin;
  const int per_split = tiles_per_split(d, LOWER);
  x.p = p;
  x.z = local / per_split;
  int rem = local - x.z * per_split;
  if (LOWER) {
    int ti = 0;
    while (rem >= lower_row_tiles(d, ti)) rem -= lower_row_tiles(d, ti++);
    x.m0 = ti * FBM;
    x.n0 = rem * FBN;
  } else {
    x.m0 = (rem / d.tiles_n) * FBM;
    x.n0 = (rem % d.tiles_n) * FBN;
  }
  x.kbeg = x.z * d.kchunk;
  const int kend = min(d.K, x.kbeg + d.kchunk);
  x.nkb = kend > x.kbeg ? (kend - x.kbeg + FBK - 1) / FBK : 0;
  return x;
}

// Windows of a unit: K blocks [w * kWinKb, min(nkb, (w + 1) * kWinKb)).
__device__ __forceinline__ int windows(int nkb) { return (nkb + kWinKb - 1) / kWinKb; }

template <bool LOWER, int COMB>
__device__ __forceinline__ void epilogue(const FGroup &g, uint32_t tmem, double *stw, int warp, int lane,
                                         volatile int *s_err, uint64_t *tfull_bar, uint64_t *tempty_bar);

// The persistent product.  A window (up to kWinKb K blocks of one unit) is
// the unit of hand-over between the MMA warp and the epilogue: window t of
// this CTA (counted over all its units) uses accumulator set t % 2.
// 168 registers a thread (the epilogue's 32 totals take 64): ten warps put
// three on some sub-partitions, whose 16K registers then allow 170.
template <bool LOWER, int COMB>
__global__ void __maxnreg__(168) k_fgemm(const __grid_constant__ FGroup g) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  double *epi = (double *)(smem + (size_t)kStages * kStageBytes);
  __shared__ __align__(8) uint64_t full_bar[kStages];
  __shared__ __align__(8) uint64_t empty_bar[kStages];
  __shared__ __align__(8) uint64_t tfull_bar[2];
  __shared__ __align__(8) uint64_t tempty_bar[2];
  __shared__ __align__(8) uint64_t drain_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int s_err;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int units = g.total_tiles;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
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
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      uint32_t it = 0;
      bool ok = true;
      uint32_t last_it[kStages];
      for (int s = 0; s < kStages; ++s) last_it[s] = 0xFFFFFFFFu;
      for (int u = blockIdx.x; u < units && ok; u += gridDim.x) {
        const Unit x = decode_unit<LOWER>(g, u);
        const FDesc &d = g.d[x.p];
        for (int kb = 0; kb < x.nkb; ++kb, ++it) {
          const int s = (int)(it % kStages);
          if (it >= (uint32_t)kStages && !mbar_wait_or_abort(&empty_bar[s], ((it / kStages) - 1) & 1u, &s_err)) {
            s_err = 1;
            ok = false;
            break;
          }
          uint8_t *sa = smem + s * kStageBytes;
          uint8_t *sb = sa + kSlices * kATile;
          mbar_expect_tx(&full_bar[s], kStageBytes);
          const int kx = x.kbeg + kb * FBK;
          tma_load_3d(sa, &d.ta, d.ax + kx, d.ay + x.m0, 0, &full_bar[s]);
          tma_load_3d(sb, &d.tb, d.bx + kx, d.by + x.n0, 0, &full_bar[s]);
          last_it[s] = it;
        }
      }
      if (!ok) {  // failure: let copies in flight land before the CTA exits (bounded)
        for (int s = 0; s < kStages; ++s)
          if (last_it[s] != 0xFFFFFFFFu) {
            const unsigned long long t0 = globaltimer();
            while (!mbar_try_wait(&full_bar[s], (last_it[s] / kStages) & 1u) && globaltimer() - t0 < kTimeoutNs / 8) {
            }
          }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      uint32_t it = 0, t = 0;
      bool issued = false, ok = true;
      for (int u = blockIdx.x; u < units && ok; u += gridDim.x) {
        const Unit x = decode_unit<LOWER>(g, u);
        const int nw = windows(x.nkb);
        for (int w = 0; w < nw && ok; ++w, ++t) {
          const int b = (int)(t & 1u);
          if (t >= 2 && !mbar_wait_or_abort(&tempty_bar[b], ((t >> 1) - 1) & 1u, &s_err)) {
            s_err = 1;
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t acc = tmem + (uint32_t)(b * kAccCols);
          const int kb1 = min(x.nkb, (w + 1) * kWinKb);
          bool first = true;
          for (int kb = w * kWinKb; kb < kb1; ++kb, ++it) {
            const int s = (int)(it % kStages);
            if (!mbar_wait_or_abort(&full_bar[s], (it / kStages) & 1u, &s_err)) {
              s_err = 1;
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t sa = smem_u32(smem + s * kStageBytes);
            const uint32_t sb = sa + kSlices * kATile;
#pragma unroll
            for (int kk = 0; kk < FBK / 16; ++kk) {
#pragma unroll
              for (int q = 0; q < kProds; ++q) {
                const uint64_t ad = sw128_desc(sa + prod_a(q) * kATile + kk * 32);
                const uint64_t bd = sw128_desc(sb + prod_b(q) * kBTile + kk * 32);
                // the first product of each accumulator in a window overwrites it
                const bool init = first && kk == 0 && (q == 0 || q == 1 || q == 3 || q == 6);
                mma_bf16_id(acc + (uint32_t)(prod_acc(q) * FBN), ad, bd, kFIdesc, init ? 0u : 1u);
              }
            }
            first = false;
            issued = true;
            mma_commit(&empty_bar[s]);
          }
          if (!ok) break;
          mma_commit(&tfull_bar[b]);
        }
      }
      if (s_err && issued) {  // failure: issued products finish before tensor memory is freed
        mma_commit(&drain_bar);
        mbar_wait(&drain_bar, 0);
      }
    }
    __syncwarp();
  } else {
    epilogue<LOWER, COMB>(g, tmem, epi + (size_t)(warp - 2) * 32 * kStageLd, warp, lane, &s_err, tfull_bar, tempty_bar);
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
  }
  if (threadIdx.x == 0 && s_err && g.err) atomicExch(g.err, CD_ETIMEOUT);
}

// Writes the staged 32 x 8 block (rows rbase.., columns j0..) of FP64 product
// values under mode COMB: lane l takes column j0 + l % 8 of rows l / 8 + 4 k.
template <int COMB, bool LOWER>
__device__ __forceinline__ void write_block8(const FDesc &d, const double *stw, int rbase, int nrows, int j0,
                                             int lane) {
  constexpr bool kUseCin = COMB >= kAdd;
  const int c = lane & 7, h = lane >> 3, j = j0 + c;
  if (j >= d.N) return;
  double cin[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int rr = h + 4 * k, i = rbase + rr;
    cin[k] = (kUseCin && rr < nrows && !(LOWER && j > i)) ? d.Cin[(long long)i * d.ldcin + j] : 0.0;
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int rr = h + 4 * k, i = rbase + rr;
    if (rr < nrows && !(LOWER && j > i))
      d.Cout[(long long)i * d.ldcout + j] = combine<COMB>(stw[rr * kStageLd + c], cin[k], d.alpha, d.beta);
  }
}

// Epilogue warp (warps 2-9): tensor-memory lane quarter warp % 4 (32 rows,
// lane = row) and columns [32 half, 32 half + 32) of the 64-wide tile.  The
// 64-bit running totals of its 32 elements stay in registers across the
// unit's windows; each window's four accumulators are added to them and the
// set is handed back to the MMA warp at once.
template <bool LOWER, int COMB>
__device__ __forceinline__ void epilogue(const FGroup &g, uint32_t tmem, double *stw, int warp, int lane,
                                         volatile int *s_err, uint64_t *tfull_bar, uint64_t *tempty_bar) {
  const int qd = warp & 3, half = (warp - 2) / 4;
  const uint32_t lane_base = (uint32_t)(qd * 32) << 16;
  uint32_t t = 0;
  for (int u = blockIdx.x; u < g.total_tiles; u += gridDim.x) {
    const Unit x = decode_unit<LOWER>(g, u);
    const FDesc &d = g.d[x.p];
    const int rbase = x.m0 + qd * 32, nrows = max(0, min(32, d.M - rbase));
    const int i = rbase + lane;
    const int nw = windows(x.nkb);  // 0: an empty split-K part, which writes zeros
    long long tot[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) tot[q] = 0;
    for (int w = 0; w < nw; ++w, ++t) {
      const int b = (int)(t & 1u);
      const bool got = mbar_wait_or_abort(&tfull_bar[b], (t >> 1) & 1u, s_err);
      if (!__all_sync(0xffffffffu, got)) {
        *s_err = 1;
        return;
      }
      tc_fence_after();
      const uint32_t acc = tmem + lane_base + (uint32_t)(b * kAccCols + 32 * half);
#pragma unroll
      for (int a = 0; a < kAccs; ++a) {  // one accumulator's 32 columns: four loads, one wait
        uint32_t x0[8], x1[8], x2[8], x3[8];
        tmem_ld8(acc + (uint32_t)(a * FBN), x0);
        tmem_ld8(acc + (uint32_t)(a * FBN + 8), x1);
        tmem_ld8(acc + (uint32_t)(a * FBN + 16), x2);
        tmem_ld8(acc + (uint32_t)(a * FBN + 24), x3);
        tmem_wait_ld();
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          tot[q] += f32_to_fix(__uint_as_float(x0[q]));
          tot[8 + q] += f32_to_fix(__uint_as_float(x1[q]));
          tot[16 + q] += f32_to_fix(__uint_as_float(x2[q]));
          tot[24 + q] += f32_to_fix(__uint_as_float(x3[q]));
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty_bar[b]);
    }
    const int j0 = x.n0 + 32 * half;
    if (d.splits > 1) {
      if (lane < nrows) {
        long long *pp = d.part + ((long long)x.z * d.M + i) * d.N;
#pragma unroll
        for (int q = 0; q < 32; ++q)
          if (j0 + q < d.N && !(LOWER && j0 + q > i)) pp[j0 + q] = tot[q];
      }
      continue;
    }
    const int ea = (i < d.M) ? d.exa[d.ay + i] : 0;
    const int jl = j0 + lane;
    const int ebl = jl < d.N ? d.exb[d.by + jl] : 0;
#pragma unroll
    for (int h8 = 0; h8 < 4; ++h8) {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int eb = __shfl_sync(0xffffffffu, ebl, h8 * 8 + q);
        stw[lane * kStageLd + q] = fix_to_f64(tot[h8 * 8 + q], ea + eb - 46);
      }
      __syncwarp();
      write_block8<COMB, LOWER>(d, stw, rbase, nrows, j0 + h8 * 8, lane);
      __syncwarp();
    }
  }
}

// Split-K reduction: the 64-bit partial totals summed exactly, then one
// rounding to FP64 and the output formed as in the product's epilogue.
template <int COMB, bool LOWER>
__device__ __forceinline__ void freduce_loop(const FDesc &d) {
  const long long total = (long long)d.M * d.N;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / d.N), j = (int)(e - (long long)i * d.N);
    if (LOWER && j > i) continue;
    long long v = 0;
    for (int z = 0; z < d.splits; ++z) v += d.part[(long long)z * total + e];
    const double a = fix_to_f64(v, d.exa[d.ay + i] + d.exb[d.by + j] - 46);
    const double cin = COMB >= kAdd ? d.Cin[(long long)i * d.ldcin + j] : 0.0;
    d.Cout[(long long)i * d.ldcout + j] = combine<COMB>(a, cin, d.alpha, d.beta);
  }
}

template <bool LOWER>
__global__ void k_freduce(const __grid_constant__ FGroup g) {
  const FDesc &d = g.d[blockIdx.y];
  if (d.splits <= 1) return;
  switch (d.comb) {
    case kCopy: freduce_loop<kCopy, LOWER>(d); break;
    case kNeg: freduce_loop<kNeg, LOWER>(d); break;
    case kScale: freduce_loop<kScale, LOWER>(d); break;
    case kAdd: freduce_loop<kAdd, LOWER>(d); break;
    case kSub: freduce_loop<kSub, LOWER>(d); break;
    case kAxpy: freduce_loop<kAxpy, LOWER>(d); break;
    default: freduce_loop<kGeneral, LOWER>(d); break;
  }
}

// The source value that destination element (rr, cc) of a (non-transposed)
// split views, or 0 outside the view; modes as for the split-BF16 splits
// (0 full, 1 lower triangle, 2 symmetric view with doubled diagonal).
__device__ __forceinline__ double view_value(const SplitArgs &a, int rr, int cc) {
  const int r = a.reg_r0 + rr - a.dst_r0, c = a.reg_c0 + cc - a.dst_c0;
  if (r < 0 || c < 0 || r >= a.rows || c >= a.cols) return 0.0;
  const bool upper = r < c;
  if (a.mode == 1 && upper) return 0.0;
  if (a.mode == 2) {
    if (upper) return a.src[(long long)c * a.lds + r];
    return r == c ? 2.0 * a.src[(long long)r * a.lds + c] : a.src[(long long)r * a.lds + c];
  }
  return a.src[(long long)r * a.lds + c];
}

constexpr int kMaxFSplit = 24;
struct SplitGroupF {
  int count, pad_;
  SplitArgs a[kMaxFSplit];
};
static_assert(sizeof(SplitGroupF) <= 4096, "kernel parameter block too large");

// One warp per destination row of each split: E_r over the row's region.
__global__ void k_rowexp_group(const __grid_constant__ SplitGroupF g) {
  const SplitArgs &a = g.a[blockIdx.y];
  const int warps = blockDim.x >> 5, lane = threadIdx.x & 31;
  for (int rr = blockIdx.x * warps + (threadIdx.x >> 5); rr < a.dst_h; rr += gridDim.x * warps) {
    double m = 0.0;
    for (int cc = lane; cc < a.dst_w; cc += 32) m = fmax(m, fabs(view_value(a, rr, cc)));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) a.ex[a.reg_r0 + rr] = exp_above(m);
  }
}

// E_i of the factor's row i from the diagonal of Sigma: |L_ik| <= sqrt(Sigma_ii)
// since Sigma_ii = sum_k L_ik^2; with a margin of 2^-10 for rounding,
// sqrt(Sigma_ii (1 + 2^-10)) < 2^E for E = ceil(e / 2), Sigma_ii (1 + 2^-10) < 2^e.
// A diagonal that is not positive (the factorisation will report it) gives 0.
__global__ void k_diagexp(const double *S, long long lds, int n, int *ex) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double d = S[(long long)i * lds + i];
  int E = 0;
  if (d > 0.0) {
    const int e = exp_above(d * (1.0 + 0x1p-10));
    E = e == kZeroExp ? kZeroExp : (e + 1) >> 1;
  }
  ex[i] = E;
}

// Fixed-point split: 32 x 32 destination tiles, slice s of element (r, c) at
// dst + (s dst_rows + r) ldd + c, each a_s 2^(-8 s) with a_s in [-128, 128]:
// Q = a_0 2^24 + a_1 2^16 + a_2 2^8 + a_3, digits taken from the top.
__global__ void __launch_bounds__(256) k_fsplit_group(const __grid_constant__ SplitGroupF g) {
  const SplitArgs &a = g.a[blockIdx.y];
  __nv_bfloat16 *dst = (__nv_bfloat16 *)a.dst;
  const long long ts = a.dst_rows * a.ldd;
  const int tiles_c = (a.dst_w + 31) / 32;
  const int tiles = ((a.dst_h + 31) / 32) * tiles_c;
  for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
    const int rr0 = (t / tiles_c) * 32, cc0 = (t % tiles_c) * 32;
    for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
      const int rr = rr0 + (e >> 5), cc = cc0 + (e & 31);
      if (rr >= a.dst_h || cc >= a.dst_w) continue;
      const int row = a.reg_r0 + rr;
      write_fixed_slices(dst, ts, (long long)row * a.ldd + a.reg_c0 + cc, fixed_q(view_value(a, rr, cc), a.ex[row]));
    }
  }
}

typedef CUresult (*FEncodeFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                              const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
FEncodeFn g_fencode = nullptr;

bool encode_fmap(CUtensorMap *m, const MOp &op, int box_rows) {
  if (!g_fencode) return false;
  if (!op.base || (op.ld % 64) != 0 || ((uintptr_t)op.base % 16) != 0 || op.rows <= 0 || op.T != kSlices)
    return false;
  cuuint64_t dims[3] = {(cuuint64_t)op.ld, (cuuint64_t)op.rows, (cuuint64_t)kSlices};
  cuuint64_t strides[2] = {(cuuint64_t)op.ld * 2, (cuuint64_t)op.ld * 2 * (cuuint64_t)op.rows};
  cuuint32_t box[3] = {(cuuint32_t)FBK, (cuuint32_t)box_rows, (cuuint32_t)kSlices};
  cuuint32_t estr[3] = {1, 1, 1};
  return g_fencode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(op.base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int fsm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
    return 148;
  return n;
}

// Per device: function attributes (the dynamic shared-memory limit) are set
// on the current device.
constexpr int kMaxDev = 64;
bool g_fready[kMaxDev];

}  // namespace

int fixed_init() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return CD_ECUDA;
  if (g_fready[dev]) return CD_OK;
  void *fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || fn == nullptr) {
    cudaGetLastError();
    return CD_ECUDA;
  }
  g_fencode = (FEncodeFn)fn;
  const int sm = (int)kDynSmem;
  cudaError_t e = cudaFuncSetAttribute(k_fgemm<false, kCopy>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (!e) e = cudaFuncSetAttribute(k_fgemm<false, kSub>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (!e) e = cudaFuncSetAttribute(k_fgemm<true, kCopy>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (!e) e = cudaFuncSetAttribute(k_fgemm<true, kSub>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  const int carve = cudaSharedmemCarveoutMaxShared;
  if (!e) e = cudaFuncSetAttribute(k_freduce<true>, cudaFuncAttributePreferredSharedMemoryCarveout, carve);
  if (!e) e = cudaFuncSetAttribute(k_freduce<false>, cudaFuncAttributePreferredSharedMemoryCarveout, carve);
  if (!e) e = cudaFuncSetAttribute(k_fsplit_group, cudaFuncAttributePreferredSharedMemoryCarveout, carve);
  if (!e) e = cudaFuncSetAttribute(k_rowexp_group, cudaFuncAttributePreferredSharedMemoryCarveout, carve);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return CD_ECUDA;
  }
  g_fready[dev] = true;
  return CD_OK;
}

cudaError_t fixed_gemm_launch(const MProblem *probs, int count, bool lower, int *dev_err, cudaStream_t s,
                              int *launches, int max_units) {
  max_units = std::max(1, max_units);
  int i = 0;
  while (i < count) {
    FGroup g;
    memset(&g, 0, sizeof(g));
    g.lower = lower ? 1 : 0;
    g.err = dev_err;
    bool any_split = false;
    long long biggest = 0;
    for (; i < count && g.count < kMaxF; ++i) {
      const MProblem &P = probs[i];
      if (P.M <= 0 || P.N <= 0 || P.K <= 0) continue;
      if ((P.A.x0 % 8) || (P.B.x0 % 8) || P.A.x0 < 0 || P.B.x0 < 0 || P.A.y0 < 0 || P.B.y0 < 0 ||
          (P.kchunk % FBK) || P.kchunk <= 0 || !P.A.ex || !P.B.ex || (lower && P.M != P.N) ||
          (P.splits > 1 && !P.part))
        return cudaErrorInvalidValue;
      FDesc &d = g.d[g.count];
      if (!encode_fmap(&d.ta, P.A, FBM) || !encode_fmap(&d.tb, P.B, FBN)) return cudaErrorInvalidValue;
      d.Cin = P.Cin;
      d.Cout = P.Cout;
      d.part = reinterpret_cast<long long *>(P.part);  // splits * M * N 8-byte words
      d.exa = P.A.ex;
      d.exb = P.B.ex;
      // output modes of the fixed-point product: C = A B^T (copy) or C = Cin - A B^T
      d.comb = (P.beta == 0.0 && P.alpha == 1.0) ? kCopy : (P.beta == 1.0 && P.alpha == -1.0) ? kSub : -1;
      if (d.comb < 0 || (g.count > 0 && d.comb != g.d[0].comb)) return cudaErrorInvalidValue;
      d.ldcin = P.ldcin;
      d.ldcout = P.ldcout;
      d.alpha = P.alpha;
      d.beta = P.beta;
      d.M = P.M;
      d.N = P.N;
      d.K = P.K;
      d.splits = P.splits;
      d.kchunk = P.kchunk;
      d.tiles_m = (P.M + FBM - 1) / FBM;
      d.tiles_n = (P.N + FBN - 1) / FBN;
      d.tile_begin = g.total_tiles;
      d.ax = P.A.x0;
      d.ay = P.A.y0;
      d.bx = P.B.x0;
      d.by = P.B.y0;
      int per = 0;
      if (lower)
        for (int ti = 0; ti < d.tiles_m; ++ti) per += std::min(d.tiles_n, 2 * ti + 2);
      else
        per = d.tiles_m * d.tiles_n;
      g.total_tiles += per * P.splits;
      if (P.splits > 1) {
        any_split = true;
        biggest = std::max(biggest, (long long)P.M * P.N);
      }
      ++g.count;
    }
    if (g.count == 0) continue;
    const int units = g.total_tiles;
    const int grid = std::min(units, std::max(fsm_count(), (units + max_units - 1) / max_units));
    const int comb = g.d[0].comb;  // one output mode per launch (checked above)
    if (lower)
      (comb == kCopy ? k_fgemm<true, kCopy> : k_fgemm<true, kSub>)<<<grid, kThreads, kDynSmem, s>>>(g);
    else
      (comb == kCopy ? k_fgemm<false, kCopy> : k_fgemm<false, kSub>)<<<grid, kThreads, kDynSmem, s>>>(g);
    if (launches) ++*launches;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (any_split) {
      const long long blocks = std::min<long long>(1024, (biggest + 255) / 256);
      const dim3 rg((unsigned)blocks, (unsigned)g.count);
      if (lower)
        k_freduce<true><<<rg, 256, 0, s>>>(g);
      else
        k_freduce<false><<<rg, 256, 0, s>>>(g);
      if (launches) ++*launches;
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

// Row exponents of each split's destination rows (max over the region),
// then the slices; or the slices alone when the exponents are given.
cudaError_t fixed_split_group_launch(const SplitArgs *a, int count, bool compute_exponents, cudaStream_t s,
                                     int *launches) {
  int i = 0;
  while (i < count) {
    SplitGroupF g;
    memset(&g, 0, sizeof(g));
    long long tiles = 0, rows = 0;
    for (; i < count && g.count < kMaxFSplit; ++i) {
      if ((long long)a[i].dst_h * a[i].dst_w <= 0) continue;
      if (a[i].T != kSlices || !a[i].dst || !a[i].ex || a[i].transpose) return cudaErrorInvalidValue;
      g.a[g.count++] = a[i];
      tiles = std::max(tiles, (long long)((a[i].dst_h + 31) / 32) * ((a[i].dst_w + 31) / 32));
      rows = std::max(rows, (long long)a[i].dst_h);
    }
    if (g.count == 0) continue;
    if (compute_exponents) {
      const long long blocks = std::max<long long>(1, std::min<long long>(4096, (rows + 7) / 8));
      k_rowexp_group<<<dim3((unsigned)blocks, (unsigned)g.count), 256, 0, s>>>(g);
      if (launches) ++*launches;
      const cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    const long long blocks = std::max<long long>(1, std::min<long long>(4096, tiles));
    k_fsplit_group<<<dim3((unsigned)blocks, (unsigned)g.count), 256, 0, s>>>(g);
    if (launches) ++*launches;
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t fixed_diag_exponents(const double *S, long long lds, int n, int *ex, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_diagexp<<<(n + 255) / 256, 256, 0, s>>>(S, lds, n, ex);
  return cudaGetLastError();
}

}  // namespace cd
