// Device helpers shared by the tensor-core products of libcholdiff
// (cd_mixed.cu, cd_fixed.cu): mbarrier waits bounded by %globaltimer, TMA
// tile loads, tcgen05 descriptors, issue, commit and tensor-memory loads,
// the integer-only FP32 -> FP64 widening and the epilogue's combine modes.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace cd {
namespace tc {

constexpr unsigned long long kTimeoutNs = 2000000000ULL;

// How an FP64 output is formed from the accumulated product a (chosen on
// the host from alpha and beta, so that the common cases need no FP64
// multiply: on this GPU every FP64 instruction occupies a narrow unit for
// about 64 cycles per warp).
enum Comb { kCopy = 0, kNeg = 1, kScale = 2, kAdd = 3, kSub = 4, kAxpy = 5, kGeneral = 6 };


__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// IEEE-754 conversions written with integer operations.  On this GPU the
// conversion instructions between FP32 and FP64 run on the FP64 unit (about
// 80 cycles per warp), while integer and FP32 instructions issue every few
// cycles; these run once per element of every product and every split.

// binary32 -> binary64 without branches: rebias the exponent and widen the
// significand (exact for normal numbers, zeros, infinities and NaN); a
// subnormal binary32 (below 2^-126) is taken as zero.
__device__ __forceinline__ double f32_to_f64(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t e = (b >> 23) & 0xFFu;
  const uint32_t hi = (b & 0x80000000u) | ((e == 0xFFu ? 0x7FFu : e + 896u) << 20) | ((b & 0x7FFFFFu) >> 3);
  const uint32_t lo = b << 29;
  return e == 0 ? __longlong_as_double((long long)(uint64_t)(b & 0x80000000u) << 32)
                : __hiloint2double((int)hi, (int)lo);
}


// The output from the accumulated product a, for one Comb mode.  The mode is
// a template argument so that each row loop holds exactly its own arithmetic:
// with a runtime switch the compiler evaluates every case under predicates,
// and each predicated-off FP64 instruction still holds the FP64 unit.
template <int COMB>
__device__ __forceinline__ double combine(double a, double cin, double alpha, double beta) {
  if (COMB == kCopy) return a;
  if (COMB == kNeg) return __longlong_as_double(__double_as_longlong(a) ^ (long long)0x8000000000000000ull);
  if (COMB == kScale) return alpha * a;
  if (COMB == kAdd) return cin + a;
  if (COMB == kSub) return cin - a;
  if (COMB == kAxpy) return fma(alpha, a, cin);
  return fma(alpha, a, beta * cin);
}


__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: false if the phase did not complete within kTimeoutNs.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (globaltimer() - t0 > kTimeoutNs) return false;
  }
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_u32(dst)),
      "l"((unsigned long long)map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major tile in the 128-byte swizzle
// layout: 8-row groups 1024 B apart (SBO), descriptor version 1, layout 2.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;              // leading byte offset (unused for this layout)
  d |= (uint64_t)(1024 >> 4) << 32;    // stride byte offset
  d |= (uint64_t)1 << 46;              // descriptor version
  d |= (uint64_t)2 << 61;              // SWIZZLE_128B
  return d;
}

__device__ __forceinline__ void mma_bf16_id(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::
          "r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}


// Bounded wait that also gives up as soon as another role of the CTA has
// recorded a failure in *abort.
__device__ __forceinline__ bool mbar_wait_or_abort(uint64_t *bar, uint32_t parity, const volatile int *abort) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort || globaltimer() - t0 > kTimeoutNs) return false;
  }
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}


}  // namespace tc
}  // namespace cd
