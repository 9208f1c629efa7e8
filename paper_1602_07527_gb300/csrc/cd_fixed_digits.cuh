// Fixed-point slices of a binary64 row (the operand format of the fixed-point
// product, cd_fixed.cu), shared by the split kernel and the diagonal tile
// kernel, which writes its inverse in this format directly.
//
// Row r of a matrix with 0 < |x| < 2^E_r for every x in the row is held as
// Q = x 2^(31 - E_r) rounded to an integer (|Q| < 2^31), cut into four digits
// a_0..a_3 in [-128, 128] taken from the top, Q = a_0 2^24 + a_1 2^16 +
// a_2 2^8 + a_3; slice s holds a_s 2^(-8 s) in BF16 (exact: 9-bit integers).
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

namespace cd {

constexpr int kZeroExp = -1000;  // the exponent of a row of zeros

// Exponent E with 0 < x < 2^E for a non-negative binary64 x (the biased
// exponent field gives x < 2^(field - 1022)); zero and subnormals give
// kZeroExp, infinities and NaN 0.
__device__ __forceinline__ int exp_above(double x) {
  const int f = (int)((__double_as_longlong(x) >> 52) & 0x7FF);
  return f == 0 ? kZeroExp : f == 0x7FF ? 0 : f - 1022;
}

// x 2^(31 - E) rounded to an integer (|x| < 2^E gives |Q| < 2^31), from the
// bits of x; beyond the bound (not reached for valid exponents) it clamps.
__device__ __forceinline__ long long fixed_q(double x, int E) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FF);
  if (e == 0) return 0;
  const long long m = (long long)((b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull);
  const int sh = e - 1044 - E;  // x 2^(31 - E) = m 2^(e - 1075 + 31 - E)
  long long q;
  if (e == 0x7FF || sh >= 0)
    q = 0x7FFFFFFFll;
  else
    q = sh < -63 ? 0 : ((m >> (-sh - 1)) + 1) >> 1;
  q = min(q, 0x7FFFFFFFll);
  return (b >> 63) ? -q : q;
}

// The four slices of Q at dst[o], dst[ts + o], dst[2 ts + o], dst[3 ts + o].
__device__ __forceinline__ void write_fixed_slices(__nv_bfloat16 *dst, long long ts, long long o, long long q) {
  const long long a0 = (q + (1ll << 23)) >> 24;
  q -= a0 << 24;
  const long long a1 = (q + (1ll << 15)) >> 16;
  q -= a1 << 16;
  const long long a2 = (q + (1ll << 7)) >> 8;
  q -= a2 << 8;
  dst[o] = __float2bfloat16_rn((float)a0);
  dst[ts + o] = __float2bfloat16_rn((float)a1 * 0x1p-8f);
  dst[2 * ts + o] = __float2bfloat16_rn((float)a2 * 0x1p-16f);
  dst[3 * ts + o] = __float2bfloat16_rn((float)q * 0x1p-24f);
}

}  // namespace cd
