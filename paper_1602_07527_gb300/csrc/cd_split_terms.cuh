// The three-term split-BF16 format of the tensor-core products (cd_mixed.cu),
// shared by the split kernel and the diagonal tile kernel, which writes its
// inverse in this format directly: an element x is split into FP32 pieces
// hi + lo, then into T = 2 or 3 BF16 terms t0 + t1 (+ t2), term s of element
// (r, c) at dst + (s rows + r) ld + c.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

namespace cd {

// binary64 x -> (hi, lo) in binary32: hi is x with its significand cut to 24
// bits (exact), lo the remaining 29 bits rounded to 24, so that
// |x - hi - lo| <= 2^-47 |x|.  Outside FP32's normal range: below it both
// parts are zero, above it hi is +-inf, NaN stays NaN.
__device__ __forceinline__ void f64_to_f32x2(double x, float &hi, float &lo) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const uint32_t sg = (uint32_t)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7FF);
  const uint64_t m = b & 0xFFFFFFFFFFFFFull;
  const int fe = e - 896;  // binary32 biased exponent of x
  lo = 0.0f;
  if (fe >= 1 && fe <= 254) {
    hi = __uint_as_float(sg | ((uint32_t)fe << 23) | (uint32_t)(m >> 29));
    const uint32_t r = (uint32_t)(m & 0x1FFFFFFFu);  // remainder r 2^(e - 1075)
    if (r != 0) {
      const uint32_t rb = __float_as_uint(__uint2float_rn(r));
      const int re = (int)(rb >> 23) + (e - 1075);  // rescale through the exponent field
      if (re >= 1) lo = __uint_as_float(sg | ((uint32_t)re << 23) | (rb & 0x7FFFFFu));
    }
  } else if (e == 0x7FF) {
    hi = __uint_as_float(sg | 0x7F800000u | (m ? 0x400000u : 0u));
  } else {
    hi = __uint_as_float(fe > 254 ? (sg | 0x7F800000u) : sg);
  }
}

// The T BF16 terms of one element from its FP32 pieces, at dst[o], dst[ts + o] (and dst[2 ts + o]).
__device__ __forceinline__ void write_split_terms(__nv_bfloat16 *dst, long long ts, long long o, float hi, float lo,
                                                  int T) {
  const __nv_bfloat16 t0 = __float2bfloat16_rn(hi);
  const float d0 = hi - __bfloat162float(t0);
  const __nv_bfloat16 t1 = __float2bfloat16_rn(d0 + lo);
  dst[o] = t0;
  dst[ts + o] = t1;
  if (T == 3) dst[2 * ts + o] = __float2bfloat16_rn((d0 - __bfloat162float(t1)) + lo);
}

}  // namespace cd
