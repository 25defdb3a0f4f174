// Helpers of the mixed-precision forms: splitting a value into BF16 terms
// x = t0 + t1 (+ t2), each term the round-to-nearest BF16 of the remainder so far.
#pragma once

#include <cuda_bf16.h>

#include <cstdint>

namespace fnl {

__device__ __forceinline__ void store_terms(__nv_bfloat16* p, int64_t stride, int nterms, float x) {
  const __nv_bfloat16 h0 = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(h0);
  const __nv_bfloat16 h1 = __float2bfloat16_rn(r1);
  p[0] = h0;
  p[stride] = h1;
  if (nterms > 2) p[2 * stride] = __float2bfloat16_rn(r1 - __bfloat162float(h1));
}

__device__ __forceinline__ void store_terms_d(__nv_bfloat16* p, int64_t stride, int nterms, double x) {
  const __nv_bfloat16 h0 = __double2bfloat16(x);
  const double r1 = x - (double)__bfloat162float(h0);
  const __nv_bfloat16 h1 = __double2bfloat16(r1);
  p[0] = h0;
  p[stride] = h1;
  if (nterms > 2) p[2 * stride] = __double2bfloat16(r1 - (double)__bfloat162float(h1));
}

}  // namespace fnl
