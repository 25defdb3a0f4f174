// Counter-based noise of the generator: Philox4x64-10 (Salmon, Moraes, Dror & Shaw,
// "Parallel random numbers: as easy as 1, 2, 3", SC'11) followed by Box-Muller.
//
// The paper keeps the seeds of each realisation so that Phi_L can be regenerated at any
// radius (Sect. 3, memory reduction).  Here the white noise n_lm(r_j) is a pure function
// of (seed, realisation, j, idx(l, m)), so every kernel can draw exactly the numbers it
// needs, in any order, with nothing stored.
#pragma once

#include <cstdint>

namespace fnl {

__device__ __forceinline__ void philox4x64_10(uint64_t c[4], uint64_t k0, uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += W0;
      k1 += W1;
    }
    const uint64_t lo0 = M0 * c[0], hi0 = __umul64hi(M0, c[0]);
    const uint64_t lo1 = M1 * c[2], hi1 = __umul64hi(M1, c[2]);
    const uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
}

// The four output words for noise entry idx of shells 4 jq .. 4 jq + 3: counter
// (idx, jq, realisation, 0), key (seed, 0); shell j takes word j & 3.
__device__ __forceinline__ void noise_words(uint64_t seed, uint64_t real, int64_t idx, int jq,
                                            uint64_t w[4]) {
  w[0] = (uint64_t)idx;
  w[1] = (uint64_t)jq;
  w[2] = real;
  w[3] = 0;
  philox4x64_10(w, seed, 0);
}

// Box-Muller in FP64 from one 64-bit word: u1 = ((w >> 32) + 1) 2^-32 in (0, 1],
// u2 = (w mod 2^32) 2^-32 in [0, 1), (g1, g2) = sqrt(-2 ln u1) (cos 2 pi u2, sin 2 pi u2).
__device__ __forceinline__ double2 box_muller(uint64_t w) {
  const double u1 = (double)((w >> 32) + 1) * 0x1p-32;
  const double u2 = (double)(w & 0xffffffffull) * 0x1p-32;
  const double rho = sqrt(-2.0 * log(u1));
  double s, c;
  sincospi(2.0 * u2, &s, &c);
  return make_double2(rho * c, rho * s);
}

// n_lm(r_j) from a Box-Muller pair: unit complex variance for m > 0, real N(0,1) for m = 0.
__device__ __forceinline__ double2 noise_value(double2 g, int m) {
  if (m == 0) return make_double2(g.x, 0.0);
  const double h = 0.70710678118654752440;
  return make_double2(g.x * h, g.y * h);
}

// Noise in FP32 from the same words as the FP64 path (the FP32 and mixed forms): the uniforms
// are the FP64 path's rounded once to FP32 (relative 2^-24), so draws agree with it to ~1e-7.
__device__ __forceinline__ float2 box_muller_f32(uint64_t w) {
  const uint32_t hi = (uint32_t)(w >> 32), lo = (uint32_t)w;
  const float u1 = hi == 0xffffffffu ? 1.0f : __uint2float_rn(hi + 1u) * 0x1p-32f;
  const float u2 = __uint2float_rn(lo) * 0x1p-32f;
  const float rho = sqrtf(-2.0f * logf(u1));
  float s, c;
  sincospif(2.0f * u2, &s, &c);
  return make_float2(rho * c, rho * s);
}

__device__ __forceinline__ float2 noise_value_f32(float2 g, int m) {
  if (m == 0) return make_float2(g.x, 0.f);
  const float h = 0.70710678118654752f;
  return make_float2(g.x * h, g.y * h);
}

}  // namespace fnl
