// Step (i) of the tensor-core forms on the 5th-generation tensor cores: the noise n_lm(r_j) is
// drawn (Philox4x64-10 + FP32 Box-Muller, as in the FP32 form) and Phi_L = K_l n (Eq. 9) is a GEMM
// per degree l:
//   D[i][col] = sum_j K_l[j0 + i][j] n[j][col],  M = 128 shells i, N = 64 columns (32 orders m,
//   re and im), K = 128 noise shells j
// with both operands split into three BF16 terms (24 bits, so the split of an FP32 value is exact)
// and the six products of terms (ta, tb), ta + tb < 3, accumulated in FP32 in tensor memory (the
// leading product and the corrections in two accumulators).  The linear part a^X_L = v^X . n
// (Eq. 5 applied to Eq. 9) is summed from the same noise in double-float, and the per-shell sums
// of |Phi_L,lm|^2 for the Parseval monopole from the results.
//
// One persistent CTA per SM takes degrees in a snake order over the CTAs (largest first); a
// degree's orders run in chunks of 32.  Warp roles, pipelined over the chunks (two noise buffers,
// two accumulator sets):
//   warps 0-10  noise: Philox words, Box-Muller, the BF16 terms of the noise tile written into
//               shared memory in the MMA's layout (N-major rows of 64 columns, 128B swizzle);
//               a lane takes one order of the chunk, a warp up to three quads of shells, and
//               each lane's partial sums of a^X_L over its shells go to shared memory
//   warps 11-18 epilogue, two per TMEM lane quadrant (a lane = a shell), each taking half of a
//               chunk's orders: the a^X_L sums over the noise warps' partials, tcgen05.ld of
//               the two accumulators, Phi_L as BF16 terms of the synthesis operand, the
//               monopole sums
//   warp 19     allocates TMEM, loads K_l (all three terms in one TMA box of 96 KB per degree)
//               and issues the MMAs from one lane
// Every mbarrier wait is bounded; on expiry the kernel records an error and unwinds.
#include <cuda_bf16.h>

#include <algorithm>
#include <vector>

#include "fnl_internal.cuh"
#include "philox.cuh"
#include "tc_gemm.cuh"
#include "tc_ptx.cuh"

namespace fnl {

namespace {

constexpr int kFtcNoiseWarps = 11;                // warps 0 .. 10: noise
constexpr int kFtcEpiWarps = 8;                   // warps 11 .. 18: epilogue, two per TMEM lane quadrant
constexpr int kFtcMmaWarp = kFtcNoiseWarps + kFtcEpiWarps;  // warp 19
constexpr int kFtcThreads = 32 * (kFtcMmaWarp + 1);
constexpr int kFtcCols = 64;                       // N: 32 orders x (re, im)
constexpr uint32_t kFtcKTerm = 128u * 128u * 2u;   // one BF16 term of K_l: 2 halves x 128 j x 128 B
constexpr uint32_t kFtcNTerm = 128u * 128u;        // one BF16 term of a noise tile: 128 j x 128 B
constexpr uint32_t kFtcNBuf = 3u * kFtcNTerm;      // a noise buffer (three terms)
constexpr int kFtcQuads = (32 + kFtcNoiseWarps - 1) / kFtcNoiseWarps;  // shell quads of a noise warp, at most
constexpr int kFtcVs = 4 * kFtcQuads;              // its shells
// a^X_L partials: [buffer][noise warp][32 orders][T re, T im, E re, E im][hi, lo]
constexpr uint32_t kFtcPart = 2u * kFtcNoiseWarps * 32u * 8u * 4u;
constexpr uint32_t kFtcSmem = 1024 + 3 * kFtcKTerm + 2 * kFtcNBuf + kFtcNoiseWarps * 4 * kFtcVs * 4 + kFtcPart + 256;

struct FtcArgs {
  int L, nr, j0, ncol;    // the object's rows are shells j0 .. j0 + nr - 1; noise shells 0 .. ncol - 1
  int nterms, Cpad;       // BF16 terms and row length of the synthesis operand written here
  int64_t term_stride;    // elements between its terms
  int64_t nalm;
  const double* vT;       // [L+1][ncol]
  const double* vE;
  uint64_t seed, real;
  const double* noise;    // explicit [ncol][nalm][2], or NULL: Philox
  const int64_t* row32;
  __nv_bfloat16* phiT;
  double* phi_api;        // [nalm][nr][2] or NULL
  double* aLT;            // [nalm][2]
  double* aLE;
  double* psum_part;      // [L+1][2][nr] or NULL (the two halves of the orders)
  int* err;
};

// Instruction descriptor, kind::f16: BF16 x BF16 -> FP32, A and B MN-major, M = 128, N = 64.
__device__ __forceinline__ uint32_t idesc_ftc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) | ((uint32_t)(kFtcCols >> 3) << 17) |
         ((128u >> 4) << 24);
}

__device__ __forceinline__ void df_add(float& hi, float& lo, float p, float e) {
  const float s = hi + p;
  const float bb = s - hi;
  const float err = (hi - (s - bb)) + (p - bb) + lo + e;
  hi = s + err;
  lo = err - (hi - s);
}

// Packed FP32 pairs (one f32x2 instruction for both lanes of the pair).
__device__ __forceinline__ float2 pk2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }

// df_add on two independent double-float sums at once.
__device__ __forceinline__ void df_add2(float2& hi, float2& lo, float2 p, float2 e) {
  const float2 s = __fadd2_rn(hi, p);
  const float2 bb = sub2(s, hi);
  const float2 err = __fadd2_rn(__fadd2_rn(__fadd2_rn(sub2(hi, sub2(s, bb)), sub2(p, bb)), lo), e);
  hi = __fadd2_rn(s, err);
  lo = sub2(err, sub2(hi, s));
}

// The BF16 terms of the pair (x, y) (three terms: exact to 24 significant bits).
__device__ __forceinline__ void split_pair(float2 v, __nv_bfloat162& t0, __nv_bfloat162& t1, __nv_bfloat162& t2) {
  t0 = __floats2bfloat162_rn(v.x, v.y);
  const float2 r1 = sub2(v, make_float2(__low2float(t0), __high2float(t0)));
  t1 = __floats2bfloat162_rn(r1.x, r1.y);
  t2 = __floats2bfloat162_rn(r1.x - __low2float(t1), r1.y - __high2float(t1));
}

// Box-Muller of the tensor-core forms' noise from one Philox word, as box_muller_f32 but with the
// hardware's approximate transcendentals (absolute error of each below 2^-21 on the ranges used
// here): u1 = ((w >> 32) + 1) 2^-32, u2 = (w mod 2^32) 2^-32, rho = sqrt(-2 ln u1) and
// (cos, sin)(2 pi u2), the angle taken as 2 pi (u2 - 1/2) + pi so that the argument of the
// sine and cosine stays in [-pi, pi).
__device__ __forceinline__ float2 box_muller_fast(uint64_t w) {
  const uint32_t hi = (uint32_t)(w >> 32), lo = (uint32_t)w;
  const float u1 = hi == 0xffffffffu ? 1.0f : __uint2float_rn(hi + 1u) * 0x1p-32f;
  const float u2 = __uint2float_rn(lo) * 0x1p-32f;
  const float x = fmaxf(-2.0f * __logf(u1), 0.0f);
  const float rho = x > 0.0f ? x * rsqrtf(x) : 0.0f;
  float s, c;
  __sincosf(6.28318530717958648f * (u2 - 0.5f), &s, &c);
  return make_float2(-rho * c, -rho * s);
}

// Degree of round r for CTA b of G (snake order over the CTAs, largest degrees first); -1 past the end.
__device__ __forceinline__ int degree_of(int r, int b, int G, int L) {
  const int jb = r * G + ((r & 1) ? G - 1 - b : b);
  return jb > L ? -1 : L - jb;
}

__global__ void __launch_bounds__(kFtcThreads, 1)
    k_filter_tc(const __grid_constant__ FtcArgs a, const __grid_constant__ CUtensorMap tmK) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sK = smem;                            // [term][half][128 j][64 i], 128B swizzle
  unsigned char* sN = smem + 3 * kFtcKTerm;            // [buffer][term][128 j][64 col], 128B swizzle
  // per noise warp [4][16]: v^T hi, v^E hi, v^T lo, v^E lo of its 16 shells for the current degree
  // (no barrier across the noise warps, which could be left waiting if one of them unwinds)
  float* vs_all = (float*)(sN + 2 * kFtcNBuf);
  float* part = vs_all + kFtcNoiseWarps * 4 * kFtcVs;
  uint64_t* bars = (uint64_t*)(part + kFtcPart / 4);
  uint64_t* kfull = bars;       // K_l has landed
  uint64_t* kempty = bars + 1;  // the MMAs of the previous degree are done with K
  uint64_t* nfull = bars + 2;   // [2] noise buffer written (one arrive per noise warp)
  uint64_t* nempty = bars + 4;  // [2] noise buffer read by the MMAs
  uint64_t* tfull = bars + 6;   // [2] accumulator set complete
  uint64_t* tempty = bars + 8;  // [2] accumulator set read (one arrive per epilogue warp)
  uint64_t* drain = bars + 10;
  uint64_t* afull = bars + 11;   // [2] a^X_L partials written (one arrive per noise warp)
  uint64_t* aempty = bars + 13;  // [2] a^X_L partials summed (one arrive per epilogue warp)
  uint32_t* tslot = (uint32_t*)(bars + 15);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int G = gridDim.x, b = blockIdx.x, L = a.L;

  if (threadIdx.x == 0) {
    mbar_init(kfull, 1);
    mbar_init(kempty, 1);
    for (int s = 0; s < 2; ++s) {
      mbar_init(&nfull[s], kFtcNoiseWarps);
      mbar_init(&nempty[s], 1);
      mbar_init(&tfull[s], 1);
      mbar_init(&tempty[s], kFtcEpiWarps);
      mbar_init(&afull[s], kFtcNoiseWarps);
      mbar_init(&aempty[s], kFtcEpiWarps);
    }
    mbar_init(drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kFtcMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_u32(tslot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // the noise buffers start zeroed: rows of shells j >= ncol are never written and meet zero
  // columns of K_l (a stale NaN there would spoil every product)
  for (uint32_t e = threadIdx.x; e < 2 * kFtcNBuf / 16; e += blockDim.x) ((uint4*)sN)[e] = make_uint4(0, 0, 0, 0);
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp < kFtcNoiseWarps) {
    // ---------------------------------------------------------------- noise and a^X_L partials
    // lane = order m0 + lane of the chunk, warp w = shell quads w, w + 11, w + 22: a warp writes
    // whole 128-byte rows of the tile, and each lane sums its shells of a^X_L itself
    float* vs = vs_all + warp * 4 * kFtcVs;  // [4][kFtcVs]
    int cc = 0;
    bool ok = true;
    for (int r = 0; ok; ++r) {
      const int l = degree_of(r, b, G, L);
      if (l < 0) break;
      __syncwarp();  // the warp is done with the previous degree's v
      for (int e = lane; e < kFtcVs; e += 32) {
        const int j = 4 * (warp + kFtcNoiseWarps * (e >> 2)) + (e & 3);  // >= 128 past the last quad
        double t = 0.0, u = 0.0;
        if (j < a.ncol) t = a.vT[(size_t)l * a.ncol + j], u = a.vE[(size_t)l * a.ncol + j];
        vs[e] = (float)t;
        vs[kFtcVs + e] = (float)u;
        vs[2 * kFtcVs + e] = (float)(t - (double)(float)t);
        vs[3 * kFtcVs + e] = (float)(u - (double)(float)u);
      }
      __syncwarp();
      const int nch = l / 32 + 1;
      for (int c = 0; c < nch; ++c, ++cc) {
        const int s = cc & 1;
        const uint32_t ph = (cc >> 1) & 1;
        if (!mbar_wait(&nempty[s], ph ^ 1, a.err, 11) || !mbar_wait(&aempty[s], ph ^ 1, a.err, 17)) {
          ok = false;
          break;
        }
        unsigned char* nb = sN + (size_t)s * kFtcNBuf;
        const int m = 32 * c + lane;
        const bool mvalid = m <= l;
        const int64_t idx = mvalid ? alm_idx(l, m, L) : 0;
        // (re, im) double-float sums of T and E
        float2 h2[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)}, lo2[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll 1
        for (int qd = 0; qd < kFtcQuads; ++qd) {
          const int jq = warp + kFtcNoiseWarps * qd;
          if (4 * jq >= a.ncol) break;  // warp-uniform
          float2 nz[4] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
          if (mvalid) {
            if (a.noise) {
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                const int j = 4 * jq + e;
                if (j < a.ncol) {
                  const double2 d = ((const double2*)a.noise)[(size_t)j * a.nalm + idx];
                  nz[e] = make_float2((float)d.x, m == 0 ? 0.f : (float)d.y);
                }
              }
            } else {
              uint64_t w[4];
              noise_words(a.seed, a.real, idx, jq, w);
#pragma unroll
              for (int e = 0; e < 4; ++e)
                if (4 * jq + e < a.ncol) nz[e] = noise_value_f32(box_muller_fast(w[e]), m);
            }
          }
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int j = 4 * jq + e;
            if (j >= a.ncol) break;
            // row j of the tile, column pair (2 lane, 2 lane + 1), three terms
            __nv_bfloat162 p0, p1, p2;
            split_pair(nz[e], p0, p1, p2);
            const uint32_t off = (uint32_t)j * 128u + ((((uint32_t)lane >> 2) ^ ((uint32_t)j & 7u)) << 4) +
                                 (((uint32_t)lane & 3u) << 2);
            *(__nv_bfloat162*)(nb + off) = p0;
            *(__nv_bfloat162*)(nb + kFtcNTerm + off) = p1;
            *(__nv_bfloat162*)(nb + 2 * kFtcNTerm + off) = p2;
            const int ve = 4 * qd + e;
#pragma unroll
            for (int f = 0; f < 2; ++f) {
              const float2 vh = pk2(vs[kFtcVs * f + ve]), vl = pk2(vs[kFtcVs * (2 + f) + ve]);
              const float2 pr = __fmul2_rn(vh, nz[e]);
              df_add2(h2[f], lo2[f], pr, __ffma2_rn(vl, nz[e], __ffma2_rn(vh, nz[e], make_float2(-pr.x, -pr.y))));
            }
          }
        }
        float* pw = part + (((size_t)s * kFtcNoiseWarps + warp) * 32 + lane) * 8;
#pragma unroll
        for (int f = 0; f < 2; ++f) {  // [T re, T im, E re, E im][hi, lo]
          *(float4*)(pw + 4 * f) = make_float4(h2[f].x, lo2[f].x, h2[f].y, lo2[f].y);
        }
        fence_proxy_async();  // the tile's generic-proxy writes, visible to the tensor core
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&nfull[s]);
          mbar_arrive(&afull[s]);
        }
      }
    }
  } else if (warp < kFtcMmaWarp) {
    // ---------------------------------------------------------------- epilogue
    const int q = warp & 3;           // TMEM lane quadrant: shells 32 q .. 32 q + 31
    const int h = (warp - kFtcNoiseWarps) >> 2;  // which half of a chunk's orders: 16 h .. 16 h + 15
    const int i = 32 * q + lane;      // this lane's shell (local index)
    const bool ivalid = i < a.nr;
    // sum_m w_m |Phi_L,lm(r_i)|^2 of the current degree, double-float: (re^2, im^2) pairs in two
    // independent sums (orders m mod 2), joined at the end of the degree
    float2 ph[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)}, pl[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    int cc = 0;
    bool ok = true;
    for (int r = 0; ok; ++r) {
      const int l = degree_of(r, b, G, L);
      if (l < 0) break;
      const int nch = l / 32 + 1;
      for (int c = 0; c < nch; ++c, ++cc) {
        const int s = cc & 1;
        const uint32_t par = (cc >> 1) & 1;
        // a^X_L of the chunk's orders: thread (order, value) adds the noise warps' partials
        if (!mbar_wait(&afull[s], par, a.err, 18)) {
          ok = false;
          break;
        }
        {
          // the half's 16 orders x 4 values over 128 threads: two threads per sum (noise warps
          // of either parity), joined across the lane pair
          const int t = 32 * q + lane, mi = 16 * h + (t >> 3), v = (t >> 1) & 3, par2 = t & 1;
          const int m = 32 * c + mi;
          float hs = 0.f, ls = 0.f;
#pragma unroll
          for (int w = par2; w < kFtcNoiseWarps; w += 2) {
            const float* pw = part + (((size_t)s * kFtcNoiseWarps + w) * 32 + mi) * 8 + 2 * v;
            df_add(hs, ls, pw[0], pw[1]);
          }
          const float oh = __shfl_xor_sync(0xffffffffu, hs, 1), ol = __shfl_xor_sync(0xffffffffu, ls, 1);
          df_add(hs, ls, oh, ol);
          if (par2 == 0 && m <= l) {
            const int64_t idx = alm_idx(l, m, L);
            (v < 2 ? a.aLT : a.aLE)[2 * idx + (v & 1)] = (double)hs + (double)ls;
          }
          __syncwarp();
          if (lane == 0) mbar_arrive(&aempty[s]);
        }
        if (!mbar_wait(&tfull[s], par, a.err, 12)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t ta = tmem + (uint32_t)(s * 2 * kFtcCols) + ((uint32_t)(32 * q) << 16);
        // the Phi row of order m0 + lane, passed to the other lanes by shuffles
        int64_t rowv = 0;
        {
          const int m = 32 * c + lane;
          if (m <= l) rowv = a.row32[2 * m + ((l - m) & 1)] + ((l - m) >> 1);
        }
        // the half's two groups of 8 orders: 16 columns of both accumulators each
#pragma unroll 1
        for (int g = 2 * h; g < 2 * h + 2; ++g) {
          float v[16];
          {
            float y[16];
            tmem_ld16_pair(ta + (uint32_t)(16 * g), ta + (uint32_t)(kFtcCols + 16 * g), v, y);
#pragma unroll
            for (int k = 0; k < 16; ++k) v[k] += y[k];
          }
          if (g == 2 * h + 1) {
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[s]);
          }
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const int mi = 8 * g + k, m = 32 * c + mi;
            const int64_t row = __shfl_sync(0xffffffffu, rowv, mi);
            if (!ivalid || m > l) continue;
            const float2 z = make_float2(v[2 * k], v[2 * k + 1]);
            __nv_bfloat162 t0, t1, t2;
            split_pair(z, t0, t1, t2);
            __nv_bfloat16* dst = a.phiT + row * a.Cpad + 2 * i;
            *(__nv_bfloat162*)dst = t0;
            *(__nv_bfloat162*)(dst + a.term_stride) = t1;
            if (a.nterms > 2) *(__nv_bfloat162*)(dst + 2 * a.term_stride) = t2;
            if (a.phi_api) {
              const int64_t idx = alm_idx(l, m, L);
              *(double2*)(a.phi_api + ((size_t)idx * a.nr + i) * 2) = make_double2((double)z.x, (double)z.y);
            }
            // w_m (re^2, im^2) exactly as p + e (w is 1 or 2)
            const float2 zw = __fmul2_rn(z, pk2(m == 0 ? 1.f : 2.f));
            const float2 p = __fmul2_rn(zw, z);
            df_add2(ph[k & 1], pl[k & 1], p, __ffma2_rn(zw, z, make_float2(-p.x, -p.y)));
          }
        }
      }
      if (!ok) break;
      df_add2(ph[0], pl[0], ph[1], pl[1]);
      float sh = ph[0].x, sl = pl[0].x;
      df_add(sh, sl, ph[0].y, pl[0].y);
      if (a.psum_part && ivalid) a.psum_part[((size_t)l * 2 + h) * a.nr + i] = (double)sh + (double)sl;
#pragma unroll
      for (int k = 0; k < 2; ++k) ph[k] = pl[k] = make_float2(0.f, 0.f);
    }
  } else if (lane == 0) {
    // ---------------------------------------------------------------- K_l loads and MMAs
    const uint32_t idesc = idesc_ftc();
    const uint32_t kbase = smem_u32(sK), nbase = smem_u32(sN);
    int cc = 0;
    uint32_t kf_par = 0, ke_par = 0;
    bool ok = true, kpending = false;
    for (int r = 0; ok; ++r) {
      const int l = degree_of(r, b, G, L);
      if (l < 0) break;
      if (r > 0) {  // the previous degree's MMAs are done with the K buffer
        if (!mbar_wait(kempty, ke_par, a.err, 13)) break;
        ke_par ^= 1;
      }
      mbar_expect_tx(kfull, 3 * kFtcKTerm);
      tma_load_5d(kbase, &tmK, 0, 0, 0, l, 0, kfull);
      kpending = true;
      const int nch = l / 32 + 1;
      for (int c = 0; c < nch; ++c, ++cc) {
        const int s = cc & 1;
        const uint32_t par = (cc >> 1) & 1;
        if (!mbar_wait(&tempty[s], par ^ 1, a.err, 14) || !mbar_wait(&nfull[s], par, a.err, 15)) {
          ok = false;
          break;
        }
        if (c == 0) {
          if (!mbar_wait(kfull, kf_par, a.err, 16)) {
            ok = false;
            break;
          }
          kf_par ^= 1;
          kpending = false;
        }
        tc_fence_after();
        const uint32_t d0 = tmem + (uint32_t)(s * 2 * kFtcCols), d1 = d0 + (uint32_t)kFtcCols;
        const uint32_t nb = nbase + (uint32_t)s * kFtcNBuf;
        // A: 16 KB between the 64-shell halves, 1 KB per 8 k rows, 128B swizzle; B: one 64-column
        // block, 1 KB per 8 k rows; a k step of 16 rows is 2 KB further in both
        const uint64_t da = sdesc(kbase, 16384, 1024, 2), db = sdesc(nb, 16384, 1024, 2);
        int corr = 0;
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
#pragma unroll
          for (int ta = 0; ta < 3; ++ta) {
#pragma unroll
            for (int tb = 0; ta + tb < 3; ++tb) {
              const uint64_t ad = da + (uint64_t)((ta * kFtcKTerm + kk * 2048u) >> 4);
              const uint64_t bd = db + (uint64_t)((tb * kFtcNTerm + kk * 2048u) >> 4);
              if (ta | tb) {
                tc_mma(d1, ad, bd, idesc, corr ? 1u : 0u);
                ++corr;
              } else {
                tc_mma(d0, ad, bd, idesc, kk ? 1u : 0u);
              }
            }
          }
        }
        tc_commit(&nempty[s]);
        tc_commit(&tfull[s]);
      }
      if (!ok) break;
      tc_commit(kempty);
    }
    if (kpending) {  // a K load still in flight lands before the CTA unwinds (bounded)
      for (uint32_t t = 0; t < kTcWaitLimit && !mbar_try_wait(kfull, kf_par); ++t) {
      }
    }
    // every MMA this thread issued has completed before TMEM is released (bounded)
    tc_commit(drain);
    for (uint32_t t = 0; t < kTcWaitLimit && !mbar_try_wait(drain, 0); ++t) {
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == kFtcMmaWarp) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem) : "memory");
  }
}

}  // namespace

// BF16 terms of the filters for the tensor-core filter and their tensor map: [term][l][j][i] with
// shells i (the object's rows) contiguous, 128 x 128 per degree (zero outside rows < nr, columns
// j <= j0 + i); one TMA box holds a degree's three terms as [term][half of i][j][64 i].
void build_filter_terms(fnl_shells* sh, const std::vector<double>& Kf) {
  const int L = sh->lmax, nr = sh->nr, j0 = sh->j0, ncol = j0 + nr;
  const size_t per = 128 * 128, nl = (size_t)L + 1;
  std::vector<__nv_bfloat16> kt(3 * nl * per, __float2bfloat16_rn(0.f));
  for (int l = 0; l <= L; ++l)
    for (int i = 0; i < nr; ++i)
      for (int j = 0; j <= j0 + i && j < ncol; ++j) {
        const float v = (float)Kf[((size_t)l * nr + i) * ncol + j];
        const __nv_bfloat16 t0 = __float2bfloat16_rn(v);
        const float r1 = v - __bfloat162float(t0);
        const __nv_bfloat16 t1 = __float2bfloat16_rn(r1);
        const __nv_bfloat16 t2 = __float2bfloat16_rn(r1 - __bfloat162float(t1));
        const size_t o = ((size_t)l * 128 + j) * 128 + i;
        kt[o] = t0;
        kt[nl * per + o] = t1;
        kt[2 * nl * per + o] = t2;
      }
  const size_t bytes = sizeof(__nv_bfloat16) * kt.size();
  void* d = device_malloc(bytes);
  sh->allocations.push_back(d);
  sh->device_bytes += bytes;
  FNL_CUDA(cudaMemcpy(d, kt.data(), bytes, cudaMemcpyHostToDevice));
  sh->d_Kterm = d;
  const uint64_t dims[5] = {64, 128, 2, nl, 3};
  const uint64_t str[4] = {256, 128, 128 * 256, nl * 128 * 256};
  const uint32_t box[5] = {64, 128, 2, 1, 3};
  sh->tmK = make_tensor_map_bf16(sh->d_Kterm, 5, dims, str, box, 128);
}

// Step (i) on the tensor cores; psum_part [L+1][nr] receives the per-degree monopole sums (or NULL).
void launch_filter_tc(const fnl_shells* sh, uint64_t seed, uint64_t real, const double* noise, double* aLT,
                      double* aLE, double* phi_api, double* psum_part, cudaStream_t st) {
  FtcArgs a;
  a.L = sh->lmax;
  a.nr = sh->nr;
  a.j0 = sh->j0;
  a.ncol = sh->j0 + sh->nr;
  a.nterms = sh->nterms;
  a.Cpad = sh->Cpad;
  a.term_stride = sh->phiT_stride;
  a.nalm = sh->nalm;
  a.vT = sh->d_vT;
  a.vE = sh->d_vE;
  a.seed = seed;
  a.real = real;
  a.noise = noise;
  a.row32 = sh->d_row32;
  a.phiT = (__nv_bfloat16*)sh->d_phiT;
  a.phi_api = phi_api;
  a.aLT = aLT;
  a.aLE = aLE;
  a.psum_part = psum_part;
  a.err = sh->d_err;
  FNL_CUDA(cudaFuncSetAttribute(k_filter_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFtcSmem));
  const int grid = std::max(1, std::min(sh->sms, sh->lmax + 1));
  k_filter_tc<<<grid, kFtcThreads, kFtcSmem, st>>>(a, sh->tmK);
  FNL_CUDA(cudaGetLastError());
}

}  // namespace fnl
