// Kernels of the mixed-precision forms (FNL_BF16X2, FNL_BF16X3) around the tensor-core
// Legendre GEMMs:
//   k_filter_gemm     step (i) in FP32: Phi_L = K_l n (Eq. 9) written as BF16 terms, and
//                     a^X_L = v^X_l . n (Eq. 5) summed in FP32 and stored as FP64; also the
//                     per-shell sums of |Phi_L,lm|^2 for the Parseval monopole
//   k_lambda_mixed    lambda_lm(x_jp) from the FP64 recurrence, split into BF16 terms in the
//                     two K-contiguous layouts of the synthesis and analysis GEMMs
//   k_alm_to_terms    API coefficients -> BF16 terms of the synthesis operand
//   k_combine_mixed   a^X_NL = sum over column tiles of the GEMM epilogue's FP64 partials,
//                     a^X = a^X_L + f_NL a^X_NL (Eq. 3)
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "fnl_internal.cuh"
#include "mixed.cuh"
#include "philox.cuh"

namespace fnl {

namespace {

constexpr int kThreads = 256;

// Double-float accumulation (hi + lo, ~48 significant bits from FP32 operations):
// the exact square of x (product and fmaf residual) is added with a two-sum.
__device__ __forceinline__ void df_add(float& hi, float& lo, float p, float e) {
  const float s = hi + p;
  const float bb = s - hi;
  const float err = (hi - (s - bb)) + (p - bb) + lo + e;
  hi = s + err;
  lo = err - (hi - s);
}

__device__ __forceinline__ void df_add_square(float& hi, float& lo, float x, float w) {
  const float xw = x * w;  // w is 1 or 2: exact
  const float p = xw * x;
  const float e = fmaf(xw, x, -p);
  const float s = hi + p;
  const float bb = s - hi;
  const float err = (hi - (s - bb)) + (p - bb) + lo + e;
  hi = s + err;
  lo = err - (hi - s);
}

// Step (i) as a register-tiled FP32 GEMM per degree l (block per l, largest first):
//   Phi_l[i][col] = sum_{j <= j0 + i} K_l[j0 + i][j] n_l[j][col],  col = 2 (m - m0) + {re, im}
// over chunks of 32 orders m (64 columns), for the object's nr rows, shells j0 .. j0 + nr - 1
// of its configuration (j0 = 0 unless it is a shell shard), which need the noise of shells
// 0 .. ncol - 1 (ncol = j0 + nr).  K_l is staged transposed in shared memory.  K_l is lower
// triangular, so row tile t (rows 4t .. 4t + 3) needs j0 + 4t + 4 terms: each thread owns
// the 4-row tiles r and nt4 - 1 - r (r = thread row, warp-uniform up to one) times 4 columns,
// which gives every thread and every warp the same number of multiply-adds.  The noise tile
// is drawn by all threads (Philox4x64, one call per four shells, + FP32 Box-Muller); a^X_L = v^X_l . n per column
// (Eq. 5 applied to Eq. 9), each dot product split over two threads.
constexpr int kFCols = 64;

// Row stride of the output tile [col][i]: a multiple of 4 floats with an odd quotient, so
// that the float4 stores of 8 lanes (consecutive column blocks) hit distinct bank quads.
__host__ __device__ inline int out_stride(int nrp) { return nrp + 4; }

__device__ __forceinline__ void filter_body(int l, int L, int nr, int j0, int ncol, int Cpad, int nterms,
                                            int64_t term_stride,
                                                             const float* __restrict__ Kft,
                                                             const double* __restrict__ vT,
                                                             const double* __restrict__ vE, uint64_t seed,
                                                             uint64_t real, const double* __restrict__ noise,
                                                             const int64_t* __restrict__ row32,
                                                             __nv_bfloat16* __restrict__ phiT,
                                                             double* __restrict__ phi_api, double* __restrict__ aLT,
                                                             double* __restrict__ aLE, double* __restrict__ psum) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int nrp = (nr + 7) / 8 * 8;        // rows padded to the 8-row thread tiles
  float* Kt = (float*)smem;                // [ncol][nrp]  Kt[j][i] = K_l[j0 + i][j]
  // output tile [col][i], row stride os (see out_stride)
  const int os = out_stride(nrp);
  float* nt = Kt + (size_t)ncol * nrp;     // [ncol][kFCols] noise tile, then [kFCols][os] output tile
  // [4][ncol]: v^T hi, v^E hi, v^T lo, v^E lo; then [2][kFCols][2] partial a^X_L sums (dfp)
  float* vs = nt + (size_t)max(ncol * kFCols, kFCols * os);
  // K_l arrives transposed and padded (set-up): a straight copy of ncol * nrp floats
  {
    const float4* src = (const float4*)(Kft + (size_t)l * ncol * nrp);
    float4* dst = (float4*)Kt;
    for (int e = threadIdx.x; e < ncol * nrp / 4; e += kThreads) dst[e] = src[e];
  }
  for (int e = threadIdx.x; e < ncol; e += kThreads) {
    const double t = vT[(size_t)l * ncol + e], u = vE[(size_t)l * ncol + e];
    vs[e] = (float)t;
    vs[ncol + e] = (float)u;
    vs[2 * ncol + e] = (float)(t - (double)(float)t);
    vs[3 * ncol + e] = (float)(u - (double)(float)u);
  }
  const int64_t nalm = (int64_t)(L + 1) * (L + 2) / 2;
  const int nquad = (ncol + 3) / 4;
  // GEMM: thread row r = tid / 16 owns row tiles ta = r and tb = nt4 - 1 - r, columns 4 cb ..
  const int r4 = threadIdx.x >> 4, cb = threadIdx.x & 15;
  const int nt4 = nrp / 4, ta = r4, tb = nt4 - 1 - r4;
  const bool rows_active = r4 < nt4 / 2;
  const int ja = min(ncol, j0 + 4 * ta + 4), jb = min(ncol, j0 + 4 * tb + 4);
  float* dfp = vs + 4 * ncol;              // [2][kFCols][2]: second halves of the a^X_L sums
  // write-out phase: thread -> shell ws = threadIdx.x % 128, orders mb = threadIdx.x / 128 (+2 ...)
  const int ws = threadIdx.x & 127, wh = threadIdx.x >> 7;
  float ph = 0.f, pl = 0.f;  // sum_m w_m |Phi_L,lm(r_ws)|^2 over this thread's orders (double-float)

  for (int m0 = 0; m0 <= l; m0 += kFCols / 2) {
    const int nm = min(kFCols / 2, l + 1 - m0);
    __syncthreads();
    // ---- noise tile n[j][col]
    if (noise) {
      for (int t = threadIdx.x; t < ncol * (kFCols / 2); t += kThreads) {
        const int j = t / (kFCols / 2), mb = t % (kFCols / 2), m = m0 + mb;
        float2 v = make_float2(0.f, 0.f);
        if (mb < nm) {
          const double2 d = ((const double2*)noise)[(size_t)j * nalm + alm_idx(l, m, L)];
          v = make_float2((float)d.x, m == 0 ? 0.f : (float)d.y);
        }
        *(float2*)(nt + (size_t)j * kFCols + 2 * mb) = v;
      }
    } else {
      // one Philox call gives the draws of four shells (one 64-bit word each)
      for (int t = threadIdx.x; t < nquad * (kFCols / 2); t += kThreads) {
        const int jq = t / (kFCols / 2), mb = t % (kFCols / 2), m = m0 + mb;
        uint64_t w[4] = {0, 0, 0, 0};
        if (mb < nm) noise_words(seed, real, alm_idx(l, m, L), jq, w);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int j = 4 * jq + q;
          if (j >= ncol) break;
          const float2 v = mb < nm ? noise_value_f32(box_muller_f32(w[q]), m) : make_float2(0.f, 0.f);
          *(float2*)(nt + (size_t)j * kFCols + 2 * mb) = v;
        }
      }
    }
    __syncthreads();
    // ---- a^X_L for the chunk: thread (half h, field f, column col) sums half of the j range;
    // exact products, double-float sums; the second halves are added after the next barrier
    const int acol = threadIdx.x & (kFCols - 1), af = (threadIdx.x >> 6) & 1, ah = threadIdx.x >> 7;
    const bool a_active = (acol >> 1) < nm;
    float sh = 0.f, sl = 0.f;
    if (a_active) {
      const float* vh = vs + af * ncol;
      const float* vl = vs + (2 + af) * ncol;
      const int jlo = ah ? ncol / 2 : 0, jhi = ah ? ncol : ncol / 2;
      for (int j = jlo; j < jhi; ++j) {
        const float n = nt[(size_t)j * kFCols + acol];
        const float p = vh[j] * n;
        df_add(sh, sl, p, fmaf(vh[j], n, -p) + vl[j] * n);
      }
      if (ah) {
        dfp[(af * kFCols + acol) * 2] = sh;
        dfp[(af * kFCols + acol) * 2 + 1] = sl;
      }
    }
    // ---- Phi_L for the chunk: row tiles ta and tb x 4 columns per thread
    float acc[8][4];
#pragma unroll
    for (int q = 0; q < 8; ++q)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[q][c] = 0.f;
    if (rows_active) {
      const float* kta = Kt + 4 * ta;
      const float* ktb = Kt + 4 * tb;
      const float* nvp = nt + 4 * cb;
      int j = 0;
      for (; j < ja; ++j) {
        const float4 k0 = *(const float4*)(kta + (size_t)j * nrp);
        const float4 k1 = *(const float4*)(ktb + (size_t)j * nrp);
        const float4 nv = *(const float4*)(nvp + (size_t)j * kFCols);
        const float kk[8] = {k0.x, k0.y, k0.z, k0.w, k1.x, k1.y, k1.z, k1.w};
        const float nn[4] = {nv.x, nv.y, nv.z, nv.w};
#pragma unroll
        for (int q = 0; q < 8; ++q)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[q][c] = fmaf(kk[q], nn[c], acc[q][c]);
      }
      for (; j < jb; ++j) {
        const float4 k1 = *(const float4*)(ktb + (size_t)j * nrp);
        const float4 nv = *(const float4*)(nvp + (size_t)j * kFCols);
        const float kk[4] = {k1.x, k1.y, k1.z, k1.w};
        const float nn[4] = {nv.x, nv.y, nv.z, nv.w};
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[4 + q][c] = fmaf(kk[q], nn[c], acc[4 + q][c]);
      }
    }
    __syncthreads();  // the noise tile is no longer read: reuse it as the output tile [col][i]
    if (a_active && !ah) {
      df_add(sh, sl, dfp[(af * kFCols + acol) * 2], dfp[(af * kFCols + acol) * 2 + 1]);
      const int64_t idx = alm_idx(l, m0 + (acol >> 1), L);
      (af ? aLE : aLT)[2 * idx + (acol & 1)] = (double)sh + (double)sl;
    }
    if (rows_active) {
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        float* o = nt + (size_t)(4 * cb + c) * os;
        *(float4*)(o + 4 * ta) = make_float4(acc[0][c], acc[1][c], acc[2][c], acc[3][c]);
        *(float4*)(o + 4 * tb) = make_float4(acc[4][c], acc[5][c], acc[6][c], acc[7][c]);
      }
    }
    __syncthreads();
    // ---- write-out: rows (l, m) of Phi as BF16 terms, c = 2 i + {re, im} contiguous
    if (ws < nr) {
      for (int mb = wh; mb < nm; mb += kThreads / 128) {
        const int m = m0 + mb;
        const int p = (l - m) & 1;
        const int64_t row = row32[2 * m + p] + ((l - m) >> 1);
        const float re = nt[(size_t)(2 * mb) * os + ws];
        const float im = nt[(size_t)(2 * mb + 1) * os + ws];
        __nv_bfloat162 t0, t1, t2;
        const __nv_bfloat16 r0 = __float2bfloat16_rn(re), i0 = __float2bfloat16_rn(im);
        const float rr1 = re - __bfloat162float(r0), ir1 = im - __bfloat162float(i0);
        const __nv_bfloat16 r1 = __float2bfloat16_rn(rr1), i1 = __float2bfloat16_rn(ir1);
        t0.x = r0; t0.y = i0;
        t1.x = r1; t1.y = i1;
        t2.x = __float2bfloat16_rn(rr1 - __bfloat162float(r1));
        t2.y = __float2bfloat16_rn(ir1 - __bfloat162float(i1));
        __nv_bfloat16* dst = phiT + row * Cpad + 2 * ws;
        *(__nv_bfloat162*)dst = t0;
        *(__nv_bfloat162*)(dst + term_stride) = t1;
        if (nterms > 2) *(__nv_bfloat162*)(dst + 2 * term_stride) = t2;
        if (phi_api) {
          const int64_t idx = alm_idx(l, m, L);
          *(double2*)(phi_api + ((size_t)idx * nr + ws) * 2) = make_double2((double)re, (double)im);
        }
        if (psum) {
          const float wm = m == 0 ? 1.f : 2.f;
          df_add_square(ph, pl, re, wm);
          df_add_square(ph, pl, im, wm);
        }
      }
    }
  }
  // one partial per (l, half of the orders, shell): summed in a fixed order by k_psum_reduce,
  // so the monopole (and every result) is reproducible bit for bit
  if (psum && ws < nr) psum[((size_t)(L - l) * (kThreads / 128) + wh) * nr + ws] = (double)ph + (double)pl;
}

// One configuration: block b takes degree l = L - b (largest first).
__global__ void __launch_bounds__(kThreads, 2) k_filter_gemm(int L, int nr, int j0, int Cpad, int nterms,
                                                             int64_t term_stride,
                                                             const float* __restrict__ Kft,
                                                             const double* __restrict__ vT,
                                                             const double* __restrict__ vE, uint64_t seed,
                                                             uint64_t real, const double* __restrict__ noise,
                                                             const int64_t* __restrict__ row32,
                                                             __nv_bfloat16* __restrict__ phiT,
                                                             double* __restrict__ phi_api, double* __restrict__ aLT,
                                                             double* __restrict__ aLE, double* __restrict__ psum) {
  filter_body(L - (int)blockIdx.x, L, nr, j0, j0 + nr, Cpad, nterms, term_stride, Kft, vT, vE, seed, real, noise,
              row32, phiT, phi_api, aLT, aLE, psum);
}

// Several instances in one launch: block b takes (instance, degree) = blocks[b] (ordered by
// descending degree across instances); the noise keys come with the launch.
__global__ void __launch_bounds__(kThreads, 2) k_filter_multi(const FilterInst* __restrict__ inst,
                                                              const int2* __restrict__ blocks, const MultiKeys keys) {
  const int2 b = blocks[blockIdx.x];
  const FilterInst f = inst[b.x];
  filter_body(b.y, f.L, f.nr, 0, f.nr, f.Cpad, f.nterms, f.term_stride, f.Kft, f.vT, f.vE, keys.seed[b.x],
              keys.real[b.x], nullptr, f.row32, f.phiT, nullptr, f.aLT, f.aLE, f.psum_part);
}

// psum[s] = sum over the filter's partials of shell s: strided per-thread sums, then a tree
// over the block, both in a fixed order (the result does not depend on timing).
__device__ __forceinline__ void psum_body(int s, int nparts, int nr, const double* __restrict__ part,
                                          double* __restrict__ psum) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int e = threadIdx.x; e < nparts; e += 256) acc += part[(size_t)e * nr + s];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) psum[s] = red[0];
}

__global__ void __launch_bounds__(256) k_psum_reduce(int nparts, int nr, const double* __restrict__ part,
                                                     double* __restrict__ psum) {
  psum_body(blockIdx.x, nparts, nr, part, psum);
}

// Several instances: block (s, i) sums shell s of instance i.
__global__ void __launch_bounds__(256) k_psum_multi(const FilterInst* __restrict__ inst) {
  const FilterInst& f = inst[blockIdx.y];
  if ((int)blockIdx.x >= f.nr) return;
  psum_body(blockIdx.x, (f.L + 1) * (kThreads / 128), f.nr, f.psum_part, f.psum);
}

__device__ __forceinline__ double flushed(double v) { return fabs(v) < 1e-290 ? 0.0 : v; }

// One thread per (jp, m): lambda_lm(x_jp) for l = m..L by the FP64 recurrence, written as BF16
// terms into Lambda_syn[slab(mp, k / 32)][jp][k % 32] and Lambda_ana[row16(mp) + k][jp].
__global__ void k_lambda_mixed(const double* __restrict__ x, const double* __restrict__ mant,
                               const int* __restrict__ expo, const double2* __restrict__ ab,
                               const int64_t* __restrict__ row32, const int64_t* __restrict__ row16, int npairs,
                               int npj, int L, int nterms, int64_t syn_stride, int64_t ana_stride,
                               __nv_bfloat16* __restrict__ lsyn, __nv_bfloat16* __restrict__ lana) {
  const int jp = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = blockIdx.y;
  if (jp >= npairs) return;
  const double xx = x[jp];
  double y1 = mant[(size_t)m * npairs + jp], y2 = 0.0;
  int e = expo[(size_t)m * npairs + jp];
  const int64_t base = alm_idx(0, m, L);
  for (int l = m; l <= L; ++l) {
    if (l > m) {
      const double2 c = ab[base + l];
      const double y = c.x * (xx * y1 - c.y * y2);
      y2 = y1;
      y1 = y;
      if (fabs(y1) > 0x1p500) {
        y1 *= 0x1p-500;
        y2 *= 0x1p-500;
        e += 500;
      }
    }
    const double v = flushed(ldexp(y1, e));
    const int d = l - m, p = d & 1, k = d >> 1;
    const int mp = 2 * m + p;
    const int64_t slab = row32[mp] / 32 + k / 32;
    store_terms_d(lsyn + (slab * npairs + jp) * 32 + (k & 31), syn_stride, nterms, v);
    store_terms_d(lana + (row16[mp] + k) * (int64_t)npj + jp, ana_stride, nterms, v);
  }
}

// API coefficients [nalm][nr][2] -> BF16 terms of Phi rows (row32 packing, Cpad columns).
__global__ void k_alm_to_terms(int L, int nr, int Cpad, int64_t nalm, int nterms, int64_t term_stride,
                               const int64_t* __restrict__ row32, const double* __restrict__ alm,
                               __nv_bfloat16* __restrict__ phiT) {
  const int C = 2 * nr;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nalm * C) return;
  const int64_t idx = t / C;
  const int c = (int)(t % C);
  const float b = 2.0f * L + 3.0f;
  int m = (int)floorf((b - sqrtf(fmaxf(b * b - 8.0f * (float)idx, 0.0f))) * 0.5f);
  m = max(0, min(m, L));
  while (m > 0 && alm_idx(m, m, L) > idx) --m;
  while (m < L && alm_idx(m + 1, m + 1, L) <= idx) ++m;
  const int l = (int)(idx - alm_idx(0, m, L));
  double v = alm[(size_t)idx * C + c];
  if (m == 0 && (c & 1)) v = 0.0;
  store_terms(phiT + (row32[2 * m + ((l - m) & 1)] + ((l - m) >> 1)) * Cpad + c, term_stride, nterms, (float)v);
}

// a^X_NL,lm = sum over column tiles of the epilogue partials; for (l, m) = (0, 0) the
// monopole comes from Parseval's identity instead:
//   Phi_NL,00(r_i) = (sum_lm w_m |Phi_L,lm(r_i)|^2 - 4 pi mu_i) / sqrt(4 pi),  w_0 = 1, w_m>0 = 2,
// a difference of two nearly equal numbers that FP32 grid sums would resolve poorly.  The
// identity is what the grid's own analysis gives on every grid the library accepts, not only
// on the exact-square ones: the monopole integrates f^2, whose ring mean is exact once
// n_phi > 2 l_max (frequencies up to 2 l_max, none aliased onto m = 0), and whose ring means
// |F_m(theta)|^2 are polynomials of degree <= 2 l_max in cos theta, which the n_theta-point
// Gauss-Legendre rule integrates exactly once n_theta >= l_max + 1.
__device__ __forceinline__ void combine_body(int64_t i, int64_t nalm, int nct, int nr, double fnl,
                                             const double2* __restrict__ part, const double* __restrict__ psum,
                                             const double* __restrict__ mu, const double* __restrict__ qT,
                                             const double* __restrict__ qE, const double2* __restrict__ aLT,
                                             const double2* __restrict__ aLE, double2* __restrict__ aNLT,
                                             double2* __restrict__ aNLE, double2* __restrict__ aT,
                                             double2* __restrict__ aE) {
  if (i >= nalm) return;
  double tr = 0, ti = 0, er = 0, ei = 0;
  if (i == 0 && psum) {
    for (int s = 0; s < nr; ++s) {
      const double phi00 = (psum[s] - 12.566370614359172954 * mu[s]) * 0.28209479177387814347;
      tr += qT[s] * phi00;
      er += qE[s] * phi00;
    }
  } else {
    for (int c = 0; c < nct; ++c) {
      const double2 t = part[((size_t)c * nalm + i) * 2], e = part[((size_t)c * nalm + i) * 2 + 1];
      tr += t.x;
      ti += t.y;
      er += e.x;
      ei += e.y;
    }
  }
  aNLT[i] = make_double2(tr, ti);
  aNLE[i] = make_double2(er, ei);
  if (aT) {
    const double2 a = aLT[i];
    aT[i] = make_double2(a.x + fnl * tr, a.y + fnl * ti);
  }
  if (aE) {
    const double2 a = aLE[i];
    aE[i] = make_double2(a.x + fnl * er, a.y + fnl * ei);
  }
}

__global__ void k_combine_mixed(int64_t nalm, int nct, int nr, double fnl, const double2* __restrict__ part,
                                const double* __restrict__ psum, const double* __restrict__ mu,
                                const double* __restrict__ qT, const double* __restrict__ qE,
                                const double2* __restrict__ aLT, const double2* __restrict__ aLE,
                                double2* __restrict__ aNLT, double2* __restrict__ aNLE, double2* __restrict__ aT,
                                double2* __restrict__ aE) {
  combine_body((int64_t)blockIdx.x * blockDim.x + threadIdx.x, nalm, nct, nr, fnl, part, psum, mu, qT, qE, aLT, aLE,
               aNLT, aNLE, aT, aE);
}

// Several instances: block row blockIdx.y is instance i; f_NL and the outputs come with the launch.
__global__ void k_combine_multi(const CombineInst* __restrict__ inst, const MultiOut out) {
  const int n = blockIdx.y;
  const CombineInst& c = inst[n];
  combine_body((int64_t)blockIdx.x * blockDim.x + threadIdx.x, c.nalm, c.nct, c.nr, out.fnl[n], c.part, c.psum, c.mu,
               c.qT, c.qE, c.aLT, c.aLE, c.aNLT, c.aNLE, out.aT[n], out.aE[n]);
}

}  // namespace

void launch_filter_multi(const FilterInst* inst, const int2* blocks, int nblocks, const MultiKeys& keys, int max_nr,
                         int ninst, cudaStream_t st) {
  const int nrp = (max_nr + 7) / 8 * 8;
  const size_t smem = sizeof(float) * ((size_t)max_nr * nrp +
                                       (size_t)std::max(max_nr * kFCols, kFCols * out_stride(nrp)) + 4 * max_nr +
                                       4 * kFCols);
  FNL_CUDA(cudaFuncSetAttribute(k_filter_multi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_filter_multi<<<nblocks, kThreads, smem, st>>>(inst, blocks, keys);
  FNL_CUDA(cudaGetLastError());
  k_psum_multi<<<dim3(max_nr, ninst), 256, 0, st>>>(inst);
  FNL_CUDA(cudaGetLastError());
}

void launch_combine_multi(const CombineInst* inst, int64_t max_nalm, int ninst, const MultiOut& out, cudaStream_t st) {
  k_combine_multi<<<dim3((unsigned)((max_nalm + 255) / 256), ninst), 256, 0, st>>>(inst, out);
  FNL_CUDA(cudaGetLastError());
}

void build_lambda_tables_mixed(fnl_shells* sh, cudaStream_t st) {
  const int L = sh->lmax, np = sh->npairs;
  std::vector<double> fac(L + 1, 0.0);
  for (int m = 1; m <= L; ++m) fac[m] = -std::sqrt((2.0 * m + 1.0) / (2.0 * m));
  std::vector<double2> ab((size_t)sh->nalm);
  for (int m = 0; m <= L; ++m)
    for (int l = m; l <= L; ++l) {
      double a = 0.0, b = 0.0;
      if (l > m) {
        a = std::sqrt((4.0 * l * l - 1.0) / ((double)l * l - (double)m * m));
        b = std::sqrt(((l - 1.0) * (l - 1.0) - (double)m * m) / (4.0 * (l - 1.0) * (l - 1.0) - 1.0));
      }
      ab[alm_idx(l, m, L)] = make_double2(a, b);
    }
  TempDev t_fac(sizeof(double) * (L + 1)), t_mant(sizeof(double) * (size_t)(L + 1) * np),
      t_expo(sizeof(int) * (size_t)(L + 1) * np), t_ab(sizeof(double2) * (size_t)sh->nalm);
  double* d_fac = t_fac.as<double>();
  double* d_mant = t_mant.as<double>();
  int* d_expo = t_expo.as<int>();
  double2* d_ab = t_ab.as<double2>();
  FNL_CUDA(cudaMemcpyAsync(d_fac, fac.data(), sizeof(double) * (L + 1), cudaMemcpyHostToDevice, st));
  FNL_CUDA(cudaMemcpyAsync(d_ab, ab.data(), sizeof(double2) * ab.size(), cudaMemcpyHostToDevice, st));
  launch_lambda_mm(sh->d_x, d_fac, np, L, d_mant, d_expo, st);
  dim3 grid((np + 127) / 128, L + 1);
  k_lambda_mixed<<<grid, 128, 0, st>>>(sh->d_x, d_mant, d_expo, d_ab, sh->d_row32, sh->d_row0, np, sh->npj, L,
                                       sh->nterms, sh->lsyn_stride, sh->lana_stride, (__nv_bfloat16*)sh->d_lsyn,
                                       (__nv_bfloat16*)sh->d_lana);
  FNL_CUDA(cudaGetLastError());
  FNL_CUDA(cudaStreamSynchronize(st));
}

void launch_filter_mixed(const fnl_shells* sh, uint64_t seed, uint64_t real, const double* noise, double* aLT,
                         double* aLE, double* phi_api, double* psum, cudaStream_t st) {
  if (sh->d_Kterm) {  // on the tensor cores: one monopole partial per degree and shell
    launch_filter_tc(sh, seed, real, noise, aLT, aLE, phi_api, psum ? sh->d_psum_part : nullptr, st);
    if (psum) {
      k_psum_reduce<<<sh->nr, 256, 0, st>>>(sh->lmax + 1, sh->nr, sh->d_psum_part, psum);
      FNL_CUDA(cudaGetLastError());
    }
    return;
  }
  const int nr = sh->nr, nrp = (nr + 7) / 8 * 8, ncol = sh->j0 + nr;
  const size_t smem = sizeof(float) * ((size_t)ncol * nrp + (size_t)std::max(ncol * kFCols, kFCols * out_stride(nrp)) +
                                      4 * ncol + 4 * kFCols);
  FNL_CUDA(cudaFuncSetAttribute(k_filter_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_filter_gemm<<<sh->lmax + 1, kThreads, smem, st>>>(sh->lmax, nr, sh->j0, sh->Cpad, sh->nterms, sh->phiT_stride,
                                                     sh->d_Kft, sh->d_vT, sh->d_vE, seed, real, noise,
                                                     sh->d_row32, (__nv_bfloat16*)sh->d_phiT, phi_api, aLT, aLE,
                                                     psum ? sh->d_psum_part : nullptr);
  FNL_CUDA(cudaGetLastError());
  if (psum) {
    k_psum_reduce<<<nr, 256, 0, st>>>((sh->lmax + 1) * (kThreads / 128), nr, sh->d_psum_part, psum);
    FNL_CUDA(cudaGetLastError());
  }
}

void launch_alm_to_terms(const fnl_shells* sh, const double* alm, cudaStream_t st) {
  const int64_t n = sh->nalm * sh->C;
  k_alm_to_terms<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(sh->lmax, sh->nr, sh->Cpad, sh->nalm, sh->nterms,
                                                              sh->phiT_stride, sh->d_row32, alm,
                                                              (__nv_bfloat16*)sh->d_phiT);
  FNL_CUDA(cudaGetLastError());
}

void launch_combine_mixed(const fnl_shells* sh, double fnl, const double* aLT, const double* aLE, double* aNLT,
                          double* aNLE, double* aT, double* aE, const double* psum, cudaStream_t st) {
  k_combine_mixed<<<(unsigned)((sh->nalm + 255) / 256), 256, 0, st>>>(
      sh->nalm, sh->Cpad / 128, sh->nr, fnl, (const double2*)sh->d_part, psum, sh->d_mu, sh->d_qT, sh->d_qE,
      (const double2*)aLT, (const double2*)aLE, (double2*)aNLT, (double2*)aNLE, (double2*)aT, (double2*)aE);
  FNL_CUDA(cudaGetLastError());
}

}  // namespace fnl
