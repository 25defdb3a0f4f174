// Kernels of the mixed-precision forms (FNL_BF16X2, FNL_BF16X3) around the tensor-core
// Legendre GEMMs:
//   k_filter_mixed    step (i) in FP32: Phi_L = K_l n (Eq. 9) written as BF16 terms, and
//                     a^X_L = v^X_l . n (Eq. 5) with FP32 products summed per block in FP32
//                     and stored as FP64
//   k_lambda_mixed    lambda_lm(x_jp) from the FP64 recurrence, split into BF16 terms in the
//                     two K-contiguous layouts of the synthesis and analysis GEMMs
//   k_alm_to_terms    API coefficients -> BF16 terms of the synthesis operand
//   k_combine_mixed   a^X_NL = sum over column tiles of the GEMM epilogue partials (FP64),
//                     a^X = a^X_L + f_NL a^X_NL (Eq. 3)
#include <cuda_bf16.h>

#include <cmath>
#include <vector>

#include "fnl_internal.cuh"
#include "mixed.cuh"
#include "philox.cuh"

namespace fnl {

namespace {

constexpr int kThreads = 256;

// Noise in FP32 from the same Philox words as the FP64 path: the 53-bit uniforms are
// rounded to FP32 (relative 2^-24), so draws agree with the FP64 path to ~1e-7.
__device__ __forceinline__ float2 box_muller_f32(uint64_t wa, uint64_t wb) {
  const float u1 = __ull2float_rn((wa >> 11) + 1) * 0x1p-53f;
  const float u2 = __ull2float_rn(wb >> 11) * 0x1p-53f;
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

// Step (i) in FP32, MB = 4 orders m per iteration: every thread draws one Philox block
// (two shells of one m), each K_l row read from shared memory feeds MB products, and the
// eight warps form the MB x {T, E} dot products v^X_l . n.
constexpr int kMB = 4;

__global__ void __launch_bounds__(kThreads) k_filter_mixed(int L, int nr, int Cpad, int nterms, int64_t term_stride,
                                                           const float* __restrict__ Kf, const double* __restrict__ vT,
                                                           const double* __restrict__ vE, uint64_t seed, uint64_t real,
                                                           const double* __restrict__ noise,
                                                           const int64_t* __restrict__ row32,
                                                           __nv_bfloat16* __restrict__ phiT,
                                                           double* __restrict__ phi_api,
                                                           double* __restrict__ aLT, double* __restrict__ aLE) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int l = L - blockIdx.x;
  const int C = 2 * nr;
  float2* ns = (float2*)smem;              // [kMB][nr]
  float* vs = (float*)(ns + kMB * nr);     // [2][nr]
  float* Ks = vs + 2 * nr;                 // [nr][nr + 1]
  const int ldk = nr + 1;
  const float* Kl = Kf + (size_t)l * nr * nr;
  for (int e = threadIdx.x; e < nr * nr; e += kThreads) Ks[(e / nr) * ldk + (e % nr)] = Kl[e];
  for (int e = threadIdx.x; e < nr; e += kThreads) {
    vs[e] = (float)vT[(size_t)l * nr + e];
    vs[nr + e] = (float)vE[(size_t)l * nr + e];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t nalm = (int64_t)(L + 1) * (L + 2) / 2;
  const int npair = (nr + 1) / 2;
  for (int m0 = 0; m0 <= l; m0 += kMB) {
    const int nm = min(kMB, l + 1 - m0);
    __syncthreads();
    if (noise) {
      for (int t = threadIdx.x; t < nm * nr; t += kThreads) {
        const int mb = t / nr, j = t % nr, m = m0 + mb;
        const double2 v = ((const double2*)noise)[(size_t)j * nalm + alm_idx(l, m, L)];
        ns[mb * nr + j] = make_float2((float)v.x, m == 0 ? 0.f : (float)v.y);
      }
    } else {
      for (int t = threadIdx.x; t < nm * npair; t += kThreads) {
        const int mb = t / npair, jp = t % npair, m = m0 + mb;
        uint64_t w[4];
        noise_words(seed, real, alm_idx(l, m, L), jp, w);
        ns[mb * nr + 2 * jp] = noise_value_f32(box_muller_f32(w[0], w[1]), m);
        if (2 * jp + 1 < nr) ns[mb * nr + 2 * jp + 1] = noise_value_f32(box_muller_f32(w[2], w[3]), m);
      }
    }
    __syncthreads();
    // a^X_L for the MB orders: warp w -> (order w >> 1, field w & 1)
    if (warp < 2 * kMB) {
      const int mb = warp >> 1, f = warp & 1;
      if (mb < nm) {
        float sr = 0.f, si = 0.f;
        const float* v = vs + f * nr;
        for (int j = lane; j < nr; j += 32) {
          const float2 n = ns[mb * nr + j];
          sr += v[j] * n.x;
          si += v[j] * n.y;
        }
        for (int o = 16; o; o >>= 1) {
          sr += __shfl_xor_sync(0xffffffffu, sr, o);
          si += __shfl_xor_sync(0xffffffffu, si, o);
        }
        if (lane == 0) {
          const int64_t idx = alm_idx(l, m0 + mb, L);
          ((double2*)(f ? aLE : aLT))[idx] = make_double2((double)sr, (double)si);
        }
      }
    }
    // Phi_L,lm(r_i) = sum_{j <= i} K_l[i, j] n_lm(r_j) for the MB orders
    for (int c = threadIdx.x; c < C; c += kThreads) {
      const int i = c >> 1, r = c & 1;
      float acc[kMB] = {0.f, 0.f, 0.f, 0.f};
      const float* Ki = Ks + (size_t)i * ldk;
      for (int j = 0; j <= i; ++j) {
        const float k = Ki[j];
#pragma unroll
        for (int mb = 0; mb < kMB; ++mb) {
          const float2 n = ns[mb * nr + j];
          acc[mb] += k * (r ? n.y : n.x);
        }
      }
#pragma unroll
      for (int mb = 0; mb < kMB; ++mb) {
        if (mb >= nm) break;
        const int m = m0 + mb;
        const int p = (l - m) & 1;
        const int64_t row = row32[2 * m + p] + ((l - m) >> 1);
        store_terms(phiT + row * Cpad + c, term_stride, nterms, acc[mb]);
        if (phi_api) phi_api[((size_t)alm_idx(l, m, L) * nr + i) * 2 + r] = (double)acc[mb];
      }
    }
  }
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

__global__ void k_combine_mixed(int64_t nalm, int nct, double fnl, const float4* __restrict__ part,
                                const double2* __restrict__ aLT, const double2* __restrict__ aLE,
                                double2* __restrict__ aNLT, double2* __restrict__ aNLE, double2* __restrict__ aT,
                                double2* __restrict__ aE) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nalm) return;
  double tr = 0, ti = 0, er = 0, ei = 0;
  for (int c = 0; c < nct; ++c) {
    const float4 v = part[(size_t)c * nalm + i];
    tr += v.x;
    ti += v.y;
    er += v.z;
    ei += v.w;
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

}  // namespace

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
  double *d_fac = nullptr, *d_mant = nullptr;
  int* d_expo = nullptr;
  double2* d_ab = nullptr;
  FNL_CUDA(cudaMalloc(&d_fac, sizeof(double) * (L + 1)));
  FNL_CUDA(cudaMalloc(&d_mant, sizeof(double) * (size_t)(L + 1) * np));
  FNL_CUDA(cudaMalloc(&d_expo, sizeof(int) * (size_t)(L + 1) * np));
  FNL_CUDA(cudaMalloc(&d_ab, sizeof(double2) * (size_t)sh->nalm));
  FNL_CUDA(cudaMemcpyAsync(d_fac, fac.data(), sizeof(double) * (L + 1), cudaMemcpyHostToDevice, st));
  FNL_CUDA(cudaMemcpyAsync(d_ab, ab.data(), sizeof(double2) * ab.size(), cudaMemcpyHostToDevice, st));
  launch_lambda_mm(sh->d_x, d_fac, np, L, d_mant, d_expo, st);
  dim3 grid((np + 127) / 128, L + 1);
  k_lambda_mixed<<<grid, 128, 0, st>>>(sh->d_x, d_mant, d_expo, d_ab, sh->d_row32, sh->d_row0, np, sh->npj, L,
                                       sh->nterms, sh->lsyn_stride, sh->lana_stride, (__nv_bfloat16*)sh->d_lsyn,
                                       (__nv_bfloat16*)sh->d_lana);
  FNL_CUDA(cudaGetLastError());
  FNL_CUDA(cudaStreamSynchronize(st));
  cudaFree(d_fac);
  cudaFree(d_mant);
  cudaFree(d_expo);
  cudaFree(d_ab);
}

void launch_filter_mixed(const fnl_shells* sh, uint64_t seed, uint64_t real, const double* noise, double* aLT,
                         double* aLE, double* phi_api, cudaStream_t st) {
  const int nr = sh->nr;
  const size_t smem = sizeof(float2) * kMB * nr + sizeof(float) * 2 * nr + sizeof(float) * (size_t)nr * (nr + 1);
  FNL_CUDA(cudaFuncSetAttribute(k_filter_mixed, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_filter_mixed<<<sh->lmax + 1, kThreads, smem, st>>>(sh->lmax, nr, sh->Cpad, sh->nterms, sh->phiT_stride,
                                                      (const float*)sh->d_Kf, sh->d_vT, sh->d_vE, seed, real, noise,
                                                      sh->d_row32, (__nv_bfloat16*)sh->d_phiT, phi_api, aLT, aLE);
  FNL_CUDA(cudaGetLastError());
}

void launch_alm_to_terms(const fnl_shells* sh, const double* alm, cudaStream_t st) {
  const int64_t n = sh->nalm * sh->C;
  k_alm_to_terms<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(sh->lmax, sh->nr, sh->Cpad, sh->nalm, sh->nterms,
                                                              sh->phiT_stride, sh->d_row32, alm,
                                                              (__nv_bfloat16*)sh->d_phiT);
  FNL_CUDA(cudaGetLastError());
}

void launch_combine_mixed(const fnl_shells* sh, double fnl, const double* aLT, const double* aLE, double* aNLT,
                          double* aNLE, double* aT, double* aE, cudaStream_t st) {
  k_combine_mixed<<<(unsigned)((sh->nalm + 255) / 256), 256, 0, st>>>(
      sh->nalm, sh->Cpad / 128, fnl, (const float4*)sh->d_part, (const double2*)aLT, (const double2*)aLE,
      (double2*)aNLT, (double2*)aNLE, (double2*)aT, (double2*)aE);
  FNL_CUDA(cudaGetLastError());
}

}  // namespace fnl
