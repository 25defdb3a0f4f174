// Kernels of the mixed-precision forms (FNL_BF16X2, FNL_BF16X3) around the tensor-core
// Legendre GEMMs (step (i) runs on the tensor cores too, in filter_tc.cu):
//   k_psum_reduce     the per-shell sums of |Phi_L,lm|^2 for the Parseval monopole, from the
//                     filter's per-degree partials in a fixed order
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

namespace fnl {

namespace {

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

__device__ __forceinline__ double flushed(double v) { return fabs(v) < 1e-290 ? 0.0 : v; }

// One thread per (jp, m): lambda_lm(x_jp) for l = m..L by the FP64 recurrence, written as BF16
// terms into Lambda_syn[slab(mp, k / 32)][jp][k % 32] and Lambda_ana[row16(mp) + k][jp]; jmin[m]
// becomes the first ring pair (from the pole) where some |lambda_lm| reaches kLambdaSkip.
__global__ void k_lambda_mixed(const double* __restrict__ x, const double* __restrict__ mant,
                               const int* __restrict__ expo, const double2* __restrict__ ab,
                               const int64_t* __restrict__ row32, const int64_t* __restrict__ row16, int npairs,
                               int npj, int L, int nterms, int64_t syn_stride, int64_t ana_stride,
                               __nv_bfloat16* __restrict__ lsyn, __nv_bfloat16* __restrict__ lana,
                               int* __restrict__ jmin) {
  const int jp = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = blockIdx.y;
  if (jp >= npairs) return;
  const double xx = x[jp];
  double y1 = mant[(size_t)m * npairs + jp], y2 = 0.0;
  int e = expo[(size_t)m * npairs + jp];
  const int64_t base = alm_idx(0, m, L);
  double vmax = 0.0;
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
    vmax = fmax(vmax, fabs(v));
    const int d = l - m, p = d & 1, k = d >> 1;
    const int mp = 2 * m + p;
    const int64_t slab = row32[mp] / 32 + k / 32;
    store_terms_d(lsyn + (slab * npairs + jp) * 32 + (k & 31), syn_stride, nterms, v);
    store_terms_d(lana + (row16[mp] + k) * (int64_t)npj + jp, ana_stride, nterms, v);
  }
  if (vmax >= kLambdaSkip) atomicMin(&jmin[m], jp);
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
  TempDev t_jmin(sizeof(int) * (L + 1));
  int* d_jmin = t_jmin.as<int>();
  FNL_CUDA(cudaMemsetAsync(d_jmin, 0x7f, sizeof(int) * (L + 1), st));  // above any ring pair
  dim3 grid((np + 127) / 128, L + 1);
  k_lambda_mixed<<<grid, 128, 0, st>>>(sh->d_x, d_mant, d_expo, d_ab, sh->d_row32, sh->d_row0, np, sh->npj, L,
                                       sh->nterms, sh->lsyn_stride, sh->lana_stride, (__nv_bfloat16*)sh->d_lsyn,
                                       (__nv_bfloat16*)sh->d_lana, d_jmin);
  FNL_CUDA(cudaGetLastError());
  sh->jmin.assign(L + 1, 0);
  FNL_CUDA(cudaMemcpyAsync(sh->jmin.data(), d_jmin, sizeof(int) * (L + 1), cudaMemcpyDeviceToHost, st));
  FNL_CUDA(cudaStreamSynchronize(st));
  for (int& j : sh->jmin) j = std::min(j, np);
}

void launch_filter_mixed(const fnl_shells* sh, uint64_t seed, uint64_t real, const double* noise, double* aLT,
                         double* aLE, double* phi_api, double* psum, cudaStream_t st) {
  // on the tensor cores, two monopole partials per degree and shell
  launch_filter_tc(sh, seed, real, noise, aLT, aLE, phi_api, psum ? sh->d_psum_part : nullptr, st);
  if (psum) {
    k_psum_reduce<<<sh->nr, 256, 0, st>>>(2 * (sh->lmax + 1), sh->nr, sh->d_psum_part, psum);
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
