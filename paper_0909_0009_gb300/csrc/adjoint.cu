// Adjoint of the generator (differentiation form): the SIMT forms (FP64, FP32) and the
// tensor-core forms (BF16X2, BF16X3), which run the same chain with their own kernels for the
// two syntheses (tcgen05 GEMMs), the ring product and the analysis (tcgen05, per-shell output).
//
// For a real loss L of a^T and a^E with gX = dL/da^X (pairs dL/dRe, dL/dIm) the chain rule
// through steps (i)-(v) gives
//   dL/df_NL   = sum_X <gX, a^X_NL>
//   H          = f_NL sum_X q^X_l gX                          dL/dPhi_NL (Eq. 5 transposed)
//   dL/dg      = W analysis-transpose: W_j sum_lm lambda Re(H e^{i m phi}), every m once
//   dL/df      = 2 f dL/dg                                     (Eq. 2; mu is a constant)
//   dL/dPhi_L  = c_m analysis(2 f s) + sum_X q^X_l gX,  s = synthesis(H~)
// where H~ halves the m > 0 entries of H (synthesis doubles them), c_0 = 1, c_m = 2, and the
// GL weights W cancel between the analysis transpose and the synthesis transpose.  Finally
// dL/dn_lm(r_j) = sum_{i >= j} K_l[i, j] dL/dPhi_L,lm(r_i) (Eq. 9 transposed).  The maps
// f = synthesis(Phi_L) and s are recomputed on the ring grid, never stored.
#include <algorithm>

#include "fnl_internal.cuh"
#include "mixed.cuh"

namespace fnl {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ void lm_of_entry(int64_t idx, int L, int& l, int& m) {
  // entry (m, m) sits at m (2L + 3 - m) / 2; a float estimate of m, corrected exactly
  const float b = 2.0f * L + 3.0f;
  int mm = (int)floorf((b - sqrtf(fmaxf(b * b - 8.0f * (float)idx, 0.0f))) * 0.5f);
  mm = min(max(mm, 0), L);
  while (mm > 0 && alm_idx(mm, mm, L) > idx) --mm;
  while (mm < L && alm_idx(mm + 1, mm + 1, L) <= idx) ++mm;
  m = mm;
  l = (int)(idx - alm_idx(0, mm, L));
}

// H~ in the internal rows: f_NL (q^T_l[i] gT + q^E_l[i] gE), halved for m > 0; the imaginary
// part of m = 0 is zero.  One thread per (idx, column c = 2 i + part).
template <typename T>
__global__ void k_adjoint_source(int L, int nr, int64_t nalm, const int64_t* __restrict__ row0,
                                 const double* __restrict__ qT, const double* __restrict__ qE, double fnl,
                                 const double* __restrict__ gT, const double* __restrict__ gE, T* __restrict__ phi) {
  const int C = 2 * nr;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nalm * C) return;
  const int64_t idx = t / C;
  const int c = (int)(t % C);
  const int i = c >> 1, part = c & 1;
  int l, m;
  lm_of_entry(idx, L, l, m);
  double v = 0.0;
  if (gT) v += qT[(size_t)l * nr + i] * gT[2 * idx + part];
  if (gE) v += qE[(size_t)l * nr + i] * gE[2 * idx + part];
  v *= fnl;
  if (m > 0) v *= 0.5;
  if (m == 0 && part) v = 0.0;
  phi[(row0[2 * m + ((l - m) & 1)] + ((l - m) >> 1)) * C + c] = (T)v;
}

// The same for the tensor-core forms: H~ written as BF16 terms of the synthesis operand (the
// Phi rows in their 32-row packing, Cpad columns), so that the tensor-core synthesis GEMM gives s.
__global__ void k_adjoint_source_terms(int L, int nr, int Cpad, int64_t nalm, int nterms, int64_t term_stride,
                                       const int64_t* __restrict__ row32, const double* __restrict__ qT,
                                       const double* __restrict__ qE, double fnl, const double* __restrict__ gT,
                                       const double* __restrict__ gE, __nv_bfloat16* __restrict__ phiT) {
  const int C = 2 * nr;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nalm * C) return;
  const int64_t idx = t / C;
  const int c = (int)(t % C);
  const int i = c >> 1, part = c & 1;
  int l, m;
  lm_of_entry(idx, L, l, m);
  double v = 0.0;
  if (gT) v += qT[(size_t)l * nr + i] * gT[2 * idx + part];
  if (gE) v += qE[(size_t)l * nr + i] * gE[2 * idx + part];
  v *= fnl;
  if (m > 0) v *= 0.5;
  if (m == 0 && part) v = 0.0;
  store_terms_d(phiT + (row32[2 * m + ((l - m) & 1)] + ((l - m) >> 1)) * Cpad + c, term_stride, nterms, v);
}

// dL/dn for degree l = L - blockIdx.x: Phibar = c_m phi_rows + q^T_l gT + q^E_l gE, then
// nbar_j = sum_{i >= j} K_l[i, j] Phibar_i for every m <= l.  With API_ROWS the analysis of
// 2 f s comes in the API layout [nalm][nr][2] in FP64 (the tensor-core forms' per-shell
// analysis output), else in the SIMT rows [rows][2 nr] of the real type.
template <typename T, bool API_ROWS = false>
__global__ void __launch_bounds__(kThreads) k_adjoint_filter(int L, int nr, int64_t nalm, const T* __restrict__ Kf,
                                                             const int64_t* __restrict__ row0,
                                                             const T* __restrict__ phi,
                                                             const double* __restrict__ api_rows,
                                                             const double* __restrict__ qT,
                                                             const double* __restrict__ qE,
                                                             const double* __restrict__ gT,
                                                             const double* __restrict__ gE,
                                                             double* __restrict__ grad) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int l = L - blockIdx.x;
  const int C = 2 * nr, ldk = nr + 1;
  T* pb = (T*)smem;                   // [C] Phibar of the current (l, m)
  T* Ks = pb + C;                     // [nr][nr + 1]
  const T* Kl = Kf + (size_t)l * nr * nr;
  for (int e = threadIdx.x; e < nr * nr; e += blockDim.x) Ks[(e / nr) * ldk + (e % nr)] = Kl[e];
  for (int m = 0; m <= l; ++m) {
    const int64_t idx = alm_idx(l, m, L);
    const int64_t row = row0[2 * m + ((l - m) & 1)] + ((l - m) >> 1);
    const double cm = m ? 2.0 : 1.0;
    __syncthreads();  // K staged; the previous m's Phibar consumed
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
      const int i = c >> 1, part = c & 1;
      double v = cm * (API_ROWS ? api_rows[(size_t)idx * C + c] : (double)phi[row * C + c]);
      if (gT) v += qT[(size_t)l * nr + i] * gT[2 * idx + part];
      if (gE) v += qE[(size_t)l * nr + i] * gE[2 * idx + part];
      pb[c] = (T)v;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
      const int j = c >> 1, part = c & 1;
      T acc = 0;
      for (int i = j; i < nr; ++i) acc += Ks[(size_t)i * ldk + j] * pb[2 * i + part];
      grad[((size_t)j * nalm + idx) * 2 + part] = (m == 0 && part) ? 0.0 : (double)acc;
    }
  }
}

// dL/df_NL = sum_X sum_idx (gX re aNLX re + gX im aNLX im): per-block partial sums, then
// one block adds them in a fixed order (the result does not depend on scheduling).
__global__ void __launch_bounds__(kThreads) k_dot_partial(int64_t n2, const double* __restrict__ gT,
                                                          const double* __restrict__ aT,
                                                          const double* __restrict__ gE,
                                                          const double* __restrict__ aE,
                                                          double* __restrict__ part) {
  __shared__ double red[kThreads / 32];
  double s = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n2; e += (int64_t)gridDim.x * blockDim.x) {
    if (gT) s += gT[e] * aT[e];
    if (gE) s += gE[e] * aE[e];
  }
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) t += red[w];
    part[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(kThreads) k_dot_final(int nparts, const double* __restrict__ part,
                                                        double* __restrict__ out) {
  __shared__ double red[kThreads];
  double s = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) s += part[i];
  red[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < kThreads; ++i) t += red[i];
    *out = t;
  }
}

template <typename T>
void adjoint_source_impl(const fnl_shells* sh, double fnl, const double* gT, const double* gE, cudaStream_t st) {
  const int64_t n = sh->nalm * sh->C;
  k_adjoint_source<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(sh->lmax, sh->nr, sh->nalm, sh->d_row0,
                                                                    sh->d_qT, sh->d_qE, fnl, gT, gE, (T*)sh->d_phi);
  FNL_CUDA(cudaGetLastError());
}

template <typename T>
void adjoint_filter_impl(const fnl_shells* sh, const double* gT, const double* gE, double* grad, cudaStream_t st) {
  const int nr = sh->nr;
  const size_t smem = sizeof(T) * ((size_t)2 * nr + (size_t)nr * (nr + 1));
  FNL_CUDA(cudaFuncSetAttribute(k_adjoint_filter<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  if (sh->nterms) {
    FNL_CUDA(cudaFuncSetAttribute(k_adjoint_filter<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_adjoint_filter<T, true><<<sh->lmax + 1, kThreads, smem, st>>>(sh->lmax, nr, sh->nalm, (const T*)sh->d_Kf,
                                                                    sh->d_row0, nullptr, sh->d_adjA, sh->d_qT,
                                                                    sh->d_qE, gT, gE, grad);
  } else {
    k_adjoint_filter<T><<<sh->lmax + 1, kThreads, smem, st>>>(sh->lmax, nr, sh->nalm, (const T*)sh->d_Kf, sh->d_row0,
                                                              (const T*)sh->d_phi, nullptr, sh->d_qT, sh->d_qE, gT,
                                                              gE, grad);
  }
  FNL_CUDA(cudaGetLastError());
}

}  // namespace

void launch_adjoint_source(const fnl_shells* sh, double fnl, const double* gT, const double* gE, cudaStream_t st) {
  if (sh->nterms) {
    const int64_t n = sh->nalm * sh->C;
    k_adjoint_source_terms<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
        sh->lmax, sh->nr, sh->Cpad, sh->nalm, sh->nterms, sh->phiT_stride, sh->d_row32, sh->d_qT, sh->d_qE, fnl, gT,
        gE, (__nv_bfloat16*)sh->d_phiT);
    FNL_CUDA(cudaGetLastError());
  } else if (sh->real_is_double) {
    adjoint_source_impl<double>(sh, fnl, gT, gE, st);
  } else {
    adjoint_source_impl<float>(sh, fnl, gT, gE, st);
  }
}

void launch_adjoint_filter(const fnl_shells* sh, const double* gT, const double* gE, double* grad_noise,
                           cudaStream_t st) {
  if (sh->real_is_double) adjoint_filter_impl<double>(sh, gT, gE, grad_noise, st);
  else adjoint_filter_impl<float>(sh, gT, gE, grad_noise, st);
}

void launch_dot_fnl(const fnl_shells* sh, const double* gT, const double* gE, const double* aNLT,
                    const double* aNLE, double* out, cudaStream_t st) {
  // partial sums go to the object's a^X scratch (4 nalm doubles >= blocks)
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(2 * std::max(sh->sms, 1), 1024), 4 * sh->nalm));
  k_dot_partial<<<blocks, kThreads, 0, st>>>(2 * sh->nalm, gT, aNLT, gE, aNLE, sh->d_aOut);
  FNL_CUDA(cudaGetLastError());
  k_dot_final<<<1, kThreads, 0, st>>>(blocks, sh->d_aOut, out);
  FNL_CUDA(cudaGetLastError());
}

}  // namespace fnl
