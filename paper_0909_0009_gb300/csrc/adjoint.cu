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
#include <type_traits>

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
// part of m = 0 is zero.  One warp per entry idx = (l, m): the warp finds (l, m) once, reads the
// entry's gT, gE once, and its lanes take the shells i (both parts) of the row.
// The arithmetic runs in R: FP64 for the FP64 form, FP32 for the FP32 and tensor-core forms (whose
// H~ is an FP32 or BF16-term operand).  Their weights come from the object's FP32 copies and the
// entry's g values are converted once per warp: conversions from FP64 run on the FP64 pipe,
// 1/64 of the FP32 rate on this part.
template <typename R>
struct SourceEntry {
  R gt[2], ge[2];  // gT, gE of the entry (zero where not given), times f_NL and the m > 0 half
  // called by a whole warp: lanes 0-3 form one value each, the others receive them by shuffles
  __device__ SourceEntry(const double* gT, const double* gE, int64_t idx, int m, double fnl) {
    const int lane = threadIdx.x & 31;
    R v = (R)0;
    if (lane < 4) {
      const double* g = lane < 2 ? gT : gE;
      if (g) v = (R)((m > 0 ? 0.5 * fnl : fnl) * g[2 * idx + (lane & 1)]);
    }
    gt[0] = __shfl_sync(0xffffffffu, v, 0);
    gt[1] = __shfl_sync(0xffffffffu, v, 1);
    ge[0] = __shfl_sync(0xffffffffu, v, 2);
    ge[1] = __shfl_sync(0xffffffffu, v, 3);
  }
  // (re, im) of H~ for shell i: q^T_l[i] gT + q^E_l[i] gE; the imaginary part of m = 0 is zero
  __device__ __forceinline__ void value(R qt, R qe, int m, R& re, R& im) const {
    re = qt * gt[0] + qe * ge[0];
    im = m == 0 ? (R)0 : qt * gt[1] + qe * ge[1];
  }
};

template <typename T>
__global__ void __launch_bounds__(kThreads) k_adjoint_source(int L, int nr, int64_t nalm,
                                                             const int64_t* __restrict__ row0,
                                                             const T* __restrict__ qT,
                                                             const T* __restrict__ qE, double fnl,
                                                             const double* __restrict__ gT,
                                                             const double* __restrict__ gE, T* __restrict__ phi) {
  const int64_t idx = (int64_t)blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
  if (idx >= nalm) return;
  int l, m;
  lm_of_entry(idx, L, l, m);
  const SourceEntry<T> e(gT, gE, idx, m, fnl);
  T* row = phi + (row0[2 * m + ((l - m) & 1)] + ((l - m) >> 1)) * (int64_t)(2 * nr);
  for (int i = threadIdx.x & 31; i < nr; i += 32) {
    T re, im;
    e.value(qT[(size_t)l * nr + i], qE[(size_t)l * nr + i], m, re, im);
    row[2 * i] = re;
    row[2 * i + 1] = im;
  }
}

// The same for the tensor-core forms: H~ written as BF16 terms of the synthesis operand (the
// Phi rows in their 32-row packing, Cpad columns), so that the tensor-core synthesis GEMM gives
// s; each lane writes the (re, im) pair of its shells as paired BF16 terms.
__global__ void __launch_bounds__(kThreads) k_adjoint_source_terms(int L, int nr, int Cpad, int64_t nalm, int nterms,
                                                                   int64_t term_stride,
                                                                   const int64_t* __restrict__ row32,
                                                                   const float* __restrict__ qT,
                                                                   const float* __restrict__ qE, double fnl,
                                                                   const double* __restrict__ gT,
                                                                   const double* __restrict__ gE,
                                                                   __nv_bfloat16* __restrict__ phiT) {
  const int64_t idx = (int64_t)blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
  if (idx >= nalm) return;
  int l, m;
  lm_of_entry(idx, L, l, m);
  const SourceEntry<float> e(gT, gE, idx, m, fnl);
  __nv_bfloat16* row = phiT + (row32[2 * m + ((l - m) & 1)] + ((l - m) >> 1)) * Cpad;
  for (int i = threadIdx.x & 31; i < nr; i += 32) {
    float re, im;
    e.value(qT[(size_t)l * nr + i], qE[(size_t)l * nr + i], m, re, im);
    // term t of each value: bf16 of the value less the earlier terms (exact FP32 differences)
    const __nv_bfloat162 h0 = __floats2bfloat162_rn(re, im);
    const float r1 = re - __low2float(h0), i1 = im - __high2float(h0);
    const __nv_bfloat162 h1 = __floats2bfloat162_rn(r1, i1);
    __nv_bfloat162* o = (__nv_bfloat162*)(row + 2 * i);
    o[0] = h0;
    o[term_stride / 2] = h1;
    if (nterms > 2) o[term_stride] = __floats2bfloat162_rn(r1 - __low2float(h1), i1 - __high2float(h1));
  }
}

// dL/dn for degree l = L - blockIdx.x and the orders m = kAfM blockIdx.y .. (<= l):
// Phibar = c_m phi_rows + q^T_l gT + q^E_l gE is staged as a [nr][2 kAfM] tile (columns
// (m, part)), then nbar_j = sum_{i >= j} K_l[i, j] Phibar_i for the whole tile.  K_l is staged
// with zeros above the diagonal, so each output is a plain sum over i; a thread holds a register
// tile of rows j = rg + 32 r (r < 4) and 8 columns, and runs i from its first row rg.  With
// API_ROWS the analysis of 2 f s comes in the API layout [nalm][nr][2] in FP32 (the tensor-core
// forms' per-shell analysis output: their accumulators' type), else in the SIMT rows [rows][2 nr]
// of the real type.
constexpr int kAfM = 32;                // orders per tile
constexpr int kAfCols = 2 * kAfM;       // columns (m, part) per tile
constexpr int kAfMaxRows = 4;           // rows j per thread: nr <= 128
template <typename T>
constexpr int af_ldp() { return kAfCols + 16 / (int)sizeof(T); }  // row stride of the tile (16-byte aligned)

// ROWS = ceil(nr / 32) rows per thread; the tile's arithmetic runs in T.  VEC: grad is 16-byte
// aligned and each (re, im) pair goes out as one 16-byte store.
template <typename T, int ROWS, bool API_ROWS, bool VEC>
__global__ void __launch_bounds__(kThreads) k_adjoint_filter(int L, int nr, int64_t nalm, const T* __restrict__ Kf,
                                                             const int64_t* __restrict__ row0,
                                                             const T* __restrict__ phi,
                                                             const float* __restrict__ api_rows,
                                                             const T* __restrict__ qT,
                                                             const T* __restrict__ qE,
                                                             const double* __restrict__ gT,
                                                             const double* __restrict__ gE,
                                                             double* __restrict__ grad) {
  const int l = L - blockIdx.x, m0 = kAfM * blockIdx.y;
  if (m0 > l) return;
  const int nm = min(kAfM, l + 1 - m0);  // orders of this tile
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int ldp = af_ldp<T>();
  const int C = 2 * nr, ldk = nr + 1;
  T* P = (T*)smem;                        // [nr][ldp] Phibar of the tile
  T* Ks = P + (size_t)nr * ldp;           // [nr][nr + 1] K_l, zero above the diagonal
  const T* Kl = Kf + (size_t)l * nr * nr;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = warp; i < nr; i += kThreads / 32)  // a warp per row of K_l
    for (int j = lane; j < nr; j += 32) Ks[i * ldk + j] = j <= i ? Kl[(size_t)i * nr + j] : (T)0;
  for (int ml = warp; ml < kAfM; ml += kThreads / 32) {  // a warp per order of the tile
    const int m = m0 + ml;
    int64_t idx = 0, row = 0;
    T gv = (T)0;  // the entry's gT re, gT im, gE re, gE im on lanes 0-3, converted once
    if (ml < nm) {
      idx = alm_idx(l, m, L);
      row = row0[2 * m + ((l - m) & 1)] + ((l - m) >> 1);
      if (lane < 4) {
        const double* g = lane < 2 ? gT : gE;
        if (g) gv = (T)g[2 * idx + (lane & 1)];
      }
    }
    const T gt0 = __shfl_sync(0xffffffffu, gv, 0), gt1 = __shfl_sync(0xffffffffu, gv, 1);
    const T ge0 = __shfl_sync(0xffffffffu, gv, 2), ge1 = __shfl_sync(0xffffffffu, gv, 3);
    for (int c = lane; c < C; c += 32) {
      const int i = c >> 1, part = c & 1;
      T v = (T)0;
      if (ml < nm) {
        T x = (m ? (T)2 : (T)1) * (API_ROWS ? (T)api_rows[(size_t)idx * C + c] : phi[row * C + c]);
        x += qT[(size_t)l * nr + i] * (part ? gt1 : gt0) + qE[(size_t)l * nr + i] * (part ? ge1 : ge0);
        v = x;
      }
      P[(size_t)i * ldp + 2 * ml + part] = v;
    }
  }
  __syncthreads();
  const int cg = threadIdx.x & 7, rg = threadIdx.x >> 3;  // 8 column groups x 32 row groups
  T acc[ROWS][8];
#pragma unroll
  for (int r = 0; r < ROWS; ++r)
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[r][q] = (T)0;
  for (int i = rg; i < nr; ++i) {
    T kv[ROWS];
#pragma unroll
    for (int r = 0; r < ROWS; ++r) kv[r] = rg + 32 * r < nr ? Ks[i * ldk + rg + 32 * r] : (T)0;
    T pv[8];
    {
      // 8 consecutive values of a 16-byte aligned row: two float4 or four double2 loads
      const T* src = P + (size_t)i * ldp + 8 * cg;
      if constexpr (sizeof(T) == 4) {
        const float4 u0 = ((const float4*)src)[0], u1 = ((const float4*)src)[1];
        pv[0] = u0.x, pv[1] = u0.y, pv[2] = u0.z, pv[3] = u0.w, pv[4] = u1.x, pv[5] = u1.y, pv[6] = u1.z, pv[7] = u1.w;
      } else {
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          const double2 u = ((const double2*)src)[h];
          pv[2 * h] = u.x, pv[2 * h + 1] = u.y;
        }
      }
    }
#pragma unroll
    for (int r = 0; r < ROWS; ++r)
#pragma unroll
      for (int q = 0; q < 8; ++q) acc[r][q] += kv[r] * pv[q];
  }
#pragma unroll
  for (int r = 0; r < ROWS; ++r) {
    const int j = rg + 32 * r;
    if (j >= nr) continue;
#pragma unroll
    for (int q = 0; q < 8; q += 2) {
      const int ml = (8 * cg + q) >> 1;
      if (ml >= nm) continue;
      const int m = m0 + ml;
      const int64_t idx = alm_idx(l, m, L);
      double* o = grad + ((size_t)j * nalm + idx) * 2;
      const double re = (double)acc[r][q], im = m == 0 ? 0.0 : (double)acc[r][q + 1];
      if (VEC) {
        *(double2*)o = make_double2(re, im);
      } else {
        o[0] = re;
        o[1] = im;
      }
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

unsigned warp_blocks(int64_t nalm) { return (unsigned)((nalm + kThreads / 32 - 1) / (kThreads / 32)); }

template <typename T>
void adjoint_source_impl(const fnl_shells* sh, double fnl, const double* gT, const double* gE, cudaStream_t st) {
  const T* qT = std::is_same<T, float>::value ? (const T*)sh->d_qT32 : (const T*)sh->d_qT;
  const T* qE = std::is_same<T, float>::value ? (const T*)sh->d_qE32 : (const T*)sh->d_qE;
  k_adjoint_source<T><<<warp_blocks(sh->nalm), kThreads, 0, st>>>(sh->lmax, sh->nr, sh->nalm, sh->d_row0, qT, qE, fnl,
                                                                   gT, gE, (T*)sh->d_phi);
  FNL_CUDA(cudaGetLastError());
}

template <typename T, int ROWS>
void adjoint_filter_rows(const fnl_shells* sh, const double* gT, const double* gE, double* grad, cudaStream_t st) {
  const int nr = sh->nr;
  const size_t smem = sizeof(T) * ((size_t)nr * af_ldp<T>() + (size_t)nr * (nr + 1));
  const dim3 grid(sh->lmax + 1, (sh->lmax + kAfM) / kAfM);  // (degree, order tile); tiles past l exit
  const T* qT = std::is_same<T, float>::value ? (const T*)sh->d_qT32 : (const T*)sh->d_qT;
  const T* qE = std::is_same<T, float>::value ? (const T*)sh->d_qE32 : (const T*)sh->d_qE;
  auto run = [&](auto kern, const T* phi, const float* api) {
    FNL_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<grid, kThreads, smem, st>>>(sh->lmax, nr, sh->nalm, (const T*)sh->d_Kf, sh->d_row0, phi, api, qT, qE, gT,
                                       gE, grad);
  };
  const bool vec = ((uintptr_t)grad & 15) == 0;
  if (sh->nterms) {
    if (vec) run(k_adjoint_filter<T, ROWS, true, true>, nullptr, sh->d_adjA);
    else run(k_adjoint_filter<T, ROWS, true, false>, nullptr, sh->d_adjA);
  } else {
    if (vec) run(k_adjoint_filter<T, ROWS, false, true>, (const T*)sh->d_phi, nullptr);
    else run(k_adjoint_filter<T, ROWS, false, false>, (const T*)sh->d_phi, nullptr);
  }
  FNL_CUDA(cudaGetLastError());
}

template <typename T>
void adjoint_filter_impl(const fnl_shells* sh, const double* gT, const double* gE, double* grad, cudaStream_t st) {
  switch ((sh->nr + 31) / 32) {
    case 1: adjoint_filter_rows<T, 1>(sh, gT, gE, grad, st); break;
    case 2: adjoint_filter_rows<T, 2>(sh, gT, gE, grad, st); break;
    case 3: adjoint_filter_rows<T, 3>(sh, gT, gE, grad, st); break;
    case kAfMaxRows: adjoint_filter_rows<T, kAfMaxRows>(sh, gT, gE, grad, st); break;
    default: throw Error(FNL_EUNSUPPORTED, "the adjoint filter takes at most 128 shells");
  }
}

}  // namespace

void launch_adjoint_source(const fnl_shells* sh, double fnl, const double* gT, const double* gE, cudaStream_t st) {
  if (sh->nterms) {
    k_adjoint_source_terms<<<warp_blocks(sh->nalm), kThreads, 0, st>>>(
        sh->lmax, sh->nr, sh->Cpad, sh->nalm, sh->nterms, sh->phiT_stride, sh->d_row32, sh->d_qT32, sh->d_qE32, fnl,
        gT, gE, (__nv_bfloat16*)sh->d_phiT);
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
