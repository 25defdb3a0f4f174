// The fast cubic f_NL estimator of Sect. 5 on the shells of a generator configuration:
//
//   A(r, n) = sum_{i,j} sum_lm (C^-1)^{ij}_l alpha^i_l(r) a^j_lm Y_lm(n),   B likewise with beta
//   S_prim  = int dr r^2 int d^2n A B^2,   f_NL = S_prim / N
//   N = sum_{l1<=l2<=l3} (1/Delta) sum B^{ijk} (C^-1)^{io}_l1 (C^-1)^{jp}_l2 (C^-1)^{kq}_l3 B^{opq},
//   B^{ijk} = 2 I_{l1l2l3} int dr r^2 [beta^i_l1 beta^j_l2 alpha^k_l3 + beta^k_l3 beta^i_l1 alpha^j_l2
//             + beta^j_l2 beta^k_l3 alpha^i_l1],  I = sqrt((2l1+1)(2l2+1)(2l3+1)/(4 pi)) (l1 l2 l3; 0 0 0)
//
// with, on the generator's shells: int dr r^2 -> sum_i w_i r_i^2; beta^X_l(r_i) = (K_l K_l^T q^X_l)_i
// (the covariance of Phi_L(r_i) with a^X_L, which the paper's beta is in the continuum);
// C^XY_l = v^X_l . v^Y_l with v^X = K_l^T q^X_l; C^-1 the Moore-Penrose inverse (full inverse when
// the smaller eigenvalue exceeds 1e-10 of the larger, else the leading eigenpair's v v^T / lambda);
// degrees l < 2 left out.
//
// Per call: a power-of-two scale for A and B from the largest |a_lm| (one block; the maps then
// stay O(1) in every precision form and the scale comes off S exactly), the coefficients of A
// and B on every shell (one kernel, into the Phi rows of an
// internal synthesis object with 2 N_r fields), the Legendre synthesis GEMM of that object
// (tensor-core or SIMT form, unchanged), a ring kernel that takes A and B of each (shell, ring
// pair) to the two rings and sums A B^2 (FP64 sums), and one block that adds the rings and
// shells with their weights in a fixed order.  The normalisation is summed at set-up as the
// paper writes it, in FP64 (every term is a non-negative quadratic form, so the sum is exact
// to rounding whatever the conditioning of C_l).
#include <algorithm>
#include <cmath>
#include <vector>

#include "fnl_internal.cuh"
#include "mixed.cuh"

struct fnl_ksw {
  const fnl_shells* sh = nullptr;  // configuration (not owned)
  fnl_shells* syn = nullptr;       // synthesis object of the 2 nr fields A, B (owned)
  int lmax = 0, nr = 0, npairs = 0, nphi = 0, device = 0;
  double norm = 0.0;
  double norm_seconds = 0.0;
  std::vector<int> rank;           // [L+1] rank of C_l used (0 for l < 2)
  double* d_f = nullptr;           // [2 (A, B)][2 (a^T, a^E)][L+1][nr] filter weights
  double* d_u = nullptr;           // [nr] w_i r_i^2
  double* d_part = nullptr;        // [nr][npairs] ring sums
  unsigned long long* d_amax = nullptr;  // max |a_lm| of the current call (bits of a double)
  float* d_f32 = nullptr;          // d_f in FP32 (FP32 and mixed objects)
  double fmax[2] = {0.0, 0.0};     // largest |weight| of the A and B filters
  std::vector<void*> allocations;
};

namespace fnl {

namespace {

constexpr double kRankRcond = 1e-10;
constexpr int kLmin = 2;

template <typename T>
T* kalloc(fnl_ksw* k, size_t n) {
  void* p = nullptr;
  FNL_CUDA(cudaMalloc(&p, sizeof(T) * (n ? n : 1)));
  k->allocations.push_back(p);
  return (T*)p;
}

// (l, m) of triangle entry idx.
__device__ __forceinline__ void lm_of_idx(int64_t idx, int L, int& l, int& m) {
  const float b = 2.0f * L + 3.0f;
  int mm = (int)floorf((b - sqrtf(fmaxf(b * b - 8.0f * (float)idx, 0.0f))) * 0.5f);
  mm = max(0, min(mm, L));
  while (mm > 0 && alm_idx(mm, mm, L) > idx) --mm;
  while (mm < L && alm_idx(mm + 1, mm + 1, L) <= idx) ++mm;
  m = mm;
  l = (int)(idx - alm_idx(0, mm, L));
}

// Coefficients of A (fields 0..nr-1) and B (fields nr..2nr-1) for every (l, m) and shell:
// value = f[field][T][l][s] a^T_lm + f[field][E][l][s] a^E_lm (imaginary part of m = 0 dropped),
// written as BF16 terms of the synthesis operand (nterms > 0) or in the SIMT real type.  A
// block takes one row (l, m) at a time: its 4 nr columns (field, shell, re / im) are
// consecutive threads.
// Per-call scaling of the fields: A and B are synthesised as 2^-ea A and 2^-eb B, with
// 2^ea ~ max|a_lm| max|weight of A| (likewise eb), so that the maps and the products A B^2 stay
// far inside the FP32 range whatever the units of a_lm; S_prim is homogeneous (degree 1 in A,
// 2 in B), so the reduction multiplies by 2^(ea + 2 eb), exactly.  max|a_lm| is gathered as the
// bit pattern of a non-negative double (ordered like the double) with atomicMax: the result
// does not depend on the order of the blocks.
__device__ __forceinline__ void field_exponents(unsigned long long amax_bits, double fmaxA, double fmaxB, int& ea,
                                                int& eb) {
  const double amax = __longlong_as_double((long long)amax_bits);
  ea = eb = 0;
  if (amax > 0.0 && fmaxA > 0.0) frexp(amax * fmaxA, &ea);
  if (amax > 0.0 && fmaxB > 0.0) frexp(amax * fmaxB, &eb);
}

__global__ void __launch_bounds__(256) k_ksw_amax(int64_t nalm, const double2* __restrict__ aT,
                                                  const double2* __restrict__ aE,
                                                  unsigned long long* __restrict__ amax_bits) {
  __shared__ double red[8];
  double m = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nalm; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 t = aT[i], e = aE[i];
    m = fmax(m, fmax(fmax(fabs(t.x), fabs(t.y)), fmax(fabs(e.x), fabs(e.y))));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
    atomicMax(amax_bits, (unsigned long long)__double_as_longlong(m));
  }
}

// Coefficients of A (fields 0..nr-1) and B (fields nr..2nr-1) for every (l, m) and shell:
// value = 2^-e(field) (f[field][T][l][s] a^T_lm + f[field][E][l][s] a^E_lm) (imaginary part of
// m = 0 dropped), computed in the object's real type R (FP32 for FP32 and mixed objects, whose
// synthesis takes FP32 values) and written as BF16 terms of the synthesis operand
// (nterms > 0) or in the SIMT layout.  A block takes one row (l, m) at a time: its 4 nr columns
// (field, shell, re / im) are consecutive threads.
template <typename R>
__global__ void __launch_bounds__(256) k_ksw_coeffs(int L, int nr, int64_t nalm, const R* __restrict__ f,
                                                    const double2* __restrict__ aT, const double2* __restrict__ aE,
                                                    const unsigned long long* __restrict__ amax_bits, double fmaxA,
                                                    double fmaxB, int nterms, int Cpad, int64_t term_stride,
                                                    const int64_t* __restrict__ rows, __nv_bfloat16* __restrict__ phiT,
                                                    R* __restrict__ phi) {
  const int C = 4 * nr;
  const size_t L1 = (size_t)L + 1;
  int ea, eb;
  field_exponents(*amax_bits, fmaxA, fmaxB, ea, eb);
  const R sA = (R)ldexp(1.0, -ea), sB = (R)ldexp(1.0, -eb);
  for (int64_t idx = blockIdx.x; idx < nalm; idx += gridDim.x) {
    int l, m;
    lm_of_idx(idx, L, l, m);
    const double2 at = aT[idx], ae = aE[idx];
    const R atx = (R)at.x, aty = (R)at.y, aex = (R)ae.x, aey = (R)ae.y;
    const int64_t row = rows[2 * m + ((l - m) & 1)] + ((l - m) >> 1);
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
      const int field = c / (2 * nr), s = (c >> 1) - field * nr, part = c & 1;
      const R fT = f[((size_t)(2 * field) * L1 + l) * nr + s];
      const R fE = f[((size_t)(2 * field + 1) * L1 + l) * nr + s];
      R v = (part ? fT * aty + fE * aey : fT * atx + fE * aex) * (field ? sB : sA);
      if (m == 0 && part) v = (R)0;
      if (nterms) store_terms(phiT + row * Cpad + c, term_stride, nterms, (float)v);
      else phi[row * C + c] = v;
    }
  }
}

// BF16 terms of four consecutive values: term 0 = bf16(v), term t = bf16(v - earlier terms).
__device__ __forceinline__ void store_quad_terms(__nv_bfloat16* p, int64_t stride, int nterms, float4 v) {
  const __nv_bfloat162 a0 = __floats2bfloat162_rn(v.x, v.y), b0 = __floats2bfloat162_rn(v.z, v.w);
  const float4 r = make_float4(v.x - __low2float(a0), v.y - __high2float(a0), v.z - __low2float(b0),
                               v.w - __high2float(b0));
  const __nv_bfloat162 a1 = __floats2bfloat162_rn(r.x, r.y), b1 = __floats2bfloat162_rn(r.z, r.w);
  uint2 w0, w1;
  w0.x = *(const uint32_t*)&a0;
  w0.y = *(const uint32_t*)&b0;
  w1.x = *(const uint32_t*)&a1;
  w1.y = *(const uint32_t*)&b1;
  *(uint2*)p = w0;
  *(uint2*)(p + stride) = w1;
  if (nterms > 2) {
    const __nv_bfloat162 a2 = __floats2bfloat162_rn(r.x - __low2float(a1), r.y - __high2float(a1));
    const __nv_bfloat162 b2 = __floats2bfloat162_rn(r.z - __low2float(b1), r.w - __high2float(b1));
    uint2 w2;
    w2.x = *(const uint32_t*)&a2;
    w2.y = *(const uint32_t*)&b2;
    *(uint2*)(p + 2 * stride) = w2;
  }
}

// The coefficients of the tensor-core forms (nr even): one warp per row (l, m), each lane four
// consecutive columns (shells s, s + 1 of one field, re and im) with vector loads of the
// weights and 8-byte stores of each BF16 term; eight rows in flight per block.
__global__ void __launch_bounds__(256) k_ksw_coeffs_tc(int L, int nr, int64_t nalm, const float* __restrict__ f,
                                                       const double2* __restrict__ aT, const double2* __restrict__ aE,
                                                       const unsigned long long* __restrict__ amax_bits, double fmaxA,
                                                       double fmaxB, int nterms, int Cpad, int64_t term_stride,
                                                       const int64_t* __restrict__ rows,
                                                       __nv_bfloat16* __restrict__ phiT) {
  const int C4 = nr;  // column quads: 4 nr columns
  const size_t L1 = (size_t)L + 1;
  int ea, eb;
  field_exponents(*amax_bits, fmaxA, fmaxB, ea, eb);
  const float sA = (float)ldexp(1.0, -ea), sB = (float)ldexp(1.0, -eb);
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t idx = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); idx < nalm; idx += warps) {
    int l, m;
    lm_of_idx(idx, L, l, m);
    const double2 at = aT[idx], ae = aE[idx];
    const float atx = (float)at.x, aty = m ? (float)at.y : 0.f, aex = (float)ae.x, aey = m ? (float)ae.y : 0.f;
    const int64_t row = rows[2 * m + ((l - m) & 1)] + ((l - m) >> 1);
    for (int q = lane; q < C4; q += 32) {
      const int c = 4 * q;
      const int field = c / (2 * nr), s = (c >> 1) - field * nr;
      const float2 fT = *(const float2*)(f + ((size_t)(2 * field) * L1 + l) * nr + s);
      const float2 fE = *(const float2*)(f + ((size_t)(2 * field + 1) * L1 + l) * nr + s);
      const float sc = field ? sB : sA;
      const float4 v = make_float4((fT.x * atx + fE.x * aex) * sc, (fT.x * aty + fE.x * aey) * sc,
                                   (fT.y * atx + fE.y * aex) * sc, (fT.y * aty + fE.y * aey) * sc);
      store_quad_terms(phiT + row * Cpad + c, term_stride, nterms, v);
    }
  }
}

// S = 2^(ea + 2 eb) (2 pi / nphi) sum_s u_s sum_j part[s][j], in a fixed order (one block of
// 1024 threads: thread t adds u_s part[s][j] over the flat indices t, t + 1024, ..., then a tree).
__global__ void __launch_bounds__(1024) k_ksw_reduce(int nr, int npairs, const double* __restrict__ part,
                                                     const double* __restrict__ u, double scale,
                                                     const unsigned long long* __restrict__ amax_bits, double fmaxA,
                                                     double fmaxB, double* __restrict__ S) {
  __shared__ double red[1024];
  double t = 0.0;
  const int n = nr * npairs;
  for (int i = threadIdx.x; i < n; i += blockDim.x) t += u[i / npairs] * part[i];
  red[threadIdx.x] = t;
  __syncthreads();
  for (int o = 512; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    int ea, eb;
    field_exponents(*amax_bits, fmaxA, fmaxB, ea, eb);
    *S = ldexp(red[0] * scale, ea + 2 * eb);
  }
}

// Normalisation: block l2 (2..L); per l1 = 2..l2 the block stages
//   M1^{ij}(r) = u_r beta^i_l1 beta^j_l2,   M23^{ij}(r) = u_r (beta^i_l1 alpha^j_l2 + alpha^i_l1 beta^j_l2)
// and thread t takes l3 = l2 + (l1 & 1) + 2 t (+ 2 blockDim ...) <= min(L, l1 + l2), so that
// l1 + l2 + l3 is even:  b^{ijk}/2 = sum_r M1^{ij} alpha^k_l3 + M23^{ij} beta^k_l3, and adds
// I^2 / Delta * b . (C^-1_l1 x C^-1_l2 x C^-1_l3) b.  tab: [r][alpha T, alpha E, beta T, beta E][l].
__global__ void __launch_bounds__(256) k_ksw_norm(int L, int nr, const double* __restrict__ tab,
                                                  const double* __restrict__ u, const double* __restrict__ cinv,
                                                  const double* __restrict__ lf, double* __restrict__ part) {
  extern __shared__ double sm[];
  __shared__ double red[8];
  double* M1 = sm;
  double* M23 = sm + 4 * nr;
  const int l2 = blockIdx.x + kLmin;
  const size_t L1 = (size_t)L + 1;
  double c2[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) c2[q] = cinv[4 * l2 + q];
  double acc = 0.0;
  for (int l1 = kLmin; l1 <= l2; ++l1) {
    __syncthreads();
    for (int t = threadIdx.x; t < 4 * nr; t += blockDim.x) {
      const int ij = t / nr, r = t - ij * nr, i = ij >> 1, j = ij & 1;
      const double* row = tab + (size_t)r * 4 * L1;
      const double a1 = row[i * L1 + l1], b1 = row[(2 + i) * L1 + l1];
      const double a2 = row[j * L1 + l2], b2 = row[(2 + j) * L1 + l2];
      M1[t] = u[r] * b1 * b2;
      M23[t] = u[r] * (b1 * a2 + a1 * b2);
    }
    __syncthreads();
    double c1[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) c1[q] = cinv[4 * l1 + q];
    const int l3max = min(L, l1 + l2);
    for (int l3 = l2 + (l1 & 1) + 2 * (int)threadIdx.x; l3 <= l3max; l3 += 2 * (int)blockDim.x) {
      double b[8];  // [i][j][k]
#pragma unroll
      for (int q = 0; q < 8; ++q) b[q] = 0.0;
      for (int r = 0; r < nr; ++r) {
        const double* row = tab + (size_t)r * 4 * L1;
        const double aT3 = row[l3], aE3 = row[L1 + l3], bT3 = row[2 * L1 + l3], bE3 = row[3 * L1 + l3];
#pragma unroll
        for (int ij = 0; ij < 4; ++ij) {
          const double m1 = M1[ij * nr + r], m23 = M23[ij * nr + r];
          b[2 * ij] += m1 * aT3 + m23 * bT3;
          b[2 * ij + 1] += m1 * aE3 + m23 * bE3;
        }
      }
      double c3[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) c3[q] = cinv[4 * l3 + q];
      // y = (C1 x C2 x C3) b, one factor at a time (C^-1 symmetric)
      double t1[8], t2[8], y[8];
#pragma unroll
      for (int o = 0; o < 2; ++o)
#pragma unroll
        for (int jk = 0; jk < 4; ++jk) t1[o * 4 + jk] = c1[o * 2 + 0] * b[jk] + c1[o * 2 + 1] * b[4 + jk];
#pragma unroll
      for (int o = 0; o < 2; ++o)
#pragma unroll
        for (int p = 0; p < 2; ++p)
#pragma unroll
          for (int k = 0; k < 2; ++k)
            t2[o * 4 + p * 2 + k] = c2[p * 2 + 0] * t1[o * 4 + k] + c2[p * 2 + 1] * t1[o * 4 + 2 + k];
#pragma unroll
      for (int op = 0; op < 4; ++op)
#pragma unroll
        for (int q = 0; q < 2; ++q) y[op * 2 + q] = c3[q * 2 + 0] * t2[op * 2] + c3[q * 2 + 1] * t2[op * 2 + 1];
      double quad = 0.0;
#pragma unroll
      for (int q = 0; q < 8; ++q) quad += b[q] * y[q];
      const int J = l1 + l2 + l3, g = J / 2;
      const double lw = lf[J - 2 * l1] + lf[J - 2 * l2] + lf[J - 2 * l3] - lf[J + 1] +
                        2.0 * (lf[g] - lf[g - l1] - lf[g - l2] - lf[g - l3]);
      const double I2 = (2.0 * l1 + 1.0) * (2.0 * l2 + 1.0) * (2.0 * l3 + 1.0) / (4.0 * M_PI) * exp(lw);
      const double delta = (l1 == l2 && l2 == l3) ? 6.0 : (l1 == l2 || l2 == l3) ? 2.0 : 1.0;
      acc += 4.0 * I2 / delta * quad;
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    part[blockIdx.x] = t;
  }
}

// Moore-Penrose inverse of the symmetric 2 x 2 matrix [[a, b], [b, d]] (positive semidefinite):
// the inverse when the smaller eigenvalue exceeds kRankRcond of the larger, else v v^T / lambda1.
int pinv2(double a, double b, double d, double out[4]) {
  out[0] = out[1] = out[2] = out[3] = 0.0;
  const double h = 0.5 * (a + d), q = std::sqrt(0.25 * (a - d) * (a - d) + b * b);
  const double lam1 = h + q;
  if (!(lam1 > 0.0)) return 0;
  const double lam2 = (a * d - b * b) / lam1;
  if (lam2 > kRankRcond * lam1) {
    const double det = a * d - b * b;
    out[0] = d / det;
    out[1] = out[2] = -b / det;
    out[3] = a / det;
    return 2;
  }
  // (A - lam1 I) v = 0 from either row: v = (b, lam1 - a) or (lam1 - d, b); take the longer
  double v0 = b, v1 = lam1 - a;
  const double w0 = lam1 - d, w1 = b;
  if (w0 * w0 + w1 * w1 > v0 * v0 + v1 * v1) {
    v0 = w0;
    v1 = w1;
  }
  if (v0 == 0.0 && v1 == 0.0) {
    v0 = a >= d ? 1.0 : 0.0;
    v1 = a >= d ? 0.0 : 1.0;
  }
  const double nv = std::sqrt(v0 * v0 + v1 * v1);
  v0 /= nv;
  v1 /= nv;
  out[0] = v0 * v0 / lam1;
  out[1] = out[2] = v0 * v1 / lam1;
  out[3] = v1 * v1 / lam1;
  return 1;
}

void free_ksw(fnl_ksw* k) {
  if (!k) return;
  for (void* p : k->allocations) cudaFree(p);
  if (k->syn) release_shells(k->syn);
  delete k;
}

}  // namespace

}  // namespace fnl

using namespace fnl;

extern "C" {

fnl_status fnl_ksw_create(const fnl_shells* sh, fnl_ksw** out) {
  fnl_ksw* k = nullptr;
  fnl_status st = guard([&] {
    FNL_REQUIRE(out, "out must not be NULL");
    *out = nullptr;
    check_shells(sh);
    FNL_REQUIRE(!sh->synth_only && !sh->owner && sh->host, "fnl_ksw_create: not on an internal object");
    if (sh->nside) throw Error(FNL_EUNSUPPORTED, "the estimator runs on the Gauss-Legendre grid");
    if (sh->nr != sh->nr_total)
      throw Error(FNL_EUNSUPPORTED, "the estimator needs a whole configuration, not a shell shard");
    // the tensor-core coefficient kernel takes the shells of a field two at a time
    if (sh->nterms && sh->nr % 2)
      throw Error(FNL_EUNSUPPORTED, "the estimator of the tensor-core forms needs an even shell count");
    DeviceScope scope(sh->device);
    const int L = sh->lmax, nr = sh->nr, np = sh->npairs;
    const size_t ts = sh->real_is_double ? 16 : 8;
    FNL_REQUIRE(3 * ts * (size_t)sh->nphi <= 227 * 1024, "nphi too large for the estimator's ring kernel");
    k = new fnl_ksw;
    k->sh = sh;
    k->lmax = L;
    k->nr = nr;
    k->npairs = np;
    k->nphi = sh->nphi;
    k->device = sh->device;
    const HostSetup& h = *sh->host;
    const size_t L1 = (size_t)L + 1;

    // ---- per-degree weights in FP64
    std::vector<double> u(nr), alpha(2 * L1 * nr), beta(2 * L1 * nr), cinv(4 * L1, 0.0);
    for (int i = 0; i < nr; ++i) u[i] = h.w[i] * h.r[i] * h.r[i];
    for (size_t q = 0; q < L1 * nr; ++q) {
      alpha[q] = h.alphaT[q];
      alpha[L1 * nr + q] = h.alphaE[q];
    }
    k->rank.assign(L1, 0);
    for (int l = 0; l <= L; ++l) {
      const double* Kl = h.K.data() + (size_t)l * nr * nr;
      const double* v[2] = {h.vT.data() + (size_t)l * nr, h.vE.data() + (size_t)l * nr};
      for (int x = 0; x < 2; ++x)
        for (int i = 0; i < nr; ++i) {
          double s = 0.0;
          for (int j = 0; j <= i; ++j) s += Kl[(size_t)i * nr + j] * v[x][j];
          beta[((size_t)x * L1 + l) * nr + i] = s;
        }
      if (l < kLmin) continue;
      double C[3] = {0.0, 0.0, 0.0};
      for (int i = 0; i < nr; ++i) {
        C[0] += v[0][i] * v[0][i];
        C[1] += v[0][i] * v[1][i];
        C[2] += v[1][i] * v[1][i];
      }
      k->rank[l] = pinv2(C[0], C[1], C[2], &cinv[4 * l]);
    }
    // f[field][j][l][s] = sum_i X^i_l(r_s) (C^-1)^{ij}_l, X = alpha (A) or beta (B)
    std::vector<double> f(4 * L1 * nr, 0.0);
    for (int field = 0; field < 2; ++field) {
      const std::vector<double>& X = field ? beta : alpha;
      for (int j = 0; j < 2; ++j)
        for (int l = 0; l <= L; ++l)
          for (int s = 0; s < nr; ++s)
            f[((size_t)(2 * field + j) * L1 + l) * nr + s] = X[((size_t)0 * L1 + l) * nr + s] * cinv[4 * l + 0 * 2 + j] +
                                                             X[((size_t)1 * L1 + l) * nr + s] * cinv[4 * l + 1 * 2 + j];
    }
    for (int field = 0; field < 2; ++field)
      for (size_t q = 0; q < 2 * L1 * nr; ++q)
        k->fmax[field] = std::max(k->fmax[field], std::fabs(f[(size_t)field * 2 * L1 * nr + q]));
    k->d_amax = kalloc<unsigned long long>(k, 1);
    k->d_f = kalloc<double>(k, f.size());
    {
      std::vector<float> f32(f.begin(), f.end());
      k->d_f32 = kalloc<float>(k, f32.size());
      FNL_CUDA(cudaMemcpy(k->d_f32, f32.data(), sizeof(float) * f32.size(), cudaMemcpyHostToDevice));
    }
    k->d_u = kalloc<double>(k, nr);
    k->d_part = kalloc<double>(k, (size_t)nr * np);
    FNL_CUDA(cudaMemcpy(k->d_f, f.data(), sizeof(double) * f.size(), cudaMemcpyHostToDevice));
    FNL_CUDA(cudaMemcpy(k->d_u, u.data(), sizeof(double) * nr, cudaMemcpyHostToDevice));
    FNL_CUDA(cudaMemset(k->d_part, 0, sizeof(double) * (size_t)nr * np));

    // ---- synthesis object of the 2 nr fields (same grid, degrees and precision form)
    {
      std::vector<double> r2(2 * nr), w2(2 * nr), zero(L1 * 2 * nr, 0.0), mu0(2 * nr, 0.0);
      for (int i = 0; i < 2 * nr; ++i) {
        r2[i] = h.r[i % nr];
        w2[i] = h.w[i % nr];
      }
      fnl_shell_desc d{};
      d.lmax = L;
      d.nr = 2 * nr;
      d.ntheta = sh->ntheta;
      d.nphi = sh->nphi;
      d.r = r2.data();
      d.w = w2.data();
      d.K = nullptr;
      d.alphaT = zero.data();
      d.alphaE = zero.data();
      d.mu = mu0.data();
      d.prec = sh->prec;
      k->syn = make_shells_core(&d, sh->device, true);
      if (k->syn->nterms) configure_tc(k->syn, sh->nsyn > 0 ? sh->nsyn : 256, 256);
    }

    // ---- normalisation, summed over l1 <= l2 <= l3 in FP64
    if (L >= kLmin) {
      std::vector<double> tab((size_t)nr * 4 * L1), lf(3 * L1 + 2);
      for (int s = 0; s < nr; ++s)
        for (int q = 0; q < 4; ++q)
          for (int l = 0; l <= L; ++l)
            tab[((size_t)s * 4 + q) * L1 + l] = (q < 2 ? alpha : beta)[((size_t)(q & 1) * L1 + l) * nr + s];
      for (size_t n = 0; n < lf.size(); ++n) lf[n] = std::lgamma((double)n + 1.0);
      double *d_tab = nullptr, *d_cinv = nullptr, *d_lf = nullptr, *d_np = nullptr;
      const int nb = L - kLmin + 1;
      auto release = [&] {
        cudaFree(d_tab);
        cudaFree(d_cinv);
        cudaFree(d_lf);
        cudaFree(d_np);
      };
      try {
        FNL_CUDA(cudaMalloc(&d_tab, sizeof(double) * tab.size()));
        FNL_CUDA(cudaMalloc(&d_cinv, sizeof(double) * cinv.size()));
        FNL_CUDA(cudaMalloc(&d_lf, sizeof(double) * lf.size()));
        FNL_CUDA(cudaMalloc(&d_np, sizeof(double) * nb));
        FNL_CUDA(cudaMemcpy(d_tab, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice));
        FNL_CUDA(cudaMemcpy(d_cinv, cinv.data(), sizeof(double) * cinv.size(), cudaMemcpyHostToDevice));
        FNL_CUDA(cudaMemcpy(d_lf, lf.data(), sizeof(double) * lf.size(), cudaMemcpyHostToDevice));
        cudaEvent_t e0, e1;
        FNL_CUDA(cudaEventCreate(&e0));
        FNL_CUDA(cudaEventCreate(&e1));
        const size_t smem = sizeof(double) * 8 * nr;
        FNL_CUDA(cudaEventRecord(e0, 0));
        k_ksw_norm<<<nb, 256, smem>>>(L, nr, d_tab, k->d_u, d_cinv, d_lf, d_np);
        FNL_CUDA(cudaGetLastError());
        FNL_CUDA(cudaEventRecord(e1, 0));
        FNL_CUDA(cudaEventSynchronize(e1));
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        k->norm_seconds = ms / 1e3;
        std::vector<double> part(nb);
        FNL_CUDA(cudaMemcpy(part.data(), d_np, sizeof(double) * nb, cudaMemcpyDeviceToHost));
        double n = 0.0;
        for (int i = 0; i < nb; ++i) n += part[i];
        k->norm = n;
      } catch (...) {
        release();
        throw;
      }
      release();
    }
    FNL_CUDA(cudaDeviceSynchronize());
    *out = k;
  });
  if (st != FNL_OK && k) free_ksw(k);
  return st;
}

void fnl_ksw_destroy(fnl_ksw* k) {
  if (!k) return;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(k->device);
  cudaDeviceSynchronize();
  free_ksw(k);
  if (prev >= 0) cudaSetDevice(prev);
}

fnl_status fnl_ksw_info(const fnl_ksw* k, double* norm, double* norm_seconds, int* rank) {
  return guard([&] {
    FNL_REQUIRE(k, "estimator is NULL");
    if (norm) *norm = k->norm;
    if (norm_seconds) *norm_seconds = k->norm_seconds;
    if (rank)
      for (int l = 0; l <= k->lmax; ++l) rank[l] = k->rank[l];
  });
}

fnl_status fnl_ksw_statistic(const fnl_ksw* k, const double* aT, const double* aE, double* S, void* stream) {
  return guard([&] {
    FNL_REQUIRE(k, "estimator is NULL");
    DeviceScope scope(k->device);
    check_dev_ptr(aT, "aT", false);
    check_dev_ptr(aE, "aE", false);
    check_dev_ptr(S, "S", false);
    cudaStream_t st = (cudaStream_t)stream;
    const fnl_shells* syn = k->syn;
    const unsigned blocks = (unsigned)std::min<int64_t>(syn->nalm, (int64_t)syn->sms * 16);
    FNL_CUDA(cudaMemsetAsync(k->d_amax, 0, sizeof(unsigned long long), st));
    k_ksw_amax<<<std::max(1u, std::min(blocks, (unsigned)syn->sms * 4)), 256, 0, st>>>(
        syn->nalm, (const double2*)aT, (const double2*)aE, k->d_amax);
    FNL_CUDA(cudaGetLastError());
    if (syn->nterms)
      k_ksw_coeffs_tc<<<(unsigned)std::min<int64_t>((syn->nalm + 7) / 8, (int64_t)syn->sms * 32), 256, 0, st>>>(
          k->lmax, k->nr, syn->nalm, k->d_f32, (const double2*)aT, (const double2*)aE, k->d_amax, k->fmax[0],
          k->fmax[1], syn->nterms, syn->Cpad, syn->phiT_stride, syn->d_row32, (__nv_bfloat16*)syn->d_phiT);
    else if (syn->real_is_double)
      k_ksw_coeffs<double><<<blocks, 256, 0, st>>>(k->lmax, k->nr, syn->nalm, k->d_f, (const double2*)aT,
                                                   (const double2*)aE, k->d_amax, k->fmax[0], k->fmax[1], 0, 0, 0,
                                                   syn->d_row0, nullptr, (double*)syn->d_phi);
    else
      k_ksw_coeffs<float><<<blocks, 256, 0, st>>>(k->lmax, k->nr, syn->nalm, k->d_f32, (const double2*)aT,
                                                  (const double2*)aE, k->d_amax, k->fmax[0], k->fmax[1], 0, 0, 0,
                                                  syn->d_row0, nullptr, (float*)syn->d_phi);
    FNL_CUDA(cudaGetLastError());
    launch_synthesis_gemm(syn, st);
    if (!launch_ring_cubic_sq(syn, k->nr, k->d_part, st)) launch_ring_cubic(syn, k->nr, k->d_part, st);
    k_ksw_reduce<<<1, 1024, 0, st>>>(k->nr, k->npairs, k->d_part, k->d_u, 2.0 * M_PI / k->nphi, k->d_amax,
                                     k->fmax[0], k->fmax[1], S);
    FNL_CUDA(cudaGetLastError());
  });
}

}  // extern "C"
