// Output maps: the Stokes I, Q, U maps of one realisation on the ring grid (the paper's
// deliverable is temperature and polarization maps, I, Q and U; Sect. 4).
//
//   I = sum_lm a^T_lm Y_lm,   Q +- iU = sum_lm a_{+-2,lm} +-2Y_lm,   a_{+-2,lm} = -(a^E_lm +- i a^B_lm)
//
// Tables (fnl_maps_prepare, once): lambda_lm, W_lm = (2lam + (-2)lam) / 2 and
// X_lm = (2lam - (-2)lam) / 2 on the northern rings, from the FP64 three-term recurrence for
// lambda and the spin raising / lowering operators applied twice to Y_lm:
//   W = N_l [((2 m^2 - 2 l x^2) lam_l + 2 x c_lm lam_{l-1}) / (1 - x^2) - l (l+1) lam_l]
//   X = N_l 2 m [(1 - l) x lam_l + c_lm lam_{l-1}] / (1 - x^2)
// with N_l = ((l-1) l (l+1) (l+2))^(-1/2), c_lm = sqrt((2l+1)(l^2 - m^2) / (2l-1)) and 0 for l < 2.
// The two terms of W cancel to a part in l^2, so they are formed in FP64 and only the result
// is rounded to the table type.  lambda and W have the parity of l - m under x -> -x, X the
// opposite one.
//
// Table layout: one row per (m, parity, k), l = m + parity + 2 k, rows of one m at
// alm_idx(m, m) (even degrees, then odd), each row npj ring pairs long (ring pair fastest, so
// that a warp's loads of one row are contiguous); nalm x npj entries per table.
//
// Per call (fnl_maps): per order m and group of ring pairs (one 16-byte vector of table
// entries), four threads sum interleaved slices of l with the block's coefficients staged in
// shared memory, into F in the SIMT layout (problem
// 2 m + parity, ring pair, 6 columns = I, Q, U as complex numbers):
//   I_m = sum_l T lam,  Q_m = -sum_l (E W + i B X),  U_m = sum_l (i E X - B W)
// split into the parts even and odd under x -> -x; the ring kernel of the synthesis then
// writes north = even + odd and south = even - odd rings of the three maps.
#include <cmath>
#include <vector>

#include "fnl_internal.cuh"

namespace fnl {

namespace {

__device__ __forceinline__ double flushed_d(double v) { return fabs(v) < 1e-290 ? 0.0 : v; }

__device__ __forceinline__ int64_t map_row(int m, int p, int k, int L) {
  return alm_idx(m, m, L) + (p ? (L - m + 2) / 2 : 0) + k;
}

// Ring pairs of an order m where every |lambda|, |W|, |X| stays below this bound (in the polar
// cap where the functions of that order decay) are left out of the ring sums: 2^-30 for the
// FP32 tables (the dropped terms stay below 1e-8 of the maps), 2^-60 for the FP64 ones.
template <typename T>
constexpr double maps_skip() { return sizeof(T) == 4 ? 0x1p-30 : 0x1p-60; }

// One thread per (jp, m): lambda, W, X for l = m..L into the three tables; jmin[m] becomes the
// first ring pair (from the pole) where one of them reaches maps_skip<T>().
template <typename T>
__global__ void k_maps_tables(const double* __restrict__ x, const double* __restrict__ mant,
                              const int* __restrict__ expo, const double2* __restrict__ ab, int npairs, int npj,
                              int L, T* __restrict__ tl, T* __restrict__ tw, T* __restrict__ tx,
                              int* __restrict__ jmin) {
  const int jp = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = blockIdx.y;
  if (jp >= npairs) return;
  const double xx = x[jp], s2 = (1.0 - xx) * (1.0 + xx);
  double y1 = mant[(size_t)m * npairs + jp], y2 = 0.0;  // lam_l, lam_{l-1} (mantissas, shared exponent)
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
    double w = 0.0, xv = 0.0;
    if (l >= 2) {
      const double dl = l, dm = m;
      const double nl = 1.0 / sqrt((dl - 1.0) * dl * (dl + 1.0) * (dl + 2.0));
      const double c = sqrt((2.0 * dl + 1.0) * (dl * dl - dm * dm) / (2.0 * dl - 1.0));
      w = nl * (((2.0 * dm * dm - 2.0 * dl * xx * xx) * y1 + 2.0 * xx * c * y2) / s2 - dl * (dl + 1.0) * y1);
      xv = nl * 2.0 * dm * ((1.0 - dl) * xx * y1 + c * y2) / s2;
    }
    const int d = l - m;
    const int64_t o = map_row(m, d & 1, d >> 1, L) * npj + jp;
    const double vl = flushed_d(ldexp(y1, e)), vw = flushed_d(ldexp(w, e)), vx = flushed_d(ldexp(xv, e));
    vmax = fmax(vmax, fmax(fabs(vl), fmax(fabs(vw), fabs(vx))));
    tl[o] = (T)vl;
    tw[o] = (T)vw;
    tx[o] = (T)vx;
  }
  if (vmax >= maps_skip<T>()) atomicMin(&jmin[m], jp);
}

// Stages the coefficients of m (three fields, l = m..L) into sa[3 (l - m) + field] as T.
template <typename T>
__device__ __forceinline__ void stage_alm(cplx<T>* sa, int m, int L, const double* aT, const double* aE,
                                          const double* aB) {
  const int nl = L - m + 1;
  const int64_t base = alm_idx(m, m, L);
  for (int i = threadIdx.x; i < 3 * nl; i += blockDim.x) {
    const int f = i / nl, d = i - f * nl;
    const double* a = f == 0 ? aT : f == 1 ? aE : aB;
    const double2 v = a ? ((const double2*)a)[base + d] : make_double2(0.0, 0.0);
    sa[3 * d + f] = {(T)v.x, (T)v.y};
  }
}

// 16-byte vectors of table entries: four FP32 or two FP64 ring pairs.
template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
  static constexpr int N = 4;
  __device__ static void load(const float* p, float (&v)[4]) {
    const float4 q = __ldg((const float4*)p);
    v[0] = q.x;
    v[1] = q.y;
    v[2] = q.z;
    v[3] = q.w;
  }
};
template <>
struct Vec16<double> {
  static constexpr int N = 2;
  __device__ static void load(const double* p, double (&v)[2]) {
    const double2 q = __ldg((const double2*)p);
    v[0] = q.x;
    v[1] = q.y;
  }
};

constexpr int kMapsQ = 32;       // vectors (groups of ring pairs) of a block: one warp wide
constexpr int kMapsSlices = 4;   // k slices of a block: slice s sums k = s, s + 4, ...
constexpr int kMapsBatch = 4;    // k steps of a slice whose loads are issued together

// Block (x, m): ring pairs x * 32 N .. of order m (N = 16 / sizeof(T) per thread), 128 threads =
// 32 vectors x 4 k slices.  A vector wholly below jmin[m] reads no table and writes zeros.  The coefficients of m are staged in shared memory as T; each thread
// sums its slice of l for the even and odd parts of I_m, Q_m, U_m on its N ring pairs (in T),
// loading the lambda, W, X rows of kMapsBatch steps before using them; slice 0 then adds the
// other slices' sums in a fixed order and writes F.
template <typename T>
__global__ void __launch_bounds__(kMapsQ * kMapsSlices) k_maps_rings(
    const T* __restrict__ tl, const T* __restrict__ tw, const T* __restrict__ tx, int npairs, int npj, int L,
    const double* __restrict__ aT, const double* __restrict__ aE, const double* __restrict__ aB,
    const int* __restrict__ jmin, T* __restrict__ F) {
  constexpr int N = Vec16<T>::N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int m = blockIdx.y;
  T* red = (T*)smem_raw;                                                 // [slice - 1][12 N][32]
  cplx<T>* sa = (cplx<T>*)(red + (kMapsSlices - 1) * 12 * N * kMapsQ);  // [l - m][T, E, B]
  stage_alm(sa, m, L, aT, aE, aB);
  __syncthreads();
  const int lane = threadIdx.x % kMapsQ, slice = threadIdx.x / kMapsQ;
  const int jp0 = (blockIdx.x * kMapsQ + lane) * N;
  // rows are npj (a multiple of 32) long, so a vector that starts below npairs is in bounds
  const bool live = jp0 < npairs;
  // [ring pair][parity][I re, I im, Q re, Q im, U re, U im]
  T acc[N][2][6];
#pragma unroll
  for (int j = 0; j < N; ++j)
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
      for (int c = 0; c < 6; ++c) acc[j][p][c] = (T)0;
  if (live && jp0 + N > jmin[m]) {
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      const int Kp = (L - m - p + 2) / 2;
      const size_t o0 = (size_t)map_row(m, p, 0, L) * npj + jp0;
      const cplx<T>* ca = sa + 3 * p;
      for (int k0 = slice; k0 < Kp; k0 += kMapsSlices * kMapsBatch) {
        T lv[kMapsBatch][N], wv[kMapsBatch][N], xv[kMapsBatch][N];
#pragma unroll
        for (int b = 0; b < kMapsBatch; ++b) {
          const int k = k0 + b * kMapsSlices;
          if (k < Kp) {
            const size_t o = o0 + (size_t)k * npj;
            Vec16<T>::load(tl + o, lv[b]);
            Vec16<T>::load(tw + o, wv[b]);
            Vec16<T>::load(tx + o, xv[b]);
          }
        }
#pragma unroll
        for (int b = 0; b < kMapsBatch; ++b) {
          const int k = k0 + b * kMapsSlices;
          if (k < Kp) {
            const cplx<T> t = ca[6 * k], e = ca[6 * k + 1], bb = ca[6 * k + 2];
#pragma unroll
            for (int j = 0; j < N; ++j) {
              // I: lambda has parity p
              acc[j][p][0] += lv[b][j] * t.x;
              acc[j][p][1] += lv[b][j] * t.y;
              // W terms (parity p): Q -= W E, U -= W B
              acc[j][p][2] -= wv[b][j] * e.x;
              acc[j][p][3] -= wv[b][j] * e.y;
              acc[j][p][4] -= wv[b][j] * bb.x;
              acc[j][p][5] -= wv[b][j] * bb.y;
              // X terms (parity 1 - p): Q -= i X B, U += i X E
              acc[j][1 - p][2] += xv[b][j] * bb.y;
              acc[j][1 - p][3] -= xv[b][j] * bb.x;
              acc[j][1 - p][4] -= xv[b][j] * e.y;
              acc[j][1 - p][5] += xv[b][j] * e.x;
            }
          }
        }
      }
    }
  }
  if (slice > 0) {
#pragma unroll
    for (int c = 0; c < 12 * N; ++c) red[((slice - 1) * 12 * N + c) * kMapsQ + lane] = acc[c / 12][(c / 6) % 2][c % 6];
  }
  __syncthreads();
  if (slice > 0 || !live) return;
#pragma unroll
  for (int sl = 1; sl < kMapsSlices; ++sl)
#pragma unroll
    for (int c = 0; c < 12 * N; ++c) acc[c / 12][(c / 6) % 2][c % 6] += red[((sl - 1) * 12 * N + c) * kMapsQ + lane];
#pragma unroll
  for (int j = 0; j < N; ++j) {
    if (jp0 + j >= npairs) break;
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      T* out = F + ((size_t)(2 * m + p) * npairs + jp0 + j) * 6;
#pragma unroll
      for (int c = 0; c < 6; ++c) out[c] = acc[j][p][c];
    }
  }
}

template <typename T>
void build_tables(fnl_shells* sh) {
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
  auto release = [&] {
    cudaFree(d_fac);
    cudaFree(d_mant);
    cudaFree(d_expo);
    cudaFree(d_ab);
  };
  try {
    FNL_CUDA(cudaMalloc(&d_fac, sizeof(double) * (L + 1)));
    FNL_CUDA(cudaMalloc(&d_mant, sizeof(double) * (size_t)(L + 1) * np));
    FNL_CUDA(cudaMalloc(&d_expo, sizeof(int) * (size_t)(L + 1) * np));
    FNL_CUDA(cudaMalloc(&d_ab, sizeof(double2) * (size_t)sh->nalm));
    FNL_CUDA(cudaMemcpy(d_fac, fac.data(), sizeof(double) * (L + 1), cudaMemcpyHostToDevice));
    FNL_CUDA(cudaMemcpy(d_ab, ab.data(), sizeof(double2) * ab.size(), cudaMemcpyHostToDevice));
    launch_lambda_mm(sh->d_x, d_fac, np, L, d_mant, d_expo, 0);
    const size_t bytes = sizeof(T) * (size_t)sh->nalm * sh->npj;
    for (void* t : {sh->d_mapL, sh->d_mapW, sh->d_mapX}) FNL_CUDA(cudaMemset(t, 0, bytes));
    FNL_CUDA(cudaMemset(sh->d_maps_jmin, 0x7f, sizeof(int) * (L + 1)));  // above any ring pair
    k_maps_tables<T><<<dim3((np + 127) / 128, L + 1), 128>>>(sh->d_x, d_mant, d_expo, d_ab, np, sh->npj, L,
                                                             (T*)sh->d_mapL, (T*)sh->d_mapW, (T*)sh->d_mapX,
                                                             sh->d_maps_jmin);
    FNL_CUDA(cudaGetLastError());
    FNL_CUDA(cudaDeviceSynchronize());
  } catch (...) {
    release();
    throw;
  }
  release();
}

}  // namespace

void maps_prepare(fnl_shells* sh) {
  if (sh->maps_ready) return;
  const size_t ts = sh->real_is_double ? sizeof(double) : sizeof(float);
  const size_t tb = ts * (size_t)sh->nalm * sh->npj;
  const size_t fb = ts * (size_t)2 * (sh->lmax + 1) * sh->npairs * 6;
  void* p[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  const size_t sz[5] = {tb, tb, tb, fb, sizeof(int) * (size_t)(sh->lmax + 1)};
  for (int i = 0; i < 5; ++i) {
    const cudaError_t e = cudaMalloc(&p[i], sz[i]);
    if (e != cudaSuccess) {
      for (int j = 0; j < i; ++j) cudaFree(p[j]);
      cudaGetLastError();
      throw Error(e == cudaErrorMemoryAllocation ? FNL_ENOMEM : FNL_ECUDA, "fnl_maps_prepare: allocation failed");
    }
  }
  sh->d_mapL = p[0];
  sh->d_mapW = p[1];
  sh->d_mapX = p[2];
  sh->d_Fiqu = p[3];
  sh->d_maps_jmin = (int*)p[4];
  for (int i = 0; i < 5; ++i) {
    sh->allocations.push_back(p[i]);
    sh->device_bytes += sz[i];
  }
  FNL_CUDA(cudaMemset(sh->d_Fiqu, 0, fb));
  if (sh->real_is_double) build_tables<double>(sh);
  else build_tables<float>(sh);
  sh->maps_ready = true;
}

template <typename T>
void maps_rings_impl(const fnl_shells* sh, const double* aT, const double* aE, const double* aB, cudaStream_t st) {
  constexpr int N = Vec16<T>::N;
  const int L = sh->lmax, np = sh->npairs;
  const int nvec = (np + N - 1) / N;
  const size_t smem = sizeof(T) * (kMapsSlices - 1) * 12 * N * kMapsQ + sizeof(cplx<T>) * 3 * (size_t)(L + 1);
  FNL_CUDA(cudaFuncSetAttribute(k_maps_rings<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_maps_rings<T><<<dim3((nvec + kMapsQ - 1) / kMapsQ, L + 1), kMapsQ * kMapsSlices, smem, st>>>(
      (const T*)sh->d_mapL, (const T*)sh->d_mapW, (const T*)sh->d_mapX, np, sh->npj, L, aT, aE, aB,
      sh->d_maps_jmin, (T*)sh->d_Fiqu);
  FNL_CUDA(cudaGetLastError());
}

void launch_maps(const fnl_shells* sh, const double* aT, const double* aE, const double* aB, double* maps,
                 cudaStream_t st) {
  if (sh->real_is_double) maps_rings_impl<double>(sh, aT, aE, aB, st);
  else maps_rings_impl<float>(sh, aT, aE, aB, st);
  launch_ring_synth_fields(sh, sh->d_Fiqu, 3, maps, st);
}

}  // namespace fnl
