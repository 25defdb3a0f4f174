// Normalised associated Legendre tables lambda_lm(x_jp) on the northern Gauss-Legendre
// rings, computed on the device in FP64 (the paper's SHTs came from HEALPix, which does
// this internally; the recurrence is the standard normalised three-term one).
//
//   lambda_00 = 1 / sqrt(4 pi),  lambda_mm = -sqrt((2m+1)/(2m)) sin(theta) lambda_{m-1,m-1}
//   lambda_lm = a_lm (x lambda_{l-1,m} - b_lm lambda_{l-2,m}),
//   a_lm = sqrt((4l^2-1)/(l^2-m^2)),  b_lm = sqrt(((l-1)^2-m^2)/(4(l-1)^2-1)).
//
// lambda_mm is carried as mantissa * 2^exponent so that sin(theta)^m never underflows,
// and the l recurrence runs on mantissas with a shared exponent moved by 2^500 steps.
// Values with |lambda| < 1e-290 are stored as exact zeros.
#include <algorithm>
#include <cmath>
#include <vector>

#include "fnl_internal.cuh"

namespace fnl {

namespace {

__global__ void k_lambda_mm(const double* __restrict__ x, const double* __restrict__ fac, int npairs,
                            int L, double* __restrict__ mant, int* __restrict__ expo) {
  const int jp = blockIdx.x * blockDim.x + threadIdx.x;
  if (jp >= npairs) return;
  const double xx = x[jp];
  const double s = sqrt((1.0 - xx) * (1.0 + xx));
  int e;
  double v = frexp(0.28209479177387814347, &e);  // 1 / sqrt(4 pi)
  mant[jp] = v;
  expo[jp] = e;
  for (int m = 1; m <= L; ++m) {
    int de;
    v = frexp(v * fac[m] * s, &de);
    e += de;
    mant[(size_t)m * npairs + jp] = v;
    expo[(size_t)m * npairs + jp] = e;
  }
}

__device__ __forceinline__ double flushed(double v) { return fabs(v) < 1e-290 ? 0.0 : v; }

// Ring pairs of an order where every |lambda_lm| stays below this bound are left out of the SIMT
// GEMMs: 2^-30 for the FP32 form (as the tensor-core forms), 2^-60 for the FP64 one (the dropped
// terms stay far below its 1e-12 bar).
template <typename T>
constexpr double simt_skip() { return sizeof(T) == 4 ? 0x1p-30 : 0x1p-60; }

// One thread per (jp, m); writes lambda_lm(x_jp) for l = m..L into the SIMT table
// lam[lam0[mp] + jp * KP[mp] + k], l = m + p + 2k; jmin[m] becomes the first ring pair (from
// the pole) where some |lambda_lm| reaches simt_skip<T>().
template <typename T>
__global__ void k_lambda_table(const double* __restrict__ x, const double* __restrict__ mant,
                               const int* __restrict__ expo, const double2* __restrict__ ab,
                               const int64_t* __restrict__ lam0, const int* __restrict__ K, int npairs,
                               int L, T* __restrict__ lam, int* __restrict__ jmin) {
  const int jp = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = blockIdx.y;
  if (jp >= npairs) return;
  const double xx = x[jp];
  double y1 = mant[(size_t)m * npairs + jp], y2 = 0.0;
  int e = expo[(size_t)m * npairs + jp];
  const int KP0 = (K[2 * m] + 15) / 16 * 16, KP1 = (K[2 * m + 1] + 15) / 16 * 16;
  T* row0 = lam + lam0[2 * m] + (int64_t)jp * KP0;
  T* row1 = lam + lam0[2 * m + 1] + (int64_t)jp * KP1;
  double vmax = fabs(flushed(ldexp(y1, e)));
  row0[0] = (T)flushed(ldexp(y1, e));
  const int64_t base = alm_idx(0, m, L);
  for (int l = m + 1; l <= L; ++l) {
    const double2 c = ab[base + l];
    const double y = c.x * (xx * y1 - c.y * y2);
    y2 = y1;
    y1 = y;
    if (fabs(y1) > 0x1p500) {
      y1 *= 0x1p-500;
      y2 *= 0x1p-500;
      e += 500;
    }
    const double vd = flushed(ldexp(y1, e));
    vmax = fmax(vmax, fabs(vd));
    const T v = (T)vd;
    const int d = l - m;
    if (d & 1) row1[d >> 1] = v;
    else row0[d >> 1] = v;
  }
  if (vmax >= simt_skip<T>()) atomicMin(&jmin[m], jp);
}

}  // namespace

void launch_lambda_mm(const double* x, const double* fac, int npairs, int L, double* mant, int* expo,
                      cudaStream_t st) {
  k_lambda_mm<<<(npairs + 127) / 128, 128, 0, st>>>(x, fac, npairs, L, mant, expo);
  FNL_CUDA(cudaGetLastError());
}

void build_lambda_tables(fnl_shells* sh, cudaStream_t st) {
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
  k_lambda_mm<<<(np + 127) / 128, 128, 0, st>>>(sh->d_x, d_fac, np, L, d_mant, d_expo);
  FNL_CUDA(cudaGetLastError());
  const size_t tbytes = sh->real_is_double ? sizeof(double) : sizeof(float);
  FNL_CUDA(cudaMemsetAsync(sh->d_lam, 0, tbytes * (size_t)sh->lam_total, st));
  TempDev t_jmin(sizeof(int) * (L + 1));
  int* d_jmin = t_jmin.as<int>();
  FNL_CUDA(cudaMemsetAsync(d_jmin, 0x7f, sizeof(int) * (L + 1), st));  // above any ring pair
  dim3 grid((np + 127) / 128, L + 1);
  if (sh->real_is_double)
    k_lambda_table<double><<<grid, 128, 0, st>>>(sh->d_x, d_mant, d_expo, d_ab, sh->d_lam0, sh->d_K, np, L,
                                                 (double*)sh->d_lam, d_jmin);
  else
    k_lambda_table<float><<<grid, 128, 0, st>>>(sh->d_x, d_mant, d_expo, d_ab, sh->d_lam0, sh->d_K, np, L,
                                                (float*)sh->d_lam, d_jmin);
  FNL_CUDA(cudaGetLastError());
  sh->jmin.assign(L + 1, 0);
  FNL_CUDA(cudaMemcpyAsync(sh->jmin.data(), d_jmin, sizeof(int) * (L + 1), cudaMemcpyDeviceToHost, st));
  FNL_CUDA(cudaStreamSynchronize(st));
  for (int& j : sh->jmin) j = std::min(j, np);
}

}  // namespace fnl
