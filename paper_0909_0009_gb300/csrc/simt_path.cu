// SIMT kernels of the FP64 and FP32 forms of the path (real type T = double or float):
//   k_filter        step (i), Eq. 9: Phi_L = K_l n per (l, m), with a^X_L = v^X_l . n (Eq. 5)
//   k_synth_gemm    step (ii), Legendre half: per (m, parity) F = Lambda Phi over the northern rings
//   k_analysis_gemm step (iv), Legendre half: per (m, parity) Phi = Lambda^T G
//   k_quadrature    step (v), Eq. 5 and Eq. 3, FP64 accumulation
// plus the layout conversions used by the stage entry points.
#include <cmath>

#include "fnl_internal.cuh"
#include "philox.cuh"

namespace fnl {

namespace {

constexpr int kThreads = 256;

// ---------------------------------------------------------------------------------------
// Step (i): one block per degree l (largest first); K_l and v^X_l staged in shared memory;
// for every m <= l draw (or read) n_lm(r_j), write Phi_L,lm(r_i) = sum_{j<=i} K_l[i,j] n_j
// into the internal [rows][C] buffer (and optionally the API layout), and a^X_L,lm = v . n.
// The object's nr rows are the shells j0 .. j0 + nr - 1 of its configuration (j0 = 0 unless
// it is a shell shard); they need the noise of shells 0 .. ncol - 1, ncol = j0 + nr, and the
// staged K_l is [nr][ncol] (row i holds K_l[j0 + i][0 .. ncol)).
// ---------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) k_filter(int L, int nr, int j0, int ncol, const T* __restrict__ Kf,
                                                     const double* __restrict__ vT,
                                                     const double* __restrict__ vE, uint64_t seed,
                                                     uint64_t real, const double* __restrict__ noise,
                                                     const int64_t* __restrict__ row0, T* __restrict__ phi,
                                                     double* __restrict__ phi_api, double* __restrict__ aLT,
                                                     double* __restrict__ aLE) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int l = L - blockIdx.x;
  const int C = 2 * nr;
  double2* ns = (double2*)smem;                   // [ncol] noise of the current (l, m)
  double* vs = (double*)(ns + ncol);              // [2][ncol]
  double* red = vs + 2 * ncol;                    // [4][kThreads / 32]
  T* Ks = (T*)(red + 4 * (kThreads / 32));        // [nr][ncol + 1] (padded rows: no bank conflicts)
  T* nt = Ks + (size_t)nr * (ncol + 1);           // [2][ncol] the noise in T (re, then im)
  const int ldk = ncol + 1;
  const T* Kl = Kf + (size_t)l * nr * ncol;
  for (int e = threadIdx.x; e < nr * ncol; e += kThreads) Ks[(e / ncol) * ldk + (e % ncol)] = Kl[e];
  for (int e = threadIdx.x; e < ncol; e += kThreads) {
    vs[e] = vT[(size_t)l * ncol + e];
    vs[ncol + e] = vE[(size_t)l * ncol + e];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int m = 0; m <= l; ++m) {
    const int64_t idx = alm_idx(l, m, L);
    __syncthreads();
    if (noise) {
      for (int j = threadIdx.x; j < ncol; j += kThreads) {
        double2 v = ((const double2*)noise)[(size_t)j * (size_t)(((int64_t)(L + 1) * (L + 2)) / 2) + idx];
        if (m == 0) v.y = 0.0;
        ns[j] = v;
      }
    } else {
      // the FP64 form draws in FP64; the FP32 form through the FP32 Box-Muller of the mixed
      // forms (the FP64 pipe of this part is far too slow for a transcendental per draw)
      for (int jq = threadIdx.x; jq < (ncol + 3) / 4; jq += kThreads) {
        uint64_t w[4];
        noise_words(seed, real, idx, jq, w);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int j = 4 * jq + q;
          if (j >= ncol) break;
          if (sizeof(T) == sizeof(double)) {
            ns[j] = noise_value(box_muller(w[q]), m);
          } else {
            const float2 g = noise_value_f32(box_muller_f32(w[q]), m);
            ns[j] = make_double2(g.x, g.y);
          }
        }
      }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < ncol; j += kThreads) {
      nt[j] = (T)ns[j].x;
      nt[ncol + j] = (T)ns[j].y;
    }
    // a^X_L = sum_j v^X_l[j] n_j  (FP64)
    double tr = 0.0, ti = 0.0, er = 0.0, ei = 0.0;
    for (int j = threadIdx.x; j < ncol; j += kThreads) {
      const double2 n = ns[j];
      tr += vs[j] * n.x;
      ti += vs[j] * n.y;
      er += vs[ncol + j] * n.x;
      ei += vs[ncol + j] * n.y;
    }
    for (int o = 16; o; o >>= 1) {
      tr += __shfl_xor_sync(0xffffffffu, tr, o);
      ti += __shfl_xor_sync(0xffffffffu, ti, o);
      er += __shfl_xor_sync(0xffffffffu, er, o);
      ei += __shfl_xor_sync(0xffffffffu, ei, o);
    }
    if (lane == 0) {
      red[warp] = tr;
      red[8 + warp] = ti;
      red[16 + warp] = er;
      red[24 + warp] = ei;
    }
    __syncthreads();  // nt complete
    // Phi_L,lm(r_i) = sum_{j <= j0 + i} K_l[j0 + i, j] n_j
    const int p = (l - m) & 1;
    const int64_t row = row0[2 * m + p] + ((l - m) >> 1);
    for (int c = threadIdx.x; c < C; c += kThreads) {
      const int i = c >> 1, r = c & 1;
      T acc = 0;
      const T* Ki = Ks + (size_t)i * ldk;
      const T* nj = nt + (r ? ncol : 0);
      for (int j = 0; j <= j0 + i; ++j) acc += Ki[j] * nj[j];
      phi[row * C + c] = acc;
      if (phi_api) phi_api[((size_t)idx * nr + i) * 2 + r] = (double)acc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
      for (int w = 0; w < kThreads / 32; ++w) {
        s0 += red[w];
        s1 += red[8 + w];
        s2 += red[16 + w];
        s3 += red[24 + w];
      }
      ((double2*)aLT)[idx] = make_double2(s0, s1);
      ((double2*)aLE)[idx] = make_double2(s2, s3);
    }
  }
}

// ---------------------------------------------------------------------------------------
// Grouped SIMT GEMMs.  64 x 64 output tile, 16-deep k slices, 4 x 4 outputs per thread.
// ---------------------------------------------------------------------------------------
constexpr int BM = 64, BN = 64, BK = 16;

// F[mp][jp][c] = sum_k Lambda[mp][jp][k] Phi[mp][k][c]   (rows jp, columns c, depth k)
template <typename T>
__global__ void __launch_bounds__(kThreads) k_synth_gemm(const Tile* __restrict__ tiles,
                                                         const int* __restrict__ K,
                                                         const int64_t* __restrict__ lam0,
                                                         const int64_t* __restrict__ row0,
                                                         const T* __restrict__ lam, const T* __restrict__ phi,
                                                         T* __restrict__ F, int npairs, int C) {
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  const Tile t = tiles[blockIdx.x];
  const int mp = t.mp, j0 = t.rt * BM, c0 = t.ct * BN;
  const int KP = (K[mp] + 15) / 16 * 16;
  const T* A = lam + lam0[mp];
  const T* B = phi + row0[mp] * C;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T acc[4][4] = {};
  for (int k0 = t.q0; k0 < KP; k0 += BK) {
    for (int e = threadIdx.x; e < BM * BK; e += kThreads) {
      const int r = e >> 4, kk = e & 15;
      As[kk][r] = (j0 + r < npairs) ? A[(int64_t)(j0 + r) * KP + k0 + kk] : (T)0;
    }
    for (int e = threadIdx.x; e < BN * BK; e += kThreads) {
      const int kk = e >> 6, cc = e & 63;
      Bs[kk][cc] = (c0 + cc < C) ? B[(int64_t)(k0 + kk) * C + c0 + cc] : (T)0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
    }
    __syncthreads();
  }
  T* out = F + (int64_t)mp * npairs * C;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = j0 + ty + 16 * i;
    if (r >= npairs) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = c0 + tx + 16 * j;
      if (c < C) out[(int64_t)r * C + c] = acc[i][j];
    }
  }
}

// Phi[mp][k][c] = sum_jp Lambda[mp][jp][k] G[mp][jp][c]   (rows k < K[mp], columns c, depth jp)
template <typename T>
__global__ void __launch_bounds__(kThreads) k_analysis_gemm(const Tile* __restrict__ tiles,
                                                            const int* __restrict__ K,
                                                            const int64_t* __restrict__ lam0,
                                                            const int64_t* __restrict__ row0,
                                                            const T* __restrict__ lam, const T* __restrict__ G,
                                                            T* __restrict__ phi, int npairs, int C) {
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  const Tile t = tiles[blockIdx.x];
  const int mp = t.mp, k0 = t.rt * BM, c0 = t.ct * BN;
  const int Km = K[mp];
  const int KP = (Km + 15) / 16 * 16;
  const T* A = lam + lam0[mp];
  const T* B = G + (int64_t)mp * npairs * C;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T acc[4][4] = {};
  for (int q0 = t.q0; q0 < npairs; q0 += BK) {
    for (int e = threadIdx.x; e < BM * BK; e += kThreads) {
      const int kk = e >> 6, r = e & 63;
      As[kk][r] = (q0 + kk < npairs && k0 + r < KP) ? A[(int64_t)(q0 + kk) * KP + k0 + r] : (T)0;
    }
    for (int e = threadIdx.x; e < BN * BK; e += kThreads) {
      const int kk = e >> 6, cc = e & 63;
      Bs[kk][cc] = (q0 + kk < npairs && c0 + cc < C) ? B[(int64_t)(q0 + kk) * C + c0 + cc] : (T)0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
    }
    __syncthreads();
  }
  T* out = phi + row0[mp] * C;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = k0 + ty + 16 * i;
    if (r >= Km) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = c0 + tx + 16 * j;
      if (c < C) out[(int64_t)r * C + c] = acc[i][j];
    }
  }
}

// (l, m) of triangle entry idx.
__device__ __forceinline__ void lm_of(int64_t idx, int L, int& l, int& m) {
  // start(m) = m (2L + 1 - m) / 2 is increasing in m; solve and correct by one step.
  // block m starts at m (2L + 3 - m) / 2; a float estimate is corrected exactly below
  const float b = 2.0f * L + 3.0f;
  int mm = (int)floorf((b - sqrtf(fmaxf(b * b - 8.0f * (float)idx, 0.0f))) * 0.5f);
  if (mm < 0) mm = 0;
  if (mm > L) mm = L;
  while (mm > 0 && alm_idx(mm, mm, L) > idx) --mm;
  while (mm < L && alm_idx(mm + 1, mm + 1, L) <= idx) ++mm;
  m = mm;
  l = (int)(idx - alm_idx(0, mm, L));
}

// ---------------------------------------------------------------------------------------
// Step (v): one warp per (l, m).  a^X_NL = sum_i q^X_l[i] Phi_NL(r_i) in FP64; optionally
// a^X = a^X_L + f_NL a^X_NL.  Phi comes from the internal buffer (from_internal) or from an
// API-layout array [nalm][nr][2].
// ---------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) k_quadrature(int L, int nr, int64_t nalm,
                                                         const int64_t* __restrict__ row0,
                                                         const T* __restrict__ phi_int,
                                                         const double* __restrict__ phi_api,
                                                         const double* __restrict__ qT,
                                                         const double* __restrict__ qE, double fnl,
                                                         const double* __restrict__ aLT,
                                                         const double* __restrict__ aLE,
                                                         double* __restrict__ outT, double* __restrict__ outE,
                                                         double* __restrict__ aT, double* __restrict__ aE) {
  const int64_t idx = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (idx >= nalm) return;
  int l, m;
  lm_of(idx, L, l, m);
  const int C = 2 * nr;
  double tr = 0, ti = 0, er = 0, ei = 0;
  if (phi_api) {
    const double* row = phi_api + (size_t)idx * C;
    for (int i = lane; i < nr; i += 32) {
      const double re = row[2 * i], im = row[2 * i + 1];
      const double a = qT[(size_t)l * nr + i], b = qE[(size_t)l * nr + i];
      tr += a * re;
      ti += a * im;
      er += b * re;
      ei += b * im;
    }
  } else {
    const int p = (l - m) & 1;
    const T* row = phi_int + (row0[2 * m + p] + ((l - m) >> 1)) * C;
    for (int i = lane; i < nr; i += 32) {
      const double re = (double)row[2 * i], im = (double)row[2 * i + 1];
      const double a = qT[(size_t)l * nr + i], b = qE[(size_t)l * nr + i];
      tr += a * re;
      ti += a * im;
      er += b * re;
      ei += b * im;
    }
  }
  for (int o = 16; o; o >>= 1) {
    tr += __shfl_xor_sync(0xffffffffu, tr, o);
    ti += __shfl_xor_sync(0xffffffffu, ti, o);
    er += __shfl_xor_sync(0xffffffffu, er, o);
    ei += __shfl_xor_sync(0xffffffffu, ei, o);
  }
  if (lane) return;
  if (outT) ((double2*)outT)[idx] = make_double2(tr, ti);
  if (outE) ((double2*)outE)[idx] = make_double2(er, ei);
  if (aT) {
    const double2 a = aLT ? ((const double2*)aLT)[idx] : make_double2(0.0, 0.0);
    ((double2*)aT)[idx] = make_double2(a.x + fnl * tr, a.y + fnl * ti);
  }
  if (aE) {
    const double2 a = aLE ? ((const double2*)aLE)[idx] : make_double2(0.0, 0.0);
    ((double2*)aE)[idx] = make_double2(a.x + fnl * er, a.y + fnl * ei);
  }
}

// a^X = a^X_L + f_NL a^X_NL (Eq. 3) when both parts already exist.
__global__ void k_combine(int64_t nalm, double fnl, const double2* __restrict__ aLT,
                          const double2* __restrict__ aLE, const double2* __restrict__ aNLT,
                          const double2* __restrict__ aNLE, double2* __restrict__ aT,
                          double2* __restrict__ aE) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nalm) return;
  if (aT) {
    const double2 a = aLT ? aLT[i] : make_double2(0, 0), b = aNLT ? aNLT[i] : make_double2(0, 0);
    aT[i] = make_double2(a.x + fnl * b.x, a.y + fnl * b.y);
  }
  if (aE) {
    const double2 a = aLE ? aLE[i] : make_double2(0, 0), b = aNLE ? aNLE[i] : make_double2(0, 0);
    aE[i] = make_double2(a.x + fnl * b.x, a.y + fnl * b.y);
  }
}

// API layout [nalm][nr][2] <-> internal rows.  One thread per (idx, c).
template <typename T>
__global__ void k_alm_to_phi(int L, int nr, int64_t nalm, const int64_t* __restrict__ row0,
                             const double* __restrict__ alm, T* __restrict__ phi) {
  const int C = 2 * nr;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nalm * C) return;
  const int64_t idx = t / C;
  const int c = (int)(t % C);
  int l, m;
  lm_of(idx, L, l, m);
  double v = alm[(size_t)idx * C + c];
  if (m == 0 && (c & 1)) v = 0.0;
  phi[(row0[2 * m + ((l - m) & 1)] + ((l - m) >> 1)) * C + c] = (T)v;
}

template <typename T>
__global__ void k_phi_to_alm(int L, int nr, int64_t nalm, const int64_t* __restrict__ row0,
                             const T* __restrict__ phi, double* __restrict__ alm) {
  const int C = 2 * nr;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nalm * C) return;
  const int64_t idx = t / C;
  const int c = (int)(t % C);
  int l, m;
  lm_of(idx, L, l, m);
  alm[(size_t)idx * C + c] = (double)phi[(row0[2 * m + ((l - m) & 1)] + ((l - m) >> 1)) * C + c];
}

template <typename T>
void filter_impl(const fnl_shells* sh, uint64_t seed, uint64_t real, const double* noise, double* aLT,
                 double* aLE, double* phi_api, cudaStream_t st) {
  const int nr = sh->nr, ncol = sh->j0 + sh->nr;
  const size_t smem = sizeof(double2) * ncol + sizeof(double) * 2 * ncol + sizeof(double) * 4 * (kThreads / 32) +
                      sizeof(T) * (size_t)nr * (ncol + 1) + sizeof(T) * 2 * (size_t)ncol;
  FNL_CUDA(cudaFuncSetAttribute(k_filter<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_filter<T><<<sh->lmax + 1, kThreads, smem, st>>>(sh->lmax, nr, sh->j0, ncol, (const T*)sh->d_Kf, sh->d_vT,
                                                    sh->d_vE, seed, real, noise, sh->d_row0, (T*)sh->d_phi,
                                                    phi_api, aLT, aLE);
  FNL_CUDA(cudaGetLastError());
}

}  // namespace

void launch_filter(const fnl_shells* sh, uint64_t seed, uint64_t real, const double* noise, double* aLT,
                   double* aLE, double* phi_api, cudaStream_t st) {
  if (sh->real_is_double) filter_impl<double>(sh, seed, real, noise, aLT, aLE, phi_api, st);
  else filter_impl<float>(sh, seed, real, noise, aLT, aLE, phi_api, st);
}

void launch_synth_gemm(const fnl_shells* sh, cudaStream_t st) {
  if (sh->real_is_double)
    k_synth_gemm<double><<<sh->n_tiles_syn, kThreads, 0, st>>>(sh->d_tiles_syn, sh->d_K, sh->d_lam0, sh->d_row0,
                                                              (const double*)sh->d_lam, (const double*)sh->d_phi,
                                                              (double*)sh->d_F, sh->npairs, sh->C);
  else
    k_synth_gemm<float><<<sh->n_tiles_syn, kThreads, 0, st>>>(sh->d_tiles_syn, sh->d_K, sh->d_lam0, sh->d_row0,
                                                             (const float*)sh->d_lam, (const float*)sh->d_phi,
                                                             (float*)sh->d_F, sh->npairs, sh->C);
  FNL_CUDA(cudaGetLastError());
}

void launch_synth_gemm_to(const fnl_shells* sh, void* out, cudaStream_t st) {
  if (sh->real_is_double)
    k_synth_gemm<double><<<sh->n_tiles_syn, kThreads, 0, st>>>(sh->d_tiles_syn, sh->d_K, sh->d_lam0, sh->d_row0,
                                                              (const double*)sh->d_lam, (const double*)sh->d_phi,
                                                              (double*)out, sh->npairs, sh->C);
  else
    k_synth_gemm<float><<<sh->n_tiles_syn, kThreads, 0, st>>>(sh->d_tiles_syn, sh->d_K, sh->d_lam0, sh->d_row0,
                                                             (const float*)sh->d_lam, (const float*)sh->d_phi,
                                                             (float*)out, sh->npairs, sh->C);
  FNL_CUDA(cudaGetLastError());
}

void launch_analysis_gemm(const fnl_shells* sh, cudaStream_t st) {
  if (sh->real_is_double)
    k_analysis_gemm<double><<<sh->n_tiles_ana, kThreads, 0, st>>>(
        sh->d_tiles_ana, sh->d_K, sh->d_lam0, sh->d_row0, (const double*)sh->d_lam, (const double*)sh->d_G,
        (double*)sh->d_phi, sh->npairs, sh->C);
  else
    k_analysis_gemm<float><<<sh->n_tiles_ana, kThreads, 0, st>>>(
        sh->d_tiles_ana, sh->d_K, sh->d_lam0, sh->d_row0, (const float*)sh->d_lam, (const float*)sh->d_G,
        (float*)sh->d_phi, sh->npairs, sh->C);
  FNL_CUDA(cudaGetLastError());
}

void launch_quadrature(const fnl_shells* sh, const double* phi_api, int from_internal, double fnl,
                       const double* aLT, const double* aLE, double* aT, double* aE, double* aNLT,
                       double* aNLE, int /*accumulate_into_L*/, cudaStream_t st) {
  const int64_t warps = sh->nalm;
  const unsigned blocks = (unsigned)((warps * 32 + kThreads - 1) / kThreads);
  if (sh->real_is_double)
    k_quadrature<double><<<blocks, kThreads, 0, st>>>(sh->lmax, sh->nr, sh->nalm, sh->d_row0,
                                                      from_internal ? (const double*)sh->d_phi : nullptr,
                                                      from_internal ? nullptr : phi_api, sh->d_qT, sh->d_qE, fnl,
                                                      aLT, aLE, aNLT, aNLE, aT, aE);
  else
    k_quadrature<float><<<blocks, kThreads, 0, st>>>(sh->lmax, sh->nr, sh->nalm, sh->d_row0,
                                                     from_internal ? (const float*)sh->d_phi : nullptr,
                                                     from_internal ? nullptr : phi_api, sh->d_qT, sh->d_qE, fnl,
                                                     aLT, aLE, aNLT, aNLE, aT, aE);
  FNL_CUDA(cudaGetLastError());
}

void launch_combine(const fnl_shells* sh, double fnl, const double* aLT, const double* aLE, const double* aNLT,
                    const double* aNLE, double* aT, double* aE, cudaStream_t st) {
  const unsigned blocks = (unsigned)((sh->nalm + 255) / 256);
  k_combine<<<blocks, 256, 0, st>>>(sh->nalm, fnl, (const double2*)aLT, (const double2*)aLE, (const double2*)aNLT,
                                    (const double2*)aNLE, (double2*)aT, (double2*)aE);
  FNL_CUDA(cudaGetLastError());
}

void launch_alm_to_phi(const fnl_shells* sh, const double* alm, cudaStream_t st) {
  const int64_t n = sh->nalm * sh->C;
  const unsigned blocks = (unsigned)((n + 255) / 256);
  if (sh->real_is_double)
    k_alm_to_phi<double><<<blocks, 256, 0, st>>>(sh->lmax, sh->nr, sh->nalm, sh->d_row0, alm, (double*)sh->d_phi);
  else
    k_alm_to_phi<float><<<blocks, 256, 0, st>>>(sh->lmax, sh->nr, sh->nalm, sh->d_row0, alm, (float*)sh->d_phi);
  FNL_CUDA(cudaGetLastError());
}

void launch_phi_to_alm(const fnl_shells* sh, double* alm, cudaStream_t st) {
  const int64_t n = sh->nalm * sh->C;
  const unsigned blocks = (unsigned)((n + 255) / 256);
  if (sh->real_is_double)
    k_phi_to_alm<double><<<blocks, 256, 0, st>>>(sh->lmax, sh->nr, sh->nalm, sh->d_row0, (const double*)sh->d_phi,
                                                 alm);
  else
    k_phi_to_alm<float><<<blocks, 256, 0, st>>>(sh->lmax, sh->nr, sh->nalm, sh->d_row0, (const float*)sh->d_phi,
                                                alm);
  FNL_CUDA(cudaGetLastError());
}

}  // namespace fnl
