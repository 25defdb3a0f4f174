// SIMT kernels of the FP64 and FP32 forms of the path (real type T = double or float):
//   k_filter        step (i), Eq. 9: Phi_L = K_l n per (l, m), with a^X_L = v^X_l . n (Eq. 5)
//   k_synth_gemm    step (ii), Legendre half: per (m, parity) F = Lambda Phi over the northern rings
//                   (FP32; k_synth_gemm64 for FP64)
//   k_analysis_gemm step (iv), Legendre half: per (m, parity) Phi = Lambda^T G (FP32;
//                   k_analysis_gemm64 for FP64)
//   k_quadrature    step (v), Eq. 5 and Eq. 3, FP64 accumulation
// plus the layout conversions used by the stage entry points.
#include <cmath>

#include "fnl_internal.cuh"
#include "philox.cuh"

namespace fnl {

namespace {

constexpr int kThreads = 256;

// ---------------------------------------------------------------------------------------
// Step (i) in tiles: a block per (degree l = L - blockIdx.x, largest first, and 32 orders
// m0 = 32 blockIdx.y ..).  K_l is staged with zeros right of the diagonal and v^X_l beside it;
// the tile's noise n_lm(r_j) is drawn (or read) into a [ncol][64 columns (m, part)] tile; a warp
// per order forms a^X_L,lm = v^X_l . n (FP64); and Phi_L,lm(r_i) = sum_{j <= j0 + i} K_l[j0 + i, j] n_j
// is a register tile per thread: rows i = rg + 32 r (r < ROWS), 8 columns.  The object's nr rows
// are the shells j0 .. j0 + nr - 1 of its configuration (j0 = 0 unless it is a shell shard); they
// need the noise of shells 0 .. ncol - 1, ncol = j0 + nr, and the staged K_l is [nr][ncol] (row i
// holds K_l[j0 + i][0 .. ncol)).  One block per degree with the orders in turn made the largest
// degree's block the whole kernel's time (4 ms at l_max 512 in FP32).
// ---------------------------------------------------------------------------------------
constexpr int kFlM = 32;            // orders per tile
constexpr int kFlCols = 2 * kFlM;   // columns (m, part)
constexpr int kFlMaxRows = 4;       // rows per thread: nr <= 128
template <typename T>
constexpr int fl_ldp() { return kFlCols + 16 / (int)sizeof(T); }  // noise tile row stride (16-byte aligned)

template <typename T>
size_t filter_smem(int nr, int ncol) {
  return sizeof(double) * 2 * (size_t)ncol + sizeof(T) * ((size_t)ncol * fl_ldp<T>() + (size_t)nr * (ncol + 1));
}

template <typename T, int ROWS>
__global__ void __launch_bounds__(kThreads) k_filter(int L, int nr, int j0, int ncol, const T* __restrict__ Kf,
                                                     const double* __restrict__ vT,
                                                     const double* __restrict__ vE, uint64_t seed,
                                                     uint64_t real, const double* __restrict__ noise,
                                                     const int64_t* __restrict__ row0, T* __restrict__ phi,
                                                     double* __restrict__ phi_api, double* __restrict__ aLT,
                                                     double* __restrict__ aLE) {
  const int l = L - blockIdx.x, m0 = kFlM * blockIdx.y;
  if (m0 > l) return;
  const int nm = min(kFlM, l + 1 - m0);  // orders of this tile
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int ldp = fl_ldp<T>();
  const int C = 2 * nr, ldk = ncol + 1;
  double* vs = (double*)smem;                    // [2][ncol] v^T_l, v^E_l
  T* P = (T*)(vs + 2 * ncol);                    // [ncol][ldp] the tile's noise, columns (m, part)
  T* Ks = P + (size_t)ncol * ldp;                // [nr][ncol + 1] K_l rows, zero right of the diagonal
  const T* Kl = Kf + (size_t)l * nr * ncol;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = warp; i < nr; i += kThreads / 32)
    for (int j = lane; j < ncol; j += 32) Ks[i * ldk + j] = j <= j0 + i ? Kl[(size_t)i * ncol + j] : (T)0;
  for (int e = threadIdx.x; e < ncol; e += kThreads) {
    vs[e] = vT[(size_t)l * ncol + e];
    vs[ncol + e] = vE[(size_t)l * ncol + e];
  }
  // the tile's noise: work item (order, quad of shells)
  const int nq = (ncol + 3) / 4;
  for (int e = threadIdx.x; e < kFlM * nq; e += kThreads) {
    const int ml = e / nq, jq = e % nq, m = m0 + ml;
    T re[4] = {(T)0, (T)0, (T)0, (T)0}, im[4] = {(T)0, (T)0, (T)0, (T)0};
    if (ml < nm) {
      const int64_t idx = alm_idx(l, m, L);
      if (noise) {
        const int64_t nalm = ((int64_t)(L + 1) * (L + 2)) / 2;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int j = 4 * jq + q;
          if (j < ncol) {
            const double2 v = ((const double2*)noise)[(size_t)j * nalm + idx];
            re[q] = (T)v.x;
            im[q] = m == 0 ? (T)0 : (T)v.y;
          }
        }
      } else {
        // the FP64 form draws in FP64; the FP32 form through the FP32 Box-Muller of the mixed
        // forms (the FP64 pipe of this part is far too slow for a transcendental per draw)
        uint64_t w[4];
        noise_words(seed, real, idx, jq, w);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if (sizeof(T) == sizeof(double)) {
            const double2 g = noise_value(box_muller(w[q]), m);
            re[q] = (T)g.x;
            im[q] = (T)g.y;
          } else {
            const float2 g = noise_value_f32(box_muller_f32(w[q]), m);
            re[q] = (T)g.x;
            im[q] = (T)g.y;
          }
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = 4 * jq + q;
      if (j < ncol) {
        P[(size_t)j * ldp + 2 * ml] = re[q];
        P[(size_t)j * ldp + 2 * ml + 1] = im[q];
      }
    }
  }
  __syncthreads();
  // a^X_L = sum_j v^X_l[j] n_j (FP64), a warp per order
  for (int ml = warp; ml < nm; ml += kThreads / 32) {
    double tr = 0.0, ti = 0.0, er = 0.0, ei = 0.0;
    for (int j = lane; j < ncol; j += 32) {
      const double nx = (double)P[(size_t)j * ldp + 2 * ml], ny = (double)P[(size_t)j * ldp + 2 * ml + 1];
      tr += vs[j] * nx;
      ti += vs[j] * ny;
      er += vs[ncol + j] * nx;
      ei += vs[ncol + j] * ny;
    }
    for (int o = 16; o; o >>= 1) {
      tr += __shfl_xor_sync(0xffffffffu, tr, o);
      ti += __shfl_xor_sync(0xffffffffu, ti, o);
      er += __shfl_xor_sync(0xffffffffu, er, o);
      ei += __shfl_xor_sync(0xffffffffu, ei, o);
    }
    if (lane == 0) {
      const int64_t idx = alm_idx(l, m0 + ml, L);
      ((double2*)aLT)[idx] = make_double2(tr, ti);
      ((double2*)aLE)[idx] = make_double2(er, ei);
    }
  }
  // Phi_L: rows i = rg + 32 r, columns 8 cg .. 8 cg + 7; the row of largest i bounds j
  const int cg = threadIdx.x & 7, rg = threadIdx.x >> 3;
  T acc[ROWS][8];
#pragma unroll
  for (int r = 0; r < ROWS; ++r)
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[r][q] = (T)0;
  const int jend = min(ncol, j0 + rg + 32 * (ROWS - 1) + 1);
  for (int j = 0; j < jend; ++j) {
    T kv[ROWS];
#pragma unroll
    for (int r = 0; r < ROWS; ++r) kv[r] = rg + 32 * r < nr ? Ks[(rg + 32 * r) * ldk + j] : (T)0;
    T pv[8];
    {
      const T* src = P + (size_t)j * ldp + 8 * cg;  // 8 consecutive values of a 16-byte aligned row
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
    const int i = rg + 32 * r;
    if (i >= nr) continue;
#pragma unroll
    for (int q = 0; q < 8; q += 2) {
      const int ml = (8 * cg + q) >> 1;
      if (ml >= nm) continue;
      const int m = m0 + ml;
      const int64_t row = row0[2 * m + ((l - m) & 1)] + ((l - m) >> 1);
      phi[row * C + 2 * i] = acc[r][q];
      phi[row * C + 2 * i + 1] = acc[r][q + 1];
      if (phi_api) {
        double* o = phi_api + ((size_t)alm_idx(l, m, L) * nr + i) * 2;
        o[0] = (double)acc[r][q];
        o[1] = (double)acc[r][q + 1];
      }
    }
  }
}

// ---------------------------------------------------------------------------------------
// Grouped SIMT GEMMs.  128 x 64 output tile (kSimtBM x kSimtBN), 8-deep k steps, 8 x 4 outputs
// per thread; the next step's operands are loaded into registers while the current one is
// multiplied out of shared memory.  A tile's k loop starts at its q0 (see Tile).
// ---------------------------------------------------------------------------------------
constexpr int BM = kSimtBM, BN = kSimtBN, BK = kSimtBK;
static_assert(BM == 128 && BN == 64 && BK == 8 && kThreads == 256, "the thread layout below");

// out[r][c] += sum_kk As[kk][r] Bs[kk][c] over one step, thread (tx, ty): rows 8 ty .. 8 ty + 7,
// columns 4 tx .. 4 tx + 3 (16-byte aligned rows of the staged tiles)
template <typename T>
__device__ __forceinline__ void simt_step(const T (*As)[BM + 4], const T (*Bs)[BN + 4], int tx, int ty,
                                          T (&acc)[8][4]) {
#pragma unroll
  for (int kk = 0; kk < BK; ++kk) {
    T a[8], b[4];
    if constexpr (sizeof(T) == 4) {
      const float4 a0 = *(const float4*)&As[kk][8 * ty], a1 = *(const float4*)&As[kk][8 * ty + 4];
      const float4 b0 = *(const float4*)&Bs[kk][4 * tx];
      a[0] = a0.x, a[1] = a0.y, a[2] = a0.z, a[3] = a0.w, a[4] = a1.x, a[5] = a1.y, a[6] = a1.z, a[7] = a1.w;
      b[0] = b0.x, b[1] = b0.y, b[2] = b0.z, b[3] = b0.w;
    } else {
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const double2 u = *(const double2*)&As[kk][8 * ty + 2 * h];
        a[2 * h] = u.x, a[2 * h + 1] = u.y;
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const double2 u = *(const double2*)&Bs[kk][4 * tx + 2 * h];
        b[2 * h] = u.x, b[2 * h + 1] = u.y;
      }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
  }
}

// F[mp][jp][c] = sum_k Lambda[mp][jp][k] Phi[mp][k][c]   (rows jp, columns c, depth k)
template <typename T>
__global__ void __launch_bounds__(kThreads) k_synth_gemm(const Tile* __restrict__ tiles,
                                                         const int* __restrict__ K,
                                                         const int64_t* __restrict__ lam0,
                                                         const int64_t* __restrict__ row0,
                                                         const T* __restrict__ lam, const T* __restrict__ phi,
                                                         T* __restrict__ F, int npairs, int C) {
  __shared__ __align__(16) T As[BK][BM + 4];
  __shared__ __align__(16) T Bs[BK][BN + 4];
  const Tile t = tiles[blockIdx.x];
  const int mp = t.mp, j0 = t.rt * BM, c0 = t.ct * BN;
  const int KP = (K[mp] + 15) / 16 * 16;
  const T* A = lam + lam0[mp];
  const T* B = phi + row0[mp] * C;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  // loaders: A rows (2 threads a row, 4 consecutive k each), B 2 entries a thread
  const int ar = threadIdx.x >> 1, ak = (threadIdx.x & 1) * 4;
  const bool arow = j0 + ar < npairs;
  T ra[4], rb[2];
  auto load = [&](int k0) {
#pragma unroll
    for (int i = 0; i < 4; ++i) ra[i] = arow ? A[(int64_t)(j0 + ar) * KP + k0 + ak + i] : (T)0;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int e = threadIdx.x + kThreads * i, kk = e >> 6, cc = e & 63;
      rb[i] = c0 + cc < C ? B[(int64_t)(k0 + kk) * C + c0 + cc] : (T)0;
    }
  };
  T acc[8][4] = {};
  if (t.q0 < KP) load(t.q0);
  for (int k0 = t.q0; k0 < KP; k0 += BK) {
    __syncthreads();  // the previous step's tiles are consumed
#pragma unroll
    for (int i = 0; i < 4; ++i) As[ak + i][ar] = ra[i];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int e = threadIdx.x + kThreads * i;
      Bs[e >> 6][e & 63] = rb[i];
    }
    __syncthreads();
    if (k0 + BK < KP) load(k0 + BK);
    simt_step<T>(As, Bs, tx, ty, acc);
  }
  T* out = F + (int64_t)mp * npairs * C;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int r = j0 + 8 * ty + i;
    if (r >= npairs) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = c0 + 4 * tx + j;
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
  __shared__ __align__(16) T As[BK][BM + 4];
  __shared__ __align__(16) T Bs[BK][BN + 4];
  const Tile t = tiles[blockIdx.x];
  const int mp = t.mp, k0 = t.rt * BM, c0 = t.ct * BN;
  const int Km = K[mp];
  const int KP = (Km + 15) / 16 * 16;
  const T* A = lam + lam0[mp];
  const T* B = G + (int64_t)mp * npairs * C;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  // loaders: A a ring pair's 128 degrees per 32 threads (4 each), B 2 entries a thread
  const int aq = threadIdx.x >> 5, ar = threadIdx.x & 31;
  T ra[4], rb[2];
  auto load = [&](int q0) {
    const bool qv = q0 + aq < npairs;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = ar + 32 * i;
      ra[i] = qv && k0 + r < KP ? A[(int64_t)(q0 + aq) * KP + k0 + r] : (T)0;
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int e = threadIdx.x + kThreads * i, kk = e >> 6, cc = e & 63;
      rb[i] = q0 + kk < npairs && c0 + cc < C ? B[(int64_t)(q0 + kk) * C + c0 + cc] : (T)0;
    }
  };
  T acc[8][4] = {};
  if (t.q0 < npairs) load(t.q0);
  for (int q0 = t.q0; q0 < npairs; q0 += BK) {
    __syncthreads();  // the previous step's tiles are consumed
#pragma unroll
    for (int i = 0; i < 4; ++i) As[aq][ar + 32 * i] = ra[i];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int e = threadIdx.x + kThreads * i;
      Bs[e >> 6][e & 63] = rb[i];
    }
    __syncthreads();
    if (q0 + BK < npairs) load(q0 + BK);
    simt_step<T>(As, Bs, tx, ty, acc);
  }
  T* out = phi + row0[mp] * C;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int r = k0 + 8 * ty + i;
    if (r >= Km) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = c0 + 4 * tx + j;
      if (c < C) out[(int64_t)r * C + c] = acc[i][j];
    }
  }
}

// The FP64 form's SIMT GEMMs: 64 x 64 output tiles, 16-deep k slices, 4 x 4 outputs per thread.
// The FP64 pipe bounds them, and the 128-row tiles' padding (a 385-ring-pair grid fills four
// of them) cost it more than their reuse saved: 57.5 against 51.9 ms per realisation at l_max
// 512 in FP64.
constexpr int BM64 = kSimtBM64, BN64 = 64, BK64 = 16;

// F[mp][jp][c] = sum_k Lambda[mp][jp][k] Phi[mp][k][c]   (rows jp, columns c, depth k)
template <typename T>
__global__ void __launch_bounds__(kThreads) k_synth_gemm64(const Tile* __restrict__ tiles,
                                                         const int* __restrict__ K,
                                                         const int64_t* __restrict__ lam0,
                                                         const int64_t* __restrict__ row0,
                                                         const T* __restrict__ lam, const T* __restrict__ phi,
                                                         T* __restrict__ F, int npairs, int C) {
  __shared__ T As[BK64][BM64 + 1];
  __shared__ T Bs[BK64][BN64 + 1];
  const Tile t = tiles[blockIdx.x];
  const int mp = t.mp, j0 = t.rt * BM64, c0 = t.ct * BN64;
  const int KP = (K[mp] + 15) / 16 * 16;
  const T* A = lam + lam0[mp];
  const T* B = phi + row0[mp] * C;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T acc[4][4] = {};
  for (int k0 = t.q0; k0 < KP; k0 += BK64) {
    for (int e = threadIdx.x; e < BM64 * BK64; e += kThreads) {
      const int r = e >> 4, kk = e & 15;
      As[kk][r] = (j0 + r < npairs) ? A[(int64_t)(j0 + r) * KP + k0 + kk] : (T)0;
    }
    for (int e = threadIdx.x; e < BN64 * BK64; e += kThreads) {
      const int kk = e >> 6, cc = e & 63;
      Bs[kk][cc] = (c0 + cc < C) ? B[(int64_t)(k0 + kk) * C + c0 + cc] : (T)0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK64; ++kk) {
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
__global__ void __launch_bounds__(kThreads) k_analysis_gemm64(const Tile* __restrict__ tiles,
                                                            const int* __restrict__ K,
                                                            const int64_t* __restrict__ lam0,
                                                            const int64_t* __restrict__ row0,
                                                            const T* __restrict__ lam, const T* __restrict__ G,
                                                            T* __restrict__ phi, int npairs, int C) {
  __shared__ T As[BK64][BM64 + 1];
  __shared__ T Bs[BK64][BN64 + 1];
  const Tile t = tiles[blockIdx.x];
  const int mp = t.mp, k0 = t.rt * BM64, c0 = t.ct * BN64;
  const int Km = K[mp];
  const int KP = (Km + 15) / 16 * 16;
  const T* A = lam + lam0[mp];
  const T* B = G + (int64_t)mp * npairs * C;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T acc[4][4] = {};
  for (int q0 = t.q0; q0 < npairs; q0 += BK64) {
    for (int e = threadIdx.x; e < BM64 * BK64; e += kThreads) {
      const int kk = e >> 6, r = e & 63;
      As[kk][r] = (q0 + kk < npairs && k0 + r < KP) ? A[(int64_t)(q0 + kk) * KP + k0 + r] : (T)0;
    }
    for (int e = threadIdx.x; e < BN64 * BK64; e += kThreads) {
      const int kk = e >> 6, cc = e & 63;
      Bs[kk][cc] = (q0 + kk < npairs && c0 + cc < C) ? B[(int64_t)(q0 + kk) * C + c0 + cc] : (T)0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK64; ++kk) {
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
  const size_t smem = filter_smem<T>(nr, ncol);
  const dim3 grid(sh->lmax + 1, (sh->lmax + kFlM) / kFlM);  // (degree, order tile); tiles past l exit
  auto run = [&](auto kern) {
    FNL_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<grid, kThreads, smem, st>>>(sh->lmax, nr, sh->j0, ncol, (const T*)sh->d_Kf, sh->d_vT, sh->d_vE, seed,
                                       real, noise, sh->d_row0, (T*)sh->d_phi, phi_api, aLT, aLE);
  };
  switch ((nr + 31) / 32) {
    case 1: run(k_filter<T, 1>); break;
    case 2: run(k_filter<T, 2>); break;
    case 3: run(k_filter<T, 3>); break;
    case kFlMaxRows: run(k_filter<T, kFlMaxRows>); break;
    default: throw Error(FNL_EUNSUPPORTED, "the filter takes at most 128 shells");
  }
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
    k_synth_gemm64<double><<<sh->n_tiles_syn, kThreads, 0, st>>>(sh->d_tiles_syn, sh->d_K, sh->d_lam0, sh->d_row0,
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
    k_synth_gemm64<double><<<sh->n_tiles_syn, kThreads, 0, st>>>(sh->d_tiles_syn, sh->d_K, sh->d_lam0, sh->d_row0,
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
    k_analysis_gemm64<double><<<sh->n_tiles_ana, kThreads, 0, st>>>(
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
