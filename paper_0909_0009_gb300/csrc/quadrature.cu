// Optimal radial quadrature (Sect. 3) on the device, FP64 throughout.
//
// For each degree l and field X the line-of-sight integral I = int dr r^2 alpha^X_l Phi is taken
// on a fine grid of N_tot shells, I = q . Phi (q_k = w_k r_k^2 alpha^X_l(r_k)), and approximated by
// I^ = sum_{i in S} w_i Phi(r_i) on N of those nodes.  With P_l the covariance of Phi on the fine
// grid (Eq. 7 plus the filters' relative jitter), c = P_l q and <I^2> = q . c:
//   <(I^ - I)^2> = <I^2> - 2 w . c_S + w^T P_SS w,  minimal for P_SS w = c_S, where it is
//   <I^2> - c_S^T P_SS^-1 c_S (the paper writes both through the eigenpairs of P_l).
// The greedy of the paper adds, one node at a time, the fine node that lowers the summed relative
// error sum_{l, X} err / <I^2> most.  Adding node j to S lowers err^X_l by (e^X_lj)^2 / d_lj, where
// d_lj = P_jj - P_jS P_SS^-1 P_Sj (conditional variance of Phi(r_j) given Phi_S) and
// e^X_lj = c_j - P_jS P_SS^-1 c_S (its conditional covariance with I^X).  Both are kept for every
// candidate and updated per step with one column of the pivoted Cholesky factor of P_l:
//   v = (P_l[:, j] - sum_{t < s} L_t L_t[j]) / sqrt(d_j),  d -= v^2,  e^X -= v z^X,
//   z^X_s = e^X_j / sqrt(d_j),  err^X -= (z^X_s)^2,
// so a step costs O(N_tot s) per degree instead of a solve per candidate.  The weights of the
// final S follow from L_SS^T w = z (back substitution).
//
// Kernels: k_bessel (j_l(k r) for all l by Miller's downward recurrence with normalisation
// sum (2l+1) j_l^2 = 1, or the upward recurrence where x > l_max + 60), k_cov_syrk (C_l +=
// J_l^T diag(p) J_l per chunk of k, 32 x 32 tiles, lower half), k_cov_finish (jitter, symmetric
// P, c = P q, <I^2>), then per step k_quad_score (one block per candidate, over l), k_quad_pick
// (argmax, smallest index on ties), k_quad_update (one block per l), k_quad_objective; finally
// k_quad_weights and k_quad_rule_error (the error of any given rule).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "fnl_internal.cuh"

struct fnl_quad {
  int device = 0, L = 0, nt = 0;
  double* d_P = nullptr;   // [L+1][nt][nt]
  double* d_q = nullptr;   // [2][L+1][nt]
  double* d_c = nullptr;   // [2][L+1][nt]  P q
  double* d_I2 = nullptr;  // [2][L+1]
  double cov_seconds = 0.0;
  std::vector<void*> allocations;
};

namespace fnl {

namespace {

template <typename T>
T* qalloc(fnl_quad* k, size_t n) {
  void* p = nullptr;
  FNL_CUDA(cudaMalloc(&p, sizeof(T) * (n ? n : 1)));
  k->allocations.push_back(p);
  return (T*)p;
}

// j_l(k_q r_i) for l = 0..L into J[l][q][i] (stride kc * nt between degrees); E is scratch for
// the binary exponents of the downward recurrence.
__global__ void k_bessel(int L, int nt, int kc, const double* __restrict__ kv, const double* __restrict__ r,
                         double* __restrict__ J, int* __restrict__ E) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= kc * nt) return;
  const int q = t / nt, i = t - q * nt;
  const size_t stride = (size_t)kc * nt, base = (size_t)q * nt + i;
  const double x = kv[q] * r[i];
  const double s = sin(x), c = cos(x);
  const double j0 = s / x, j1 = s / (x * x) - c / x;
  const double ix = 1.0 / x;
  if (x > L + 60.0) {
    J[base] = j0;
    if (L >= 1) J[stride + base] = j1;
    double a = j0, b = j1;
    for (int l = 1; l < L; ++l) {
      const double nb = (2.0 * l + 1.0) * ix * b - a;
      a = b;
      b = nb;
      J[(size_t)(l + 1) * stride + base] = b;
    }
    return;
  }
  const int N = L + 200 + (int)x;
  double yn = 0.0, y = 1.0, sum = 0.0;
  int e = 0;
  for (int l = N; l >= 1; --l) {
    if (l <= L) {
      J[(size_t)l * stride + base] = y;
      E[(size_t)l * stride + base] = e;
    }
    sum += (2.0 * l + 1.0) * y * y;
    const double yp = (2.0 * l + 1.0) * ix * y - yn;
    yn = y;
    y = yp;
    if (fabs(y) > 0x1p400) {
      y *= 0x1p-400;
      yn *= 0x1p-400;
      sum *= 0x1p-800;
      e += 400;
    }
  }
  J[base] = y;
  E[base] = e;
  sum += y * y;
  const double norm = 1.0 / sqrt(sum);
  double ref_true, ref_num;
  if (fabs(j0) > 0.1 * fabs(j1) || L < 1) {
    ref_true = j0;
    ref_num = y * norm;
  } else {
    ref_true = j1;
    ref_num = ldexp(J[stride + base] * norm, E[stride + base] - e);
  }
  const double sign = ((ref_true >= 0) == (ref_num >= 0)) ? 1.0 : -1.0;
  for (int l = 0; l <= L; ++l) {
    const size_t o = (size_t)l * stride + base;
    const double v = sign * ldexp(J[o] * norm, E[o] - e);
    J[o] = fabs(v) < 1e-290 ? 0.0 : v;
  }
}

// C[l][i][j] += sum_q p_q J[l][q][i] J[l][q][j] for the lower tiles (ti >= tj) of 32 x 32.
__global__ void __launch_bounds__(256) k_cov_syrk(int nt, int kc, const double* __restrict__ J,
                                                  const double* __restrict__ pk, double* __restrict__ C) {
  __shared__ double A[16][33], B[16][33];
  const int t = blockIdx.x, l = blockIdx.y;
  int ti = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
  while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
  while (ti * (ti + 1) / 2 > t) --ti;
  const int tj = t - ti * (ti + 1) / 2;
  const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
  const double* Jl = J + (size_t)l * kc * nt;
  double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
  for (int q0 = 0; q0 < kc; q0 += 16) {
    for (int e = threadIdx.x; e < 16 * 32; e += blockDim.x) {
      const int qq = e / 32, ii = e % 32, q = q0 + qq;
      const int gi = ti * 32 + ii, gj = tj * 32 + ii;
      const bool ok = q < kc;
      A[qq][ii] = (ok && gi < nt) ? Jl[(size_t)q * nt + gi] * pk[q] : 0.0;
      B[qq][ii] = (ok && gj < nt) ? Jl[(size_t)q * nt + gj] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int qq = 0; qq < 16; ++qq) {
      const double a0 = A[qq][2 * ty], a1 = A[qq][2 * ty + 1], b0 = B[qq][2 * tx], b1 = B[qq][2 * tx + 1];
      acc[0][0] += a0 * b0;
      acc[0][1] += a0 * b1;
      acc[1][0] += a1 * b0;
      acc[1][1] += a1 * b1;
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int i = ti * 32 + 2 * ty + a, j = tj * 32 + 2 * tx + b;
      if (i < nt && j < nt && j <= i) C[((size_t)l * nt + i) * nt + j] += acc[a][b];
    }
}

// Per degree: eps_l = jitter_rel * mean(diag C_l); P = C + eps I, both halves; c^X = P q^X and
// <I^2>^X = q^X . c^X (fixed-order block sums).
__global__ void __launch_bounds__(256) k_cov_finish(int nt, int L1, double jitter_rel, const double* __restrict__ C,
                                                    double* __restrict__ P, const double* __restrict__ q,
                                                    double* __restrict__ c, double* __restrict__ I2) {
  __shared__ double red[256];
  const int l = blockIdx.x;
  const double* Cl = C + (size_t)l * nt * nt;
  double* Pl = P + (size_t)l * nt * nt;
  double t = 0.0;
  for (int i = threadIdx.x; i < nt; i += blockDim.x) t += Cl[(size_t)i * nt + i];
  red[threadIdx.x] = t;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  const double eps = jitter_rel * red[0] / nt;
  __syncthreads();
  for (size_t e = threadIdx.x; e < (size_t)nt * nt; e += blockDim.x) {
    const int i = (int)(e / nt), j = (int)(e % nt);
    Pl[e] = (j <= i ? Cl[(size_t)i * nt + j] : Cl[(size_t)j * nt + i]) + (i == j ? eps : 0.0);
  }
  __syncthreads();
  for (int x = 0; x < 2; ++x) {
    const double* ql = q + ((size_t)x * L1 + l) * nt;
    double* cl = c + ((size_t)x * L1 + l) * nt;
    double s2 = 0.0;
    for (int i = threadIdx.x; i < nt; i += blockDim.x) {
      double s = 0.0;
      for (int k = 0; k < nt; ++k) s += Pl[(size_t)i * nt + k] * ql[k];
      cl[i] = s;
      s2 += ql[i] * s;
    }
    red[threadIdx.x] = s2;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
      if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) I2[(size_t)x * L1 + l] = red[0];
    __syncthreads();
  }
}

// Greedy state: d [L1][nt], e [2][L1][nt], err [2][L1], Lf [nsel][L1][nt], z [2][L1][nsel].
__global__ void __launch_bounds__(256) k_quad_init(int nt, int L1, const double* __restrict__ P,
                                                   const double* __restrict__ c, const double* __restrict__ I2,
                                                   double* __restrict__ d, double* __restrict__ e,
                                                   double* __restrict__ err) {
  const int l = blockIdx.x;
  for (int j = threadIdx.x; j < nt; j += blockDim.x) {
    d[(size_t)l * nt + j] = P[((size_t)l * nt + j) * nt + j];
    for (int x = 0; x < 2; ++x) e[((size_t)x * L1 + l) * nt + j] = c[((size_t)x * L1 + l) * nt + j];
  }
  if (threadIdx.x < 2) err[(size_t)threadIdx.x * L1 + l] = I2[(size_t)threadIdx.x * L1 + l];
}

// score[j] = sum_{l, X: <I^2> > 0} (e^X_lj)^2 / d_lj / <I^2>^X_l; -1 for a selected node.
__global__ void __launch_bounds__(256) k_quad_score(int nt, int L1, const double* __restrict__ d,
                                                    const double* __restrict__ e, const double* __restrict__ I2,
                                                    const int* __restrict__ selected, double* __restrict__ score) {
  __shared__ double red[256];
  const int j = blockIdx.x;
  double s = 0.0;
  for (int l = threadIdx.x; l < L1; l += blockDim.x) {
    const double dj = d[(size_t)l * nt + j];
    if (!(dj > 0.0)) continue;
    for (int x = 0; x < 2; ++x) {
      const double i2 = I2[(size_t)x * L1 + l];
      if (i2 > 0.0) {
        const double ej = e[((size_t)x * L1 + l) * nt + j];
        s += ej * ej / dj / i2;
      }
    }
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) score[j] = selected[j] ? -1.0 : red[0];
}

// nodes[s] = argmax_j score[j] (smallest j on ties), marked selected.
__global__ void __launch_bounds__(256) k_quad_pick(int nt, int s, const double* __restrict__ score,
                                                   int* __restrict__ selected, int* __restrict__ nodes) {
  __shared__ double bv[256];
  __shared__ int bj[256];
  double best = -2.0;
  int bi = nt;
  for (int j = threadIdx.x; j < nt; j += blockDim.x)
    if (score[j] > best) {
      best = score[j];
      bi = j;
    }
  bv[threadIdx.x] = best;
  bj[threadIdx.x] = bi;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      const double v2 = bv[threadIdx.x + o];
      const int j2 = bj[threadIdx.x + o];
      if (v2 > bv[threadIdx.x] || (v2 == bv[threadIdx.x] && j2 < bj[threadIdx.x])) {
        bv[threadIdx.x] = v2;
        bj[threadIdx.x] = j2;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    nodes[s] = bj[0];
    selected[bj[0]] = 1;
  }
}

// Column s of the pivoted Cholesky factor of P_l at the picked node, and the updates of d, e, err.
__global__ void __launch_bounds__(512) k_quad_update(int nt, int L1, int s, const double* __restrict__ P,
                                                     const int* __restrict__ nodes, double* __restrict__ Lf,
                                                     double* __restrict__ d, double* __restrict__ e,
                                                     double* __restrict__ err, double* __restrict__ z, int nsel) {
  extern __shared__ double lj[];  // [s]: L_t[j] for t < s
  __shared__ double zz[2];
  const int l = blockIdx.x;
  const int j = nodes[s];
  for (int t = threadIdx.x; t < s; t += blockDim.x) lj[t] = Lf[((size_t)t * L1 + l) * nt + j];
  const double dj = d[(size_t)l * nt + j];
  const double sq = sqrt(dj);
  __syncthreads();
  if (threadIdx.x < 2) {
    const int x = threadIdx.x;
    const double zx = e[((size_t)x * L1 + l) * nt + j] / sq;
    zz[x] = zx;
    z[((size_t)x * L1 + l) * nsel + s] = zx;
  }
  __syncthreads();
  const double* Pl = P + (size_t)l * nt * nt;
  for (int k = threadIdx.x; k < nt; k += blockDim.x) {
    double v = Pl[(size_t)j * nt + k];
    for (int t = 0; t < s; ++t) v -= Lf[((size_t)t * L1 + l) * nt + k] * lj[t];
    v /= sq;
    Lf[((size_t)s * L1 + l) * nt + k] = v;
    d[(size_t)l * nt + k] -= v * v;
    for (int x = 0; x < 2; ++x) e[((size_t)x * L1 + l) * nt + k] -= v * zz[x];
  }
  if (threadIdx.x < 2) err[(size_t)threadIdx.x * L1 + l] -= zz[threadIdx.x] * zz[threadIdx.x];
}

// objective[s] = sum_{l, X: <I^2> > 0} err^X_l / <I^2>^X_l (one block, fixed order).
__global__ void __launch_bounds__(256) k_quad_objective(int L1, int s, const double* __restrict__ err,
                                                        const double* __restrict__ I2, double* __restrict__ obj) {
  __shared__ double red[256];
  double t = 0.0;
  for (int i = threadIdx.x; i < 2 * L1; i += blockDim.x)
    if (I2[i] > 0.0) t += err[i] / I2[i];
  red[threadIdx.x] = t;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) obj[s] = red[0];
}

// w^X_l from L_SS^T w = z^X_l, L_SS[s][t] = Lf[t][l][nodes[s]]: one warp per (l, X).
__global__ void __launch_bounds__(64) k_quad_weights(int nt, int L1, int n, const double* __restrict__ Lf,
                                                     const int* __restrict__ nodes, const double* __restrict__ z,
                                                     const double* __restrict__ I2, double* __restrict__ w) {
  const int l = blockIdx.x, x = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double* wl = w + ((size_t)x * L1 + l) * n;
  const double* zl = z + ((size_t)x * L1 + l) * n;
  const bool live = I2[(size_t)x * L1 + l] > 0.0;
  for (int s = n - 1; s >= 0; --s) {
    double acc = 0.0;
    for (int s2 = s + 1 + lane; s2 < n; s2 += 32) acc += Lf[((size_t)s * L1 + l) * nt + nodes[s2]] * wl[s2];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) wl[s] = live ? (zl[s] - acc) / Lf[((size_t)s * L1 + l) * nt + nodes[s]] : 0.0;
    __syncwarp();
  }
}

// err^X_l = <I^2> - 2 w.c_S + w^T P_SS w of a given rule (nodes, w [2][L1][n]), relative to <I^2>.
__global__ void __launch_bounds__(256) k_quad_rule_error(int nt, int L1, int n, const double* __restrict__ P,
                                                         const double* __restrict__ c, const double* __restrict__ I2,
                                                         const int* __restrict__ nodes, const double* __restrict__ w,
                                                         double* __restrict__ rel) {
  __shared__ double red[256];
  const int l = blockIdx.x;
  const double* Pl = P + (size_t)l * nt * nt;
  for (int x = 0; x < 2; ++x) {
    const double* wl = w + ((size_t)x * L1 + l) * n;
    const double* cl = c + ((size_t)x * L1 + l) * nt;
    double t = 0.0;
    for (int a = threadIdx.x; a < n; a += blockDim.x) {
      double pw = 0.0;
      for (int b = 0; b < n; ++b) pw += Pl[(size_t)nodes[a] * nt + nodes[b]] * wl[b];
      t += wl[a] * (pw - 2.0 * cl[nodes[a]]);
    }
    red[threadIdx.x] = t;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
      if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      const double i2 = I2[(size_t)x * L1 + l];
      rel[(size_t)x * L1 + l] = i2 > 0.0 ? (i2 + red[0]) / i2 : 0.0;
    }
    __syncthreads();
  }
}

void free_quad(fnl_quad* k) {
  if (!k) return;
  for (void* p : k->allocations) cudaFree(p);
  delete k;
}

double seconds_since(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

}  // namespace fnl

using namespace fnl;

extern "C" {

fnl_status fnl_quad_create(const fnl_quad_desc* d, int device, fnl_quad** out) {
  fnl_quad* k = nullptr;
  fnl_status st = guard([&] {
    FNL_REQUIRE(out && d, "arguments must not be NULL");
    *out = nullptr;
    FNL_REQUIRE(d->lmax >= 0 && d->lmax <= 4096, "lmax must be in [0, 4096]");
    FNL_REQUIRE(d->ntot >= 1 && d->ntot <= 4096, "ntot must be in [1, 4096]");
    FNL_REQUIRE(d->r && d->w && d->alphaT && d->alphaE, "r, w, alphaT and alphaE must not be NULL");
    if (!d->P) {
      FNL_REQUIRE(d->nk >= 2 && d->kmin > 0 && d->kmax > d->kmin && d->A > 0, "bad covariance parameters");
      for (int i = 0; i < d->ntot; ++i) FNL_REQUIRE(d->r[i] > 0, "r_i must be > 0");
    }
    FNL_REQUIRE(d->jitter_rel >= 0, "jitter_rel must be >= 0");
    int ndev = 0;
    FNL_CUDA(cudaGetDeviceCount(&ndev));
    FNL_REQUIRE(device >= 0 && device < ndev, "no such CUDA device");
    DeviceScope scope(device);
    k = new fnl_quad;
    k->device = device;
    k->L = d->lmax;
    k->nt = d->ntot;
    const int L1 = d->lmax + 1, nt = d->ntot;
    const auto t0 = std::chrono::steady_clock::now();
    std::vector<double> q(2 * (size_t)L1 * nt);
    for (int l = 0; l < L1; ++l)
      for (int i = 0; i < nt; ++i) {
        const double u = d->w[i] * d->r[i] * d->r[i];
        q[(size_t)l * nt + i] = u * d->alphaT[(size_t)l * nt + i];
        q[((size_t)L1 + l) * nt + i] = u * d->alphaE[(size_t)l * nt + i];
      }
    k->d_P = qalloc<double>(k, (size_t)L1 * nt * nt);
    k->d_q = qalloc<double>(k, q.size());
    k->d_c = qalloc<double>(k, q.size());
    k->d_I2 = qalloc<double>(k, 2 * (size_t)L1);
    FNL_CUDA(cudaMemcpy(k->d_q, q.data(), sizeof(double) * q.size(), cudaMemcpyHostToDevice));
    double* d_C = nullptr;
    double *d_J = nullptr, *d_k = nullptr, *d_p = nullptr, *d_r = nullptr;
    int* d_E = nullptr;
    auto release = [&] {
      cudaFree(d_C);
      cudaFree(d_J);
      cudaFree(d_k);
      cudaFree(d_p);
      cudaFree(d_r);
      cudaFree(d_E);
    };
    try {
      FNL_CUDA(cudaMalloc(&d_C, sizeof(double) * (size_t)L1 * nt * nt));
      if (d->P) {
        FNL_CUDA(cudaMemcpy(d_C, d->P, sizeof(double) * (size_t)L1 * nt * nt, cudaMemcpyHostToDevice));
      } else {
        // C_l = (2/pi) sum_k wk k^2 A k^(ns-4) j_l(k r_i) j_l(k r_j), trapezoid rule in k
        FNL_CUDA(cudaMemset(d_C, 0, sizeof(double) * (size_t)L1 * nt * nt));
        const double h = (d->kmax - d->kmin) / (d->nk - 1);
        const int KC = (int)std::max<int64_t>(16, std::min<int64_t>(512, (int64_t)(1u << 28) / ((int64_t)L1 * nt)));
        FNL_CUDA(cudaMalloc(&d_J, sizeof(double) * (size_t)L1 * KC * nt));
        FNL_CUDA(cudaMalloc(&d_E, sizeof(int) * (size_t)L1 * KC * nt));
        FNL_CUDA(cudaMalloc(&d_k, sizeof(double) * KC));
        FNL_CUDA(cudaMalloc(&d_p, sizeof(double) * KC));
        FNL_CUDA(cudaMalloc(&d_r, sizeof(double) * nt));
        FNL_CUDA(cudaMemcpy(d_r, d->r, sizeof(double) * nt, cudaMemcpyHostToDevice));
        std::vector<double> kv(KC), pk(KC);
        const int ntile = (nt + 31) / 32;
        for (int k0 = 0; k0 < d->nk; k0 += KC) {
          const int kc = std::min(KC, d->nk - k0);
          for (int qq = 0; qq < kc; ++qq) {
            const int kk = k0 + qq;
            const double kval = (kk == d->nk - 1) ? d->kmax : d->kmin + kk * h;
            const double wk = (kk == 0 || kk == d->nk - 1) ? 0.5 * h : h;
            kv[qq] = kval;
            pk[qq] = (2.0 / M_PI) * wk * kval * kval * d->A * std::pow(kval, d->ns - 4.0);
          }
          FNL_CUDA(cudaMemcpy(d_k, kv.data(), sizeof(double) * kc, cudaMemcpyHostToDevice));
          FNL_CUDA(cudaMemcpy(d_p, pk.data(), sizeof(double) * kc, cudaMemcpyHostToDevice));
          k_bessel<<<(kc * nt + 127) / 128, 128>>>(d->lmax, nt, kc, d_k, d_r, d_J, d_E);
          FNL_CUDA(cudaGetLastError());
          k_cov_syrk<<<dim3(ntile * (ntile + 1) / 2, L1), 256>>>(nt, kc, d_J, d_p, d_C);
          FNL_CUDA(cudaGetLastError());
        }
      }
      k_cov_finish<<<L1, 256>>>(nt, L1, d->jitter_rel, d_C, k->d_P, k->d_q, k->d_c, k->d_I2);
      FNL_CUDA(cudaGetLastError());
      FNL_CUDA(cudaDeviceSynchronize());
    } catch (...) {
      release();
      throw;
    }
    release();
    k->cov_seconds = seconds_since(t0);
    *out = k;
  });
  if (st != FNL_OK && k) free_quad(k);
  return st;
}

void fnl_quad_destroy(fnl_quad* k) {
  if (!k) return;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(k->device);
  cudaDeviceSynchronize();
  free_quad(k);
  if (prev >= 0) cudaSetDevice(prev);
}

fnl_status fnl_quad_moments(const fnl_quad* k, double* I2, double* seconds) {
  return guard([&] {
    FNL_REQUIRE(k, "design object is NULL");
    DeviceScope scope(k->device);
    if (I2) FNL_CUDA(cudaMemcpy(I2, k->d_I2, sizeof(double) * 2 * (k->L + 1), cudaMemcpyDeviceToHost));
    if (seconds) *seconds = k->cov_seconds;
  });
}

}  // extern "C"

namespace fnl {
namespace {

// Pivoted Cholesky steps on every degree: the greedy's picks, or the given nodes when `forced`
// is set; then the optimal weights of the resulting node set.
void run_pivots(const fnl_quad* k, int nsel, const int* forced, int* nodes, double* weights, double* objective,
                double* rel_err) {
  const int L1 = k->L + 1, nt = k->nt;
  double *d_d = nullptr, *d_e = nullptr, *d_err = nullptr, *d_Lf = nullptr, *d_z = nullptr, *d_score = nullptr,
         *d_obj = nullptr, *d_w = nullptr;
  int *d_sel = nullptr, *d_nodes = nullptr;
  auto release = [&] {
    for (void* p : {(void*)d_d, (void*)d_e, (void*)d_err, (void*)d_Lf, (void*)d_z, (void*)d_score, (void*)d_obj,
                    (void*)d_w, (void*)d_sel, (void*)d_nodes})
      cudaFree(p);
  };
  try {
    FNL_CUDA(cudaMalloc(&d_d, sizeof(double) * (size_t)L1 * nt));
    FNL_CUDA(cudaMalloc(&d_e, sizeof(double) * 2 * (size_t)L1 * nt));
    FNL_CUDA(cudaMalloc(&d_err, sizeof(double) * 2 * (size_t)L1));
    FNL_CUDA(cudaMalloc(&d_Lf, sizeof(double) * (size_t)nsel * L1 * nt));
    FNL_CUDA(cudaMalloc(&d_z, sizeof(double) * 2 * (size_t)L1 * nsel));
    FNL_CUDA(cudaMalloc(&d_score, sizeof(double) * nt));
    FNL_CUDA(cudaMalloc(&d_obj, sizeof(double) * nsel));
    FNL_CUDA(cudaMalloc(&d_w, sizeof(double) * 2 * (size_t)L1 * nsel));
    FNL_CUDA(cudaMalloc(&d_sel, sizeof(int) * nt));
    FNL_CUDA(cudaMalloc(&d_nodes, sizeof(int) * nsel));
    FNL_CUDA(cudaMemset(d_sel, 0, sizeof(int) * nt));
    if (forced) FNL_CUDA(cudaMemcpy(d_nodes, forced, sizeof(int) * nsel, cudaMemcpyHostToDevice));
    k_quad_init<<<L1, 256>>>(nt, L1, k->d_P, k->d_c, k->d_I2, d_d, d_e, d_err);
    FNL_CUDA(cudaGetLastError());
    const int ut = std::min(512, (nt + 31) / 32 * 32);
    for (int s = 0; s < nsel; ++s) {
      if (!forced) {
        k_quad_score<<<nt, 256>>>(nt, L1, d_d, d_e, k->d_I2, d_sel, d_score);
        k_quad_pick<<<1, 256>>>(nt, s, d_score, d_sel, d_nodes);
      }
      k_quad_update<<<L1, ut, sizeof(double) * std::max(1, s)>>>(nt, L1, s, k->d_P, d_nodes, d_Lf, d_d, d_e, d_err,
                                                                  d_z, nsel);
      k_quad_objective<<<1, 256>>>(L1, s, d_err, k->d_I2, d_obj);
      FNL_CUDA(cudaGetLastError());
    }
    k_quad_weights<<<L1, 64>>>(nt, L1, nsel, d_Lf, d_nodes, d_z, k->d_I2, d_w);
    FNL_CUDA(cudaGetLastError());
    FNL_CUDA(cudaDeviceSynchronize());
    if (nodes) FNL_CUDA(cudaMemcpy(nodes, d_nodes, sizeof(int) * nsel, cudaMemcpyDeviceToHost));
    if (weights) FNL_CUDA(cudaMemcpy(weights, d_w, sizeof(double) * 2 * (size_t)L1 * nsel, cudaMemcpyDeviceToHost));
    if (objective) FNL_CUDA(cudaMemcpy(objective, d_obj, sizeof(double) * nsel, cudaMemcpyDeviceToHost));
    if (rel_err) {
      std::vector<double> err(2 * (size_t)L1), i2(2 * (size_t)L1);
      FNL_CUDA(cudaMemcpy(err.data(), d_err, sizeof(double) * err.size(), cudaMemcpyDeviceToHost));
      FNL_CUDA(cudaMemcpy(i2.data(), k->d_I2, sizeof(double) * i2.size(), cudaMemcpyDeviceToHost));
      for (size_t i = 0; i < err.size(); ++i) rel_err[i] = i2[i] > 0.0 ? err[i] / i2[i] : 0.0;
    }
  } catch (...) {
    release();
    throw;
  }
  release();
}

}  // namespace
}  // namespace fnl

extern "C" {

fnl_status fnl_quad_greedy(const fnl_quad* k, int nsel, int* nodes, double* weights, double* objective,
                           double* rel_err, double* seconds) {
  return guard([&] {
    FNL_REQUIRE(k, "design object is NULL");
    FNL_REQUIRE(nsel >= 1 && nsel <= k->nt, "nsel must be in [1, ntot]");
    FNL_REQUIRE(nodes, "nodes must not be NULL");
    DeviceScope scope(k->device);
    const auto t0 = std::chrono::steady_clock::now();
    run_pivots(k, nsel, nullptr, nodes, weights, objective, rel_err);
    if (seconds) *seconds = seconds_since(t0);
  });
}

fnl_status fnl_quad_fit(const fnl_quad* k, int n, const int* nodes, double* weights, double* rel_err) {
  return guard([&] {
    FNL_REQUIRE(k, "design object is NULL");
    FNL_REQUIRE(n >= 1 && n <= k->nt && nodes, "bad arguments");
    std::vector<int> seen(k->nt, 0);
    for (int i = 0; i < n; ++i) {
      FNL_REQUIRE(nodes[i] >= 0 && nodes[i] < k->nt, "node index out of range");
      FNL_REQUIRE(!seen[nodes[i]]++, "nodes must be distinct");
    }
    DeviceScope scope(k->device);
    run_pivots(k, n, nodes, nullptr, weights, nullptr, rel_err);
  });
}

fnl_status fnl_quad_error(const fnl_quad* k, int n, const int* nodes, const double* weights, double* rel_err) {
  return guard([&] {
    FNL_REQUIRE(k, "design object is NULL");
    FNL_REQUIRE(n >= 1 && n <= k->nt && nodes && weights && rel_err, "bad arguments");
    for (int i = 0; i < n; ++i) FNL_REQUIRE(nodes[i] >= 0 && nodes[i] < k->nt, "node index out of range");
    DeviceScope scope(k->device);
    const int L1 = k->L + 1;
    int* d_nodes = nullptr;
    double *d_w = nullptr, *d_rel = nullptr;
    auto release = [&] {
      cudaFree(d_nodes);
      cudaFree(d_w);
      cudaFree(d_rel);
    };
    try {
      FNL_CUDA(cudaMalloc(&d_nodes, sizeof(int) * n));
      FNL_CUDA(cudaMalloc(&d_w, sizeof(double) * 2 * (size_t)L1 * n));
      FNL_CUDA(cudaMalloc(&d_rel, sizeof(double) * 2 * (size_t)L1));
      FNL_CUDA(cudaMemcpy(d_nodes, nodes, sizeof(int) * n, cudaMemcpyHostToDevice));
      FNL_CUDA(cudaMemcpy(d_w, weights, sizeof(double) * 2 * (size_t)L1 * n, cudaMemcpyHostToDevice));
      k_quad_rule_error<<<L1, 256>>>(k->nt, L1, n, k->d_P, k->d_c, k->d_I2, d_nodes, d_w, d_rel);
      FNL_CUDA(cudaGetLastError());
      FNL_CUDA(cudaMemcpy(rel_err, d_rel, sizeof(double) * 2 * (size_t)L1, cudaMemcpyDeviceToHost));
    } catch (...) {
      release();
      throw;
    }
    release();
  });
}

}  // extern "C"
