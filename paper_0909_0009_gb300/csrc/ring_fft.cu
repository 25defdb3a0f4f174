// Ring transforms in phi (the DFT half of steps (ii) and (iv)) and the pointwise square
// of step (iii), Eq. 2.  One block per (ring pair jp, shell s).
//
// The two real rings of a pair (north f_N, south f_S) are carried as one complex sequence
// z = f_N + i f_S.  Their spectra F_N,m = E_m + O_m and F_S,m = E_m - O_m come from the
// even/odd Legendre halves; Z_m = F_N,m + i F_S,m and Z_{-m} = conj(F_N,m) + i conj(F_S,m).
//   SQUARE:      z = IDFT(Z); w = (Re z)^2 - mu_s + i ((Im z)^2 - mu_s); W = DFT(w);
//                G_N,m = (W_m + conj W_{-m}) / 2, G_S,m = (W_m - conj W_{-m}) / (2 i), m <= lmax,
//                scaled by (2 pi / nphi) w_jp and stored as S = G_N + G_S (even degrees) and
//                D = G_N - G_S (odd degrees); the equator ring is counted once.
//   SYNTH_MAP:   z = IDFT(Z) written to the two rings of the map.
//   ANALYSE_MAP: W = DFT(f_N + i f_S) from the map, then as SQUARE.
// Transforms are self-sorting mixed-radix (4, 2, 3, 5) Stockham passes between two shared
// memory buffers; twiddles e^{-2 pi i k / nphi} come from a table computed on the host.
#include <cmath>
#include <type_traits>

#include "fnl_internal.cuh"
#include "mixed.cuh"

namespace fnl {

namespace {

template <typename T>
__device__ __forceinline__ cplx<T> cmul(cplx<T> a, cplx<T> b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename T>
__device__ __forceinline__ cplx<T> cadd(cplx<T> a, cplx<T> b) {
  return {a.x + b.x, a.y + b.y};
}
template <typename T>
__device__ __forceinline__ cplx<T> csub(cplx<T> a, cplx<T> b) {
  return {a.x - b.x, a.y - b.y};
}
// i * s * a for s = +-1
template <typename T>
__device__ __forceinline__ cplx<T> imul(cplx<T> a, T s) {
  return {-s * a.y, s * a.x};
}

// In-register DFT of size R: v'[q] = sum_r v[r] e^{sgn 2 pi i q r / R}.
template <typename T>
__device__ __forceinline__ void small_dft(cplx<T>* v, int R, T sgn) {
  if (R == 2) {
    const cplx<T> a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  } else if (R == 4) {
    const cplx<T> s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
    const cplx<T> s13 = cadd(v[1], v[3]), d13 = imul(csub(v[1], v[3]), sgn);
    v[0] = cadd(s02, s13);
    v[1] = cadd(d02, d13);
    v[2] = csub(s02, s13);
    v[3] = csub(d02, d13);
  } else if (R == 3) {
    const T c = (T)-0.5, s = sgn * (T)0.86602540378443864676;  // cos, sin of 2 pi / 3
    const cplx<T> t1 = cadd(v[1], v[2]), t2 = csub(v[1], v[2]);
    const cplx<T> a = {v[0].x + c * t1.x, v[0].y + c * t1.y};
    const cplx<T> b = imul(t2, s);
    v[0] = cadd(v[0], t1);
    v[1] = cadd(a, b);
    v[2] = csub(a, b);
  } else {  // R == 5
    const T c1 = (T)0.30901699437494742410, c2 = (T)-0.80901699437494742410;     // cos 2pi/5, cos 4pi/5
    const T s1 = sgn * (T)0.95105651629515357212, s2 = sgn * (T)0.58778525229247312917;  // sin 2pi/5, sin 4pi/5
    const cplx<T> t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
    const cplx<T> d1 = csub(v[1], v[4]), d2 = csub(v[2], v[3]);
    const cplx<T> a1 = {v[0].x + c1 * t1.x + c2 * t2.x, v[0].y + c1 * t1.y + c2 * t2.y};
    const cplx<T> a2 = {v[0].x + c2 * t1.x + c1 * t2.x, v[0].y + c2 * t1.y + c1 * t2.y};
    const cplx<T> b1 = {s1 * d1.x + s2 * d2.x, s1 * d1.y + s2 * d2.y};
    const cplx<T> b2 = {s2 * d1.x - s1 * d2.x, s2 * d1.y - s1 * d2.y};
    v[0] = cadd(v[0], cadd(t1, t2));
    v[1] = cadd(a1, imul(b1, (T)1));
    v[4] = csub(a1, imul(b1, (T)1));
    v[2] = cadd(a2, imul(b2, (T)1));
    v[3] = csub(a2, imul(b2, (T)1));
  }
}

// Shared-memory index with one pad slot per 16 complex values: the strided writes of the
// first Stockham passes then spread over all banks.
__device__ __forceinline__ int padi(int i) { return i + (i >> 4); }

// ---- in-place passes with compile-time radix (register staging) -------------------------
// Every thread loads the inputs of its butterflies (at most MaxB<R> of them), the block
// synchronises, then the outputs are written over the same buffer: one N-point buffer per
// transform instead of two.  Supports N / (R * blockDim) <= kMaxB for every radix used.
template <int R>
struct MaxB {
  static constexpr int v = R == 2 ? 4 : R == 3 ? 3 : R == 4 ? 2 : R == 5 ? 2 : 1;
};

template <typename T, int R>
__device__ __forceinline__ void dft_r(cplx<T> (&v)[R], T sgn) {
  if constexpr (R == 8) {
    // radix 8 as 2 x 4: v'[q] = sum_r v[r] w8^{qr}, w8 = e^{sgn 2 pi i / 8}
    const T h = (T)0.70710678118654752440;
    cplx<T> a[4] = {v[0], v[2], v[4], v[6]}, b[4] = {v[1], v[3], v[5], v[7]};
    small_dft(a, 4, sgn);
    small_dft(b, 4, sgn);
    // twiddles w8^q for q = 0..3 applied to the odd half
    const cplx<T> b1 = {h * (b[1].x - sgn * b[1].y), h * (b[1].y + sgn * b[1].x)};
    const cplx<T> b2 = imul(b[2], sgn);
    const cplx<T> b3 = {h * (-b[3].x - sgn * b[3].y), h * (-b[3].y + sgn * b[3].x)};
    v[0] = cadd(a[0], b[0]);
    v[4] = csub(a[0], b[0]);
    v[1] = cadd(a[1], b1);
    v[5] = csub(a[1], b1);
    v[2] = cadd(a[2], b2);
    v[6] = csub(a[2], b2);
    v[3] = cadd(a[3], b3);
    v[7] = csub(a[3], b3);
  } else {
    small_dft(v, R, sgn);
  }
}

// Stockham passes from src (ping-pong with dst); returns the buffer holding the result.
// sgn = -1: forward DFT, +1: unnormalised inverse.
template <typename T>
__device__ cplx<T>* stockham(cplx<T>* src, cplx<T>* dst, const FftPlan& plan, const cplx<T>* __restrict__ tw,
                             T sgn) {
  const int N = plan.n;
  int Ns = 1;
  for (int p = 0; p < plan.nrad; ++p) {
    const int R = plan.rad[p];
    const int nb = N / R;
    const int stride = N / (Ns * R);
    for (int j = threadIdx.x; j < nb; j += blockDim.x) {
      const int k = j % Ns;
      cplx<T> v[8];
      v[0] = src[j];
      for (int r = 1; r < R; ++r) {
        cplx<T> w = tw[r * k * stride];
        w.y *= -sgn;  // table holds e^{-2 pi i k/N}; conjugate for the inverse
        v[r] = cmul(src[j + r * nb], w);
      }
      if (R == 8) {
        cplx<T> v8[8] = {v[0], v[1], v[2], v[3], v[4], v[5], v[6], v[7]};
        dft_r<T, 8>(v8, sgn);
        for (int r = 0; r < 8; ++r) v[r] = v8[r];
      } else {
        small_dft(v, R, sgn);
      }
      const int o = (j / Ns) * Ns * R + k;
      for (int r = 0; r < R; ++r) dst[o + r * Ns] = v[r];
    }
    __syncthreads();
    cplx<T>* t = src;
    src = dst;
    dst = t;
    Ns *= R;
  }
  return src;
}

// twp: this pass's twiddles, [(r - 1) Ns + k] = e^{-2 pi i r k / (Ns R)} (contiguous in k)
template <typename T, int R>
__device__ __forceinline__ void pass_inplace(cplx<T>* buf, int N, int Ns, const cplx<T>* __restrict__ twp, T sgn) {
  constexpr int MB = MaxB<R>::v;
  const int nb = N / R;
  cplx<T> v[MB][R];
#pragma unroll
  for (int b = 0; b < MB; ++b) {
    const int j = threadIdx.x + b * blockDim.x;
    if (j < nb) {
      const int k = j % Ns;
      v[b][0] = buf[padi(j)];
#pragma unroll
      for (int r = 1; r < R; ++r) {
        cplx<T> w = twp[(r - 1) * Ns + k];
        w.y *= -sgn;
        v[b][r] = cmul(buf[padi(j + r * nb)], w);
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < MB; ++b) {
    const int j = threadIdx.x + b * blockDim.x;
    if (j < nb) {
      dft_r<T, R>(v[b], sgn);
      const int k = j % Ns;
      const int o = (j / Ns) * Ns * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) buf[padi(o + r * Ns)] = v[b][r];
    }
  }
  __syncthreads();
}

template <typename T>
__device__ __noinline__ void fft_inplace(cplx<T>* buf, const FftPlan& plan, const cplx<T>* __restrict__ twp, T sgn) {
  int Ns = 1;
  for (int p = 0; p < plan.nrad; ++p) {
    const int R = plan.rad[p];
    const cplx<T>* t = twp + plan.toff[p];
    switch (R) {
      case 8: pass_inplace<T, 8>(buf, plan.n, Ns, t, sgn); break;
      case 4: pass_inplace<T, 4>(buf, plan.n, Ns, t, sgn); break;
      case 2: pass_inplace<T, 2>(buf, plan.n, Ns, t, sgn); break;
      case 3: pass_inplace<T, 3>(buf, plan.n, Ns, t, sgn); break;
      default: pass_inplace<T, 5>(buf, plan.n, Ns, t, sgn); break;
    }
    Ns *= R;
  }
}

// Ping-pong variant: one butterfly in flight per thread (load, transform, store), so only
// R complex values are live; the result alternates between the two padded buffers.
template <typename T, int R>
__device__ __forceinline__ void pass_pp(const cplx<T>* __restrict__ src, cplx<T>* __restrict__ dst, int N, int Ns,
                                        const cplx<T>* __restrict__ twp, T sgn) {
  const int nb = N / R;
#pragma unroll 1
  for (int j = threadIdx.x; j < nb; j += blockDim.x) {
    const int k = j % Ns;
    cplx<T> v[R];
    v[0] = src[padi(j)];
#pragma unroll
    for (int r = 1; r < R; ++r) {
      cplx<T> w = twp[(r - 1) * Ns + k];
      w.y *= -sgn;
      v[r] = cmul(src[padi(j + r * nb)], w);
    }
    dft_r<T, R>(v, sgn);
    const int o = (j / Ns) * Ns * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[padi(o + r * Ns)] = v[r];
  }
  __syncthreads();
}

template <typename T>
__device__ cplx<T>* fft_pp(cplx<T>* a, cplx<T>* b, const FftPlan& plan, const cplx<T>* __restrict__ twp, T sgn) {
  int Ns = 1;
  for (int p = 0; p < plan.nrad; ++p) {
    const int R = plan.rad[p];
    const cplx<T>* t = twp + plan.toff[p];
    switch (R) {
      case 8: pass_pp<T, 8>(a, b, plan.n, Ns, t, sgn); break;
      case 4: pass_pp<T, 4>(a, b, plan.n, Ns, t, sgn); break;
      case 2: pass_pp<T, 2>(a, b, plan.n, Ns, t, sgn); break;
      case 3: pass_pp<T, 3>(a, b, plan.n, Ns, t, sgn); break;
      default: pass_pp<T, 5>(a, b, plan.n, Ns, t, sgn); break;
    }
    cplx<T>* x = a;
    a = b;
    b = x;
    Ns *= R;
  }
  return a;
}

template <typename T>
struct FftArgs {
  int L, nr, ntheta, npairs, C;  // C: column count of a row of F and G
  int64_t sp, sj;                // element strides of F and G between problems mp and ring pairs jp
  int nterms;                    // 0: G in the real type T; 2 or 3: G as BF16 terms in GT
  int odd_top;                   // 1: problem 2 L + 1 holds data (field synthesis); 0: it is empty
  int64_t gt_stride;             // elements between BF16 terms
  __nv_bfloat16* GT;
  FftPlan plan;
  const cplx<T>* tw;
  const cplx<T>* twp;    // per-pass twiddles
  const T* F;            // [2(L+1)][npairs][C]
  T* G;                  // [2(L+1)][npairs][C]
  const T* F2;           // product mode: the second spectrum (NULL: G, SIMT forms)
  const double* mu;      // [nr]
  const double* wgl;     // [npairs]
  const double* maps_in; // [nr][ntheta][nphi]
  double* maps_out;      // [nr][ntheta][nphi]
};

template <typename T, int MODE>
__global__ void __launch_bounds__(256) k_ring_fft(const FftArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int N = a.plan.n;
  cplx<T>* b0 = (cplx<T>*)smem;
  cplx<T>* b1 = b0 + N;
  const int s = blockIdx.x, jp = blockIdx.y;
  const int south = a.ntheta - 1 - jp;
  const bool equator = (south == jp);
  const int L = a.L, np = a.npairs, C = a.C;
  cplx<T>* res;
  if (MODE == FFT_ANALYSE_MAP) {
    const double* rn = a.maps_in + ((size_t)s * a.ntheta + jp) * N;
    const double* rs = a.maps_in + ((size_t)s * a.ntheta + south) * N;
    for (int k = threadIdx.x; k < N; k += blockDim.x) b0[k] = {(T)rn[k], (T)rs[k]};
    __syncthreads();
    res = b0;
  } else {
    for (int k = threadIdx.x; k < N; k += blockDim.x) b0[k] = {(T)0, (T)0};
    __syncthreads();
    for (int m = threadIdx.x; m <= L; m += blockDim.x) {
      const T* e = a.F + (size_t)(2 * m) * a.sp + (size_t)jp * a.sj + 2 * s;
      const T* o = a.F + (size_t)(2 * m + 1) * a.sp + (size_t)jp * a.sj + 2 * s;
      const cplx<T> E = {e[0], e[1]};
      const cplx<T> O = (m < L || a.odd_top) ? cplx<T>{o[0], o[1]} : cplx<T>{(T)0, (T)0};
      const cplx<T> FN = cadd(E, O), FS = csub(E, O);
      if (m == 0) {
        b0[0] = {FN.x, FS.x};
      } else {
        b0[m] = {FN.x - FS.y, FN.y + FS.x};
        b0[N - m] = {FN.x + FS.y, FS.x - FN.y};
      }
    }
    __syncthreads();
    res = stockham(b0, b1, a.plan, a.tw, (T)1);
    if (MODE == FFT_SYNTH_MAP) {
      double* rn = a.maps_out + ((size_t)s * a.ntheta + jp) * N;
      double* rs = a.maps_out + ((size_t)s * a.ntheta + south) * N;
      for (int k = threadIdx.x; k < N; k += blockDim.x) {
        const cplx<T> z = res[k];
        rn[k] = (double)z.x;
        if (!equator) rs[k] = (double)z.y;
      }
      return;
    }
    const T mu = (T)a.mu[s];
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
      const cplx<T> z = res[k];
      res[k] = {z.x * z.x - mu, z.y * z.y - mu};
    }
    __syncthreads();
  }
  cplx<T>* other = (res == b0) ? b1 : b0;
  const cplx<T>* W = stockham(res, other, a.plan, a.tw, (T)-1);
  const T scale = (T)(6.28318530717958647692 / N * a.wgl[jp]);
  for (int m = threadIdx.x; m <= L; m += blockDim.x) {
    const cplx<T> wm = W[m];
    const cplx<T> wc = W[m == 0 ? 0 : N - m];
    // G_N = (W_m + conj W_-m) / 2,  G_S = (W_m - conj W_-m) / (2 i)
    const cplx<T> gn = {(wm.x + wc.x) * (T)0.5, (wm.y - wc.y) * (T)0.5};
    const cplx<T> gs = {(wm.y + wc.y) * (T)0.5, -(wm.x - wc.x) * (T)0.5};
    cplx<T> S, D;
    if (equator) {
      S = {gn.x * scale, gn.y * scale};
      D = S;
    } else {
      S = {(gn.x + gs.x) * scale, (gn.y + gs.y) * scale};
      D = {(gn.x - gs.x) * scale, (gn.y - gs.y) * scale};
    }
    const size_t oe = (size_t)(2 * m) * a.sp + (size_t)jp * a.sj + 2 * s;
    const size_t oo = (size_t)(2 * m + 1) * a.sp + (size_t)jp * a.sj + 2 * s;
    if (a.nterms) {
      store_terms(a.GT + oe, a.gt_stride, a.nterms, (float)S.x);
      store_terms(a.GT + oe + 1, a.gt_stride, a.nterms, (float)S.y);
      store_terms(a.GT + oo, a.gt_stride, a.nterms, (float)D.x);
      store_terms(a.GT + oo + 1, a.gt_stride, a.nterms, (float)D.y);
    } else {
      T* ge = a.G + oe;
      T* go = a.G + oo;
      ge[0] = S.x;
      ge[1] = S.y;
      go[0] = D.x;
      go[1] = D.y;
    }
  }
}

// Product mode of the adjoint: per (shell, ring pair) the spectra F1 = a.F and F2 (a.F2, or
// a.G in the SIMT forms) are taken to the ring values z1, z2 (north + i south) as in the square,
// w = 2 Re z1 Re z2 + i 2 Im z1 Im z2, and W = DFT(w) is written as S and D (same scale and
// equator rule as the square): over F2 in G in the SIMT forms (each block reads its entries of
// F2 before it writes), as BF16 terms in GT in the tensor-core forms.
template <typename T>
__global__ void __launch_bounds__(256) k_ring_product(const FftArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int N = a.plan.n;
  cplx<T>* b0 = (cplx<T>*)smem;
  cplx<T>* b1 = b0 + N;
  cplx<T>* b2 = b1 + N;
  cplx<T>* b3 = b2 + N;
  const int s = blockIdx.x, jp = blockIdx.y;
  const int south = a.ntheta - 1 - jp;
  const bool equator = (south == jp);
  const int L = a.L;
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    b0[k] = {(T)0, (T)0};
    b2[k] = {(T)0, (T)0};
  }
  __syncthreads();
  for (int m = threadIdx.x; m <= L; m += blockDim.x) {
    const size_t oe = (size_t)(2 * m) * a.sp + (size_t)jp * a.sj + 2 * s;
    const size_t oo = (size_t)(2 * m + 1) * a.sp + (size_t)jp * a.sj + 2 * s;
    const T* src[2] = {a.F, a.F2 ? a.F2 : a.G};
    cplx<T>* dst[2] = {b0, b2};
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const cplx<T> E = {src[q][oe], src[q][oe + 1]};
      const cplx<T> O = (m < L) ? cplx<T>{src[q][oo], src[q][oo + 1]} : cplx<T>{(T)0, (T)0};
      const cplx<T> FN = cadd(E, O), FS = csub(E, O);
      if (m == 0) {
        dst[q][0] = {FN.x, FS.x};
      } else {
        dst[q][m] = {FN.x - FS.y, FN.y + FS.x};
        dst[q][N - m] = {FN.x + FS.y, FS.x - FN.y};
      }
    }
  }
  __syncthreads();
  cplx<T>* z1 = stockham(b0, b1, a.plan, a.tw, (T)1);
  cplx<T>* z2 = stockham(b2, b3, a.plan, a.tw, (T)1);
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    const cplx<T> u = z1[k], v = z2[k];
    z1[k] = {(T)2 * u.x * v.x, (T)2 * u.y * v.y};
  }
  __syncthreads();
  const cplx<T>* W = stockham(z1, z1 == b0 ? b1 : b0, a.plan, a.tw, (T)-1);
  const T scale = (T)(6.28318530717958647692 / N * a.wgl[jp]);
  for (int m = threadIdx.x; m <= L; m += blockDim.x) {
    const cplx<T> wm = W[m];
    const cplx<T> wc = W[m == 0 ? 0 : N - m];
    const cplx<T> gn = {(wm.x + wc.x) * (T)0.5, (wm.y - wc.y) * (T)0.5};
    const cplx<T> gs = {(wm.y + wc.y) * (T)0.5, -(wm.x - wc.x) * (T)0.5};
    cplx<T> S, D;
    if (equator) {
      S = {gn.x * scale, gn.y * scale};
      D = S;
    } else {
      S = {(gn.x + gs.x) * scale, (gn.y + gs.y) * scale};
      D = {(gn.x - gs.x) * scale, (gn.y - gs.y) * scale};
    }
    const size_t oe = (size_t)(2 * m) * a.sp + (size_t)jp * a.sj + 2 * s;
    const size_t oo = (size_t)(2 * m + 1) * a.sp + (size_t)jp * a.sj + 2 * s;
    if (a.nterms) {
      store_terms(a.GT + oe, a.gt_stride, a.nterms, (float)S.x);
      store_terms(a.GT + oe + 1, a.gt_stride, a.nterms, (float)S.y);
      if (m < L) {
        store_terms(a.GT + oo, a.gt_stride, a.nterms, (float)D.x);
        store_terms(a.GT + oo + 1, a.gt_stride, a.nterms, (float)D.y);
      }
    } else {
      T* ge = a.G + oe;
      T* go = a.G + oo;
      ge[0] = S.x;
      ge[1] = S.y;
      if (m < L) {
        go[0] = D.x;
        go[1] = D.y;
      }
    }
  }
}

// HEALPix rings: per (shell s, ring pair jp) of ring length n and offset phi_0.  The packed
// spectrum Z_k' = sum_{m = k' mod n, |m| <= L} e^{i m phi_0} (F_N,m + i F_S,m) (F_X,-m = conj F_X,m;
// the short polar rings fold m above n / 2 onto their bins) goes to the ring values
// z = f_N + i f_S by an inverse DFT of length n: on the belt rings (n = 4 nside, a power of two)
// by the object's own stockham plan, on the polar caps as conj(DFT(conj Z)) with Bluestein's
// algorithm: a = (x c) zero-padded to M, A = FFT_M(a), y = IFFT_M(A Bf) / M, X_m = c_m y_m.  The
// square mode then forms w = (Re z)^2 - mu + i ((Im z)^2 - mu), takes W = DFT_n(w) the same way and
// writes S, D of G_m = e^{-i m phi_0} W_{m mod n} (north / south separated as on the Gauss-Legendre
// rings) scaled by (2 pi / n) w_j = 4 pi / N_pix.  The map modes write or read the RING-ordered
// maps [nr][N_pix].
template <typename T>
struct HpArgs {
  int L, ntheta, npairs, nmax, cap;  // cap: complex values per shared-memory buffer
  int64_t sp, sj, npix;   // F and G strides (SIMT layout), pixels per map
  FftPlan plans[fnl_shells::kHpPlans];      // plan of the power of two 2^e
  int64_t twoff[fnl_shells::kHpPlans];      // its twiddles in tw
  const cplx<T>* tw;      // e^{-2 pi i k / 2^e} for every 2^e
  FftPlan dplan;          // of nmax = 4 nside: the belt rings' length, transformed directly
  const cplx<T>* dtw;     // [nmax]
  const int* n;           // [npairs]
  const int* e;           // [npairs] log2 of the ring's Bluestein length
  const int64_t* bfoff;   // [npairs]
  const int64_t* off;     // [ntheta + 1]
  const cplx<T>* rot;     // [npairs][L+1]
  const cplx<T>* chirp;   // [npairs][nmax]
  const cplx<T>* bf;      // per ring pair, M_j
  const T* F;
  T* G;
  const double* mu;
  const double* wgl;
  const double* maps_in;
  double* maps_out;
};

// DFT_n of x[0..n) (in buf, capacity M) by Bluestein; returns the buffer whose first n entries
// hold X_m / M ... times c_m: the caller reads X_m = c_m y_m / M from it.
template <typename T>
__device__ cplx<T>* bluestein(cplx<T>* buf, cplx<T>* other, int M, const FftPlan& plan, const cplx<T>* tw, int n,
                              const cplx<T>* c, const cplx<T>* bf) {
  for (int k = threadIdx.x; k < M; k += blockDim.x) buf[k] = k < n ? cmul(buf[k], c[k]) : cplx<T>{(T)0, (T)0};
  __syncthreads();
  cplx<T>* A = stockham(buf, other, plan, tw, (T)-1);
  for (int k = threadIdx.x; k < M; k += blockDim.x) A[k] = cmul(A[k], bf[k]);
  __syncthreads();
  return stockham(A, A == buf ? other : buf, plan, tw, (T)1);
}

template <typename T, int MODE>
__global__ void __launch_bounds__(256) k_ring_healpix(const HpArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  cplx<T>* b0 = (cplx<T>*)smem;
  cplx<T>* b1 = b0 + a.cap;
  const int s = blockIdx.x, jp = blockIdx.y;
  const int south = a.ntheta - 1 - jp;
  const bool equator = (south == jp);
  const int L = a.L, n = a.n[jp];
  const bool direct = (n == a.nmax);
  const cplx<T>* rot = a.rot + (size_t)jp * (L + 1);
  const cplx<T>* c = a.chirp + (size_t)jp * a.nmax;
  const cplx<T>* bf = a.bf + a.bfoff[jp];
  const int ej = a.e[jp], M = 1 << ej;
  const FftPlan& plan = a.plans[ej];
  const cplx<T>* tw = a.tw + a.twoff[ej];
  const T invM = (T)1 / (T)M;
  cplx<T>* z;
  if (MODE == FFT_ANALYSE_MAP) {
    const double* rn = a.maps_in + (size_t)s * a.npix + a.off[jp];
    const double* rs = a.maps_in + (size_t)s * a.npix + a.off[south];
    for (int k = threadIdx.x; k < n; k += blockDim.x) b0[k] = {(T)rn[k], (T)rs[k]};
    __syncthreads();
    z = b0;
  } else {
    for (int kp = threadIdx.x; kp < n; kp += blockDim.x) {
      cplx<T> acc = {(T)0, (T)0};
      for (int m = kp - n * ((kp + L) / n); m <= L; m += n) {
        if (m < -L) continue;
        const int am = m < 0 ? -m : m;
        const T* e = a.F + (size_t)(2 * am) * a.sp + (size_t)jp * a.sj + 2 * s;
        const T* o = a.F + (size_t)(2 * am + 1) * a.sp + (size_t)jp * a.sj + 2 * s;
        cplx<T> E = {e[0], am ? e[1] : (T)0};
        cplx<T> O = (am < L) ? cplx<T>{o[0], am ? o[1] : (T)0} : cplx<T>{(T)0, (T)0};
        cplx<T> FN = cadd(E, O), FS = csub(E, O), P = rot[am];
        if (m < 0) {
          FN.y = -FN.y;
          FS.y = -FS.y;
          P.y = -P.y;
        }
        acc = cadd(acc, cmul(P, cplx<T>{FN.x - FS.y, FN.y + FS.x}));
      }
        // the belt rings (n = 4 nside) transform directly; the caps by Bluestein as conj(DFT(conj Z))
      b0[kp] = direct ? acc : cplx<T>{acc.x, -acc.y};
    }
    __syncthreads();
    if (direct) {
      z = stockham(b0, b1, a.dplan, a.dtw, (T)1);
    } else {
      cplx<T>* y = bluestein(b0, b1, M, plan, tw, n, c, bf);
      for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const cplx<T> v = cmul(c[k], y[k]);
        y[k] = {v.x * invM, -v.y * invM};
      }
      __syncthreads();
      z = y;
    }
    if (MODE == FFT_SYNTH_MAP) {
      double* rn = a.maps_out + (size_t)s * a.npix + a.off[jp];
      double* rs = a.maps_out + (size_t)s * a.npix + a.off[south];
      for (int k = threadIdx.x; k < n; k += blockDim.x) {
        rn[k] = (double)z[k].x;
        if (!equator) rs[k] = (double)z[k].y;
      }
      return;
    }
    const T mu = (T)a.mu[s];
    for (int k = threadIdx.x; k < n; k += blockDim.x) z[k] = {z[k].x * z[k].x - mu, z[k].y * z[k].y - mu};
    __syncthreads();
  }
  // W = DFT_n of the ring values
  cplx<T>* W;
  if (direct) {
    W = stockham(z, z == b0 ? b1 : b0, a.dplan, a.dtw, (T)-1);
  } else {
    W = bluestein(z, z == b0 ? b1 : b0, M, plan, tw, n, c, bf);
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      const cplx<T> v = cmul(c[k], W[k]);
      W[k] = {v.x * invM, v.y * invM};
    }
    __syncthreads();
  }
  const T scale = (T)(6.28318530717958647692 / n * a.wgl[jp]);
  for (int m = threadIdx.x; m <= L; m += blockDim.x) {
    const int kp = m % n, kc = (n - kp) % n;
    const cplx<T> wm = W[kp], wc = W[kc];
    cplx<T> gn = {(wm.x + wc.x) * (T)0.5, (wm.y - wc.y) * (T)0.5};
    cplx<T> gs = {(wm.y + wc.y) * (T)0.5, -(wm.x - wc.x) * (T)0.5};
    const cplx<T> rc = {rot[m].x, -rot[m].y};  // e^{-i m phi_0}
    gn = cmul(gn, rc);
    gs = cmul(gs, rc);
    cplx<T> S, D;
    if (equator) {
      S = {gn.x * scale, gn.y * scale};
      D = S;
    } else {
      S = {(gn.x + gs.x) * scale, (gn.y + gs.y) * scale};
      D = {(gn.x - gs.x) * scale, (gn.y - gs.y) * scale};
    }
    T* ge = a.G + (size_t)(2 * m) * a.sp + (size_t)jp * a.sj + 2 * s;
    T* go = a.G + (size_t)(2 * m + 1) * a.sp + (size_t)jp * a.sj + 2 * s;
    ge[0] = S.x;
    ge[1] = S.y;
    if (m < L) {
      go[0] = D.x;
      go[1] = D.y;
    }
  }
}

// Estimator rings: per (shell s, ring pair jp) the maps A (columns 2s, 2s + 1 of F) and B
// (columns 2 (nsh + s), + 1) on the north and south rings (inverse DFTs as in the square), then
// sum_k A B^2 on each ring (the equator once), times the ring's Gauss-Legendre weight, into
// part[s][jp] (per-thread sums in the real type, FP64 across threads).
template <typename T>
__device__ __forceinline__ void pack_rings(const FftArgs<T>& a, int jp, int col, cplx<T>* b) {
  const int N = a.plan.n, L = a.L;
  for (int k = threadIdx.x; k < N; k += blockDim.x) b[k] = {(T)0, (T)0};
  __syncthreads();
  for (int m = threadIdx.x; m <= L; m += blockDim.x) {
    const T* e = a.F + (size_t)(2 * m) * a.sp + (size_t)jp * a.sj + col;
    const T* o = a.F + (size_t)(2 * m + 1) * a.sp + (size_t)jp * a.sj + col;
    const cplx<T> E = {e[0], e[1]};
    const cplx<T> O = (m < L) ? cplx<T>{o[0], o[1]} : cplx<T>{(T)0, (T)0};
    const cplx<T> FN = cadd(E, O), FS = csub(E, O);
    if (m == 0) {
      b[0] = {FN.x, FS.x};
    } else {
      b[m] = {FN.x - FS.y, FN.y + FS.x};
      b[N - m] = {FN.x + FS.y, FS.x - FN.y};
    }
  }
  __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(256) k_ring_cubic(const FftArgs<T> a, int nsh, double* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[8];
  const int N = a.plan.n;
  cplx<T>* b0 = (cplx<T>*)smem;
  cplx<T>* b1 = b0 + N;
  cplx<T>* b2 = b1 + N;
  const int s = blockIdx.x, jp = blockIdx.y;
  const bool equator = (a.ntheta - 1 - jp == jp);
  pack_rings(a, jp, 2 * s, b0);
  const cplx<T>* A = stockham(b0, b1, a.plan, a.tw, (T)1);
  cplx<T>* x = (A == b0) ? b1 : b0;
  pack_rings(a, jp, 2 * (nsh + s), x);
  const cplx<T>* B = stockham(x, b2, a.plan, a.tw, (T)1);
  T acct = (T)0;  // per-thread sums in the real type, FP64 across threads
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    const cplx<T> av = A[k], bv = B[k];
    acct += av.x * bv.x * bv.x;
    if (!equator) acct += av.y * bv.y * bv.y;
  }
  double acc = (double)acct;
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    part[(size_t)s * a.npairs + jp] = t * a.wgl[jp];
  }
}

// Group variant: block (group of shells, ring pair); the group's rows of F are staged in
// shared memory with vector loads, every shell then runs through one in-place N-point
// buffer, its results (S, D per order m) overwrite its staged F values, and the group's
// rows of G leave with vector stores (16-byte chunks of BF16 terms, or FP32 pairs).
template <typename T>
__device__ __forceinline__ void store_group(const FftArgs<T>& a, size_t o, const cplx<T>* v, int ng) {
  if (a.nterms) {
    if (ng == 2) {
      float x[4] = {(float)v[0].x, (float)v[0].y, (float)v[1].x, (float)v[1].y};
      __align__(8) __nv_bfloat16 h[3][4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const __nv_bfloat16 h0 = __float2bfloat16_rn(x[q]);
        const float r1 = x[q] - __bfloat162float(h0);
        const __nv_bfloat16 h1 = __float2bfloat16_rn(r1);
        h[0][q] = h0;
        h[1][q] = h1;
        h[2][q] = __float2bfloat16_rn(r1 - __bfloat162float(h1));
      }
      for (int t = 0; t < a.nterms; ++t) *(uint2*)(a.GT + (size_t)t * a.gt_stride + o) = *(const uint2*)h[t];
    } else if (ng == 4) {
      float x[8] = {(float)v[0].x, (float)v[0].y, (float)v[1].x, (float)v[1].y,
                    (float)v[2].x, (float)v[2].y, (float)v[3].x, (float)v[3].y};
      __align__(16) __nv_bfloat16 h[3][8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const __nv_bfloat16 h0 = __float2bfloat16_rn(x[q]);
        const float r1 = x[q] - __bfloat162float(h0);
        const __nv_bfloat16 h1 = __float2bfloat16_rn(r1);
        h[0][q] = h0;
        h[1][q] = h1;
        h[2][q] = __float2bfloat16_rn(r1 - __bfloat162float(h1));
      }
      for (int t = 0; t < a.nterms; ++t) *(uint4*)(a.GT + (size_t)t * a.gt_stride + o) = *(const uint4*)h[t];
    } else {
      for (int g = 0; g < ng; ++g) {
        store_terms(a.GT + o + 2 * g, a.gt_stride, a.nterms, (float)v[g].x);
        store_terms(a.GT + o + 2 * g + 1, a.gt_stride, a.nterms, (float)v[g].y);
      }
    }
  } else {
    for (int g = 0; g < ng; ++g) *(cplx<T>*)(a.G + o + 2 * g) = v[g];
  }
}

template <typename T, int MODE>
__global__ void __launch_bounds__(512, 2) k_ring_fft_group(const FftArgs<T> a, int group) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int N = a.plan.n;
  const int npad = N + N / 16 + 1;
  cplx<T>* bufA = (cplx<T>*)smem;      // two padded buffers: element i at i + i / 16
  cplx<T>* bufB = bufA + npad;
  cplx<T>* stg = bufB + npad;          // [group][2 (L + 1)]: E, O of each shell, then S, D
  const int ns2 = 2 * (a.L + 1);
  cplx<T>* twp = stg + (size_t)group * ns2;  // per-pass twiddles, copied once per block
  for (int k = threadIdx.x; k < a.plan.ttotal; k += blockDim.x) twp[k] = a.twp[k];
  const int jp = blockIdx.y;
  const int south = a.ntheta - 1 - jp;
  const bool equator = (south == jp);
  const int L = a.L;
  const int s0 = blockIdx.x * group;
  const int ng = min(group, a.nr - s0);
  const T scale = (T)(6.28318530717958647692 / N * a.wgl[jp]);
  const size_t rowj = (size_t)jp * a.sj;

  if (MODE != FFT_ANALYSE_MAP) {
    for (int t = threadIdx.x; t < ns2; t += blockDim.x) {
      const int m = t >> 1, p = t & 1;
      if (p == 1 && m == L) {
        for (int g = 0; g < ng; ++g) stg[(size_t)g * ns2 + t] = {(T)0, (T)0};
        continue;
      }
      const cplx<T>* src = (const cplx<T>*)(a.F + rowj + (size_t)(2 * m + p) * a.sp + 2 * s0);
      for (int g = 0; g < ng; ++g) stg[(size_t)g * ns2 + t] = src[g];
    }
    __syncthreads();
  }
  for (int g = 0; g < ng; ++g) {
    const int s = s0 + g;
    cplx<T>* buf = bufA;  // holds the data entering the forward transform
    if (MODE == FFT_ANALYSE_MAP) {
      const double* rn = a.maps_in + ((size_t)s * a.ntheta + jp) * N;
      const double* rs = a.maps_in + ((size_t)s * a.ntheta + south) * N;
      for (int k = threadIdx.x; k < N; k += blockDim.x) buf[padi(k)] = {(T)rn[k], (T)rs[k]};
      __syncthreads();
    } else {
      for (int k = threadIdx.x; k < N; k += blockDim.x) bufA[padi(k)] = {(T)0, (T)0};
      __syncthreads();
      for (int m = threadIdx.x; m <= L; m += blockDim.x) {
        const cplx<T> E = stg[(size_t)g * ns2 + 2 * m];
        const cplx<T> O = stg[(size_t)g * ns2 + 2 * m + 1];
        const cplx<T> FN = cadd(E, O), FS = csub(E, O);
        if (m == 0) {
          bufA[0] = {FN.x, FS.x};
        } else {
          bufA[padi(m)] = {FN.x - FS.y, FN.y + FS.x};
          bufA[padi(N - m)] = {FN.x + FS.y, FS.x - FN.y};
        }
      }
      __syncthreads();
      buf = fft_pp(bufA, bufB, a.plan, twp, (T)1);
      if (MODE == FFT_SYNTH_MAP) {
        double* rn = a.maps_out + ((size_t)s * a.ntheta + jp) * N;
        double* rs = a.maps_out + ((size_t)s * a.ntheta + south) * N;
        for (int k = threadIdx.x; k < N; k += blockDim.x) {
          const cplx<T> z = buf[padi(k)];
          rn[k] = (double)z.x;
          if (!equator) rs[k] = (double)z.y;
        }
        __syncthreads();
        continue;
      }
      const T mu = (T)a.mu[s];
      for (int k = threadIdx.x; k < N; k += blockDim.x) {
        const cplx<T> z = buf[padi(k)];
        buf[padi(k)] = {z.x * z.x - mu, z.y * z.y - mu};
      }
      __syncthreads();
    }
    const cplx<T>* W = fft_pp(buf, buf == bufA ? bufB : bufA, a.plan, twp, (T)-1);
    for (int m = threadIdx.x; m <= L; m += blockDim.x) {
      const cplx<T> wm = W[padi(m)];
      const cplx<T> wc = W[padi(m == 0 ? 0 : N - m)];
      const cplx<T> gn = {(wm.x + wc.x) * (T)0.5, (wm.y - wc.y) * (T)0.5};
      const cplx<T> gs = {(wm.y + wc.y) * (T)0.5, -(wm.x - wc.x) * (T)0.5};
      cplx<T> S, D;
      if (equator) {
        S = {gn.x * scale, gn.y * scale};
        D = S;
      } else {
        S = {(gn.x + gs.x) * scale, (gn.y + gs.y) * scale};
        D = {(gn.x - gs.x) * scale, (gn.y - gs.y) * scale};
      }
      stg[(size_t)g * ns2 + 2 * m] = S;
      stg[(size_t)g * ns2 + 2 * m + 1] = D;
    }
    __syncthreads();
  }
  if (MODE != FFT_SYNTH_MAP) {
    for (int t = threadIdx.x; t < ns2; t += blockDim.x) {
      const int m = t >> 1, p = t & 1;
      cplx<T> v[4];
      for (int g = 0; g < ng; ++g) v[g] = stg[(size_t)g * ns2 + t];
      store_group(a, rowj + (size_t)(2 * m + p) * a.sp + 2 * s0, v, ng);
    }
  }
}

bool plan_fits_group(const FftPlan&, int) { return true; }

template <typename T>
void healpix_impl(const fnl_shells* sh, int mode, const double* maps_in, double* maps_out, cudaStream_t st) {
  HpArgs<T> a{};
  a.L = sh->lmax;
  a.ntheta = sh->ntheta;
  a.npairs = sh->npairs;
  a.nmax = sh->hp_nmax;
  a.cap = std::max(sh->hp_M, sh->hp_nmax);
  a.sp = (int64_t)sh->npairs * sh->C;
  a.sj = sh->C;
  a.npix = sh->npix;
  for (int e = 0; e < fnl_shells::kHpPlans; ++e) {
    a.plans[e] = sh->hp_plans[e];
    a.twoff[e] = sh->hp_twoff[e];
  }
  a.tw = (const cplx<T>*)sh->d_hp_tw;
  a.e = sh->d_hp_e;
  a.bfoff = sh->d_hp_bfoff;
  a.dplan = sh->fft;
  a.dtw = (const cplx<T>*)sh->d_tw;
  a.n = sh->d_hp_n;
  a.off = sh->d_hp_off;
  a.rot = (const cplx<T>*)sh->d_hp_rot;
  a.chirp = (const cplx<T>*)sh->d_hp_chirp;
  a.bf = (const cplx<T>*)sh->d_hp_bf;
  a.F = (const T*)sh->d_F;
  a.G = (T*)sh->d_G;
  a.mu = sh->d_mu;
  a.wgl = sh->d_wgl;
  a.maps_in = maps_in;
  a.maps_out = maps_out;
  const size_t smem = 2 * sizeof(cplx<T>) * (size_t)a.cap;
  const dim3 grid(sh->nr, sh->npairs);
  switch (mode) {
    case FFT_SQUARE:
      FNL_CUDA(cudaFuncSetAttribute(k_ring_healpix<T, FFT_SQUARE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
      k_ring_healpix<T, FFT_SQUARE><<<grid, 256, smem, st>>>(a);
      break;
    case FFT_SYNTH_MAP:
      FNL_CUDA(cudaFuncSetAttribute(k_ring_healpix<T, FFT_SYNTH_MAP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
      k_ring_healpix<T, FFT_SYNTH_MAP><<<grid, 256, smem, st>>>(a);
      break;
    default:
      FNL_CUDA(cudaFuncSetAttribute(k_ring_healpix<T, FFT_ANALYSE_MAP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
      k_ring_healpix<T, FFT_ANALYSE_MAP><<<grid, 256, smem, st>>>(a);
      break;
  }
  FNL_CUDA(cudaGetLastError());
}

template <typename T>
void fft_impl(const fnl_shells* sh, int mode, const double* maps_in, double* maps_out, cudaStream_t st) {
  if (sh->nside) return healpix_impl<T>(sh, mode, maps_in, maps_out, st);
  if (std::is_same<T, float>::value && mode == FFT_SQUARE && launch_ring_square(sh, st)) return;
  FftArgs<T> a{};
  a.L = sh->lmax;
  a.nr = sh->nr;
  a.ntheta = sh->ntheta;
  a.npairs = sh->npairs;
  a.C = sh->nterms ? sh->Cpad : sh->C;
  if (sh->nterms) {  // ring-pair-major: F[jp][mp][Cpad]
    a.sp = sh->Cpad;
    a.sj = (int64_t)2 * (sh->lmax + 1) * sh->Cpad;
  } else {           // problem-major: F[mp][jp][C]
    a.sp = (int64_t)sh->npairs * sh->C;
    a.sj = sh->C;
  }
  a.nterms = sh->nterms;
  a.gt_stride = sh->gt_stride;
  a.GT = (__nv_bfloat16*)sh->d_GT;
  a.plan = sh->fft;
  a.tw = (const cplx<T>*)sh->d_tw;
  a.twp = (const cplx<T>*)sh->d_twp;
  a.F = (const T*)sh->d_F;
  a.G = (T*)sh->d_G;
  a.mu = sh->d_mu;
  a.wgl = sh->d_wgl;
  a.maps_in = maps_in;
  a.maps_out = maps_out;
  const int threads = sh->nphi >= 1024 ? 256 : 128;
  const int gthreads = sh->nphi >= 2048 ? 512 : sh->nphi >= 1024 ? 256 : 128;
  if (!std::is_same<T, double>::value && plan_fits_group(sh->fft, gthreads)) {
    const int group = 2;
    const size_t smem1 = sizeof(cplx<T>) * (2 * (size_t)(sh->nphi + sh->nphi / 16 + 1) +
                                            (size_t)2 * (sh->lmax + 1) * group + (size_t)sh->fft.ttotal);
    dim3 g1((sh->nr + group - 1) / group, sh->npairs);
    if (smem1 > 227 * 1024) throw Error(FNL_EUNSUPPORTED, "ring FFT staging exceeds shared memory");
    switch (mode) {
      case FFT_SQUARE:
        FNL_CUDA(cudaFuncSetAttribute(k_ring_fft_group<T, FFT_SQUARE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem1));
        k_ring_fft_group<T, FFT_SQUARE><<<g1, gthreads, smem1, st>>>(a, group);
        break;
      case FFT_SYNTH_MAP:
        FNL_CUDA(cudaFuncSetAttribute(k_ring_fft_group<T, FFT_SYNTH_MAP>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem1));
        k_ring_fft_group<T, FFT_SYNTH_MAP><<<g1, gthreads, smem1, st>>>(a, group);
        break;
      default:
        FNL_CUDA(cudaFuncSetAttribute(k_ring_fft_group<T, FFT_ANALYSE_MAP>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem1));
        k_ring_fft_group<T, FFT_ANALYSE_MAP><<<g1, gthreads, smem1, st>>>(a, group);
        break;
    }
    FNL_CUDA(cudaGetLastError());
    return;
  }
  const size_t smem = 2 * sizeof(cplx<T>) * (size_t)sh->nphi;
  dim3 grid(sh->nr, sh->npairs);
  switch (mode) {
    case FFT_SQUARE:
      FNL_CUDA(cudaFuncSetAttribute(k_ring_fft<T, FFT_SQUARE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
      k_ring_fft<T, FFT_SQUARE><<<grid, threads, smem, st>>>(a);
      break;
    case FFT_SYNTH_MAP:
      FNL_CUDA(cudaFuncSetAttribute(k_ring_fft<T, FFT_SYNTH_MAP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
      k_ring_fft<T, FFT_SYNTH_MAP><<<grid, threads, smem, st>>>(a);
      break;
    default:
      FNL_CUDA(cudaFuncSetAttribute(k_ring_fft<T, FFT_ANALYSE_MAP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
      k_ring_fft<T, FFT_ANALYSE_MAP><<<grid, threads, smem, st>>>(a);
      break;
  }
  FNL_CUDA(cudaGetLastError());
}

}  // namespace

template <typename T>
void ring_product_impl(const fnl_shells* sh, cudaStream_t st) {
  FftArgs<T> a{};
  a.L = sh->lmax;
  a.nr = sh->nr;
  a.ntheta = sh->ntheta;
  a.npairs = sh->npairs;
  if (sh->nterms) {  // tensor-core forms: both spectra ring-pair-major FP32, output as BF16 terms
    a.C = sh->Cpad;
    a.sp = sh->Cpad;
    a.sj = (int64_t)2 * (sh->lmax + 1) * sh->Cpad;
    a.F2 = (const T*)sh->d_F2;
    a.nterms = sh->nterms;
    a.gt_stride = sh->gt_stride;
    a.GT = (__nv_bfloat16*)sh->d_GT;
  } else {
    a.C = sh->C;
    a.sp = (int64_t)sh->npairs * sh->C;
    a.sj = sh->C;
  }
  a.plan = sh->fft;
  a.tw = (const cplx<T>*)sh->d_tw;
  a.twp = (const cplx<T>*)sh->d_twp;
  a.F = (const T*)sh->d_F;
  a.G = (T*)sh->d_G;
  a.mu = sh->d_mu;
  a.wgl = sh->d_wgl;
  const size_t smem = 4 * sizeof(cplx<T>) * (size_t)sh->nphi;
  if (smem > 227 * 1024) throw Error(FNL_EUNSUPPORTED, "nphi too large for the adjoint ring product");
  FNL_CUDA(cudaFuncSetAttribute(k_ring_product<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_ring_product<T><<<dim3(sh->nr, sh->npairs), sh->nphi >= 1024 ? 256 : 128, smem, st>>>(a);
  FNL_CUDA(cudaGetLastError());
}

void launch_ring_product(const fnl_shells* sh, cudaStream_t st) {
  if (sh->nterms && !sh->d_F2) throw Error(FNL_EUNSUPPORTED, "this object has no second spectrum buffer");
  if (sh->nterms && launch_ring_product_sq(sh, st)) return;
  if (sh->real_is_double) ring_product_impl<double>(sh, st);
  else ring_product_impl<float>(sh, st);
}

void launch_ring_fft(const fnl_shells* sh, int mode, const double* maps_in, double* maps_out, cudaStream_t st) {
  if (sh->real_is_double) fft_impl<double>(sh, mode, maps_in, maps_out, st);
  else fft_impl<float>(sh, mode, maps_in, maps_out, st);
}

template <typename T>
void synth_fields_impl(const fnl_shells* sh, const void* F, int nf, double* maps, cudaStream_t st) {
  FftArgs<T> a{};
  a.L = sh->lmax;
  a.nr = nf;
  a.ntheta = sh->ntheta;
  a.npairs = sh->npairs;
  a.C = 2 * nf;
  a.sp = (int64_t)sh->npairs * a.C;
  a.sj = a.C;
  a.odd_top = 1;
  a.plan = sh->fft;
  a.tw = (const cplx<T>*)sh->d_tw;
  a.twp = (const cplx<T>*)sh->d_twp;
  a.F = (const T*)F;
  a.mu = sh->d_mu;
  a.wgl = sh->d_wgl;
  a.maps_out = maps;
  const size_t smem = 2 * sizeof(cplx<T>) * (size_t)sh->nphi;
  if (smem > 227 * 1024) throw Error(FNL_EUNSUPPORTED, "nphi too large for the field synthesis");
  FNL_CUDA(cudaFuncSetAttribute(k_ring_fft<T, FFT_SYNTH_MAP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_ring_fft<T, FFT_SYNTH_MAP><<<dim3(nf, sh->npairs), sh->nphi >= 1024 ? 256 : 128, smem, st>>>(a);
  FNL_CUDA(cudaGetLastError());
}

void launch_ring_synth_fields(const fnl_shells* sh, const void* F, int nf, double* maps, cudaStream_t st) {
  if (sh->real_is_double) synth_fields_impl<double>(sh, F, nf, maps, st);
  else synth_fields_impl<float>(sh, F, nf, maps, st);
}

template <typename T>
void ring_cubic_impl(const fnl_shells* sh, int nsh, double* part, cudaStream_t st) {
  FftArgs<T> a{};
  a.L = sh->lmax;
  a.nr = sh->nr;
  a.ntheta = sh->ntheta;
  a.npairs = sh->npairs;
  a.C = sh->nterms ? sh->Cpad : sh->C;
  if (sh->nterms) {
    a.sp = sh->Cpad;
    a.sj = (int64_t)2 * (sh->lmax + 1) * sh->Cpad;
  } else {
    a.sp = (int64_t)sh->npairs * sh->C;
    a.sj = sh->C;
  }
  a.plan = sh->fft;
  a.tw = (const cplx<T>*)sh->d_tw;
  a.twp = (const cplx<T>*)sh->d_twp;
  a.F = (const T*)sh->d_F;
  a.wgl = sh->d_wgl;
  const size_t smem = 3 * sizeof(cplx<T>) * (size_t)sh->nphi;
  if (smem > 227 * 1024) throw Error(FNL_EUNSUPPORTED, "nphi too large for the estimator's ring kernel");
  FNL_CUDA(cudaFuncSetAttribute(k_ring_cubic<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_ring_cubic<T><<<dim3(nsh, sh->npairs), 256, smem, st>>>(a, nsh, part);
  FNL_CUDA(cudaGetLastError());
}

void launch_ring_cubic(const fnl_shells* sh, int nsh, double* part, cudaStream_t st) {
  if (sh->real_is_double) ring_cubic_impl<double>(sh, nsh, part, st);
  else ring_cubic_impl<float>(sh, nsh, part, st);
}

}  // namespace fnl
