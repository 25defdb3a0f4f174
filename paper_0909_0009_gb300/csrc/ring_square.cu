// Ring transforms and the pointwise square of steps (ii)-(iv) (Eq. 2) for the tensor-core
// forms: one persistent kernel, a few shells of one ring pair per work item.
//
// Per (ring pair, shell) the two real rings are the complex sequence z = f_N + i f_S whose
// spectrum Z comes from the even/odd Legendre halves: Z_m = F_N,m + i F_S,m and
// Z_{N-m} = conj(F_N,m) + i conj(F_S,m), F_N = E + O, F_S = E - O, zero for l_max < m < N - l_max.
// The kernel forms w = (Re z)^2 - mu + i ((Im z)^2 - mu) with z = IDFT(Z), takes W = DFT(w)
// and writes S = G_N + G_S and D = G_N - G_S (G_N,m = (W_m + conj W_{N-m}) / 2,
// G_S,m = (W_m - conj W_{N-m}) / (2 i)), scaled by (2 pi / N) times the GL weight, as BF16 terms.
//
// Factorisation N = N1 * P * Q (N1 = 25 = 5 x 5; (P, Q) = (16, 8) for 3200, (25, 5) for 3125 =
// 5^5, (8, 8) for 1600, (8, 4) for 800, (4, 4) for 400); a shell's group is P Q threads
// rounded up to whole warps (the extra threads sit out phase 2).  With
// k = k1 + N1 (a + P b) and n = (c + Q d) + P Q n1 the inverse DFT runs as
//   phase 1a  DFT_Q over b              (thread per (k1, a))
//   phase 1b  x w_PQ^{a c}, DFT_P over a (thread per (k1, c))
//   phase 2   x w_N^{k1 (c + Q d)}, DFT_N1 over k1 (thread per (c, d))
// and leaves z in a permuted order; the square is pointwise, so phase 2 squares in registers
// and runs the first forward pass right away (DFT_N1, x w_N^{-k1 (c + Q d)}); phases 3a and
// 3b mirror 1b and 1a and return W in natural order.  Everything stays in one shared-memory
// buffer per shell: element (k1, a|d, b|c) sits at k1 + N1 (a|d) + S (b|c), S = N1 P + pad,
// which makes every phase's warp accesses free of bank conflicts.  Four passes over shared
// memory per shell in place of the ten of a radix-by-radix transform pair.
//
// Work item = (ring pair, G consecutive shells).  The block is G groups of P Q threads, one
// group per shell, synchronised by named barriers; the next item's rows of F are fetched
// with cp.async while the current item is transformed.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>

#include "fnl_internal.cuh"

namespace fnl {

namespace {

// ---- constants: cos and sin of 2 pi j / M (octant reduction, Taylor series in double) --

constexpr double kTwoPi = 6.28318530717958647692528676655900577;

constexpr double taylor_sin(double x) {
  double t = x, s = x;
  for (int k = 1; k < 12; ++k) {
    t *= -x * x / ((2.0 * k) * (2.0 * k + 1.0));
    s += t;
  }
  return s;
}
constexpr double taylor_cos(double x) {
  double t = 1.0, s = 1.0;
  for (int k = 1; k < 12; ++k) {
    t *= -x * x / ((2.0 * k - 1.0) * (2.0 * k));
    s += t;
  }
  return s;
}
constexpr double tcos(long j, long M) {
  j %= M;
  if (j < 0) j += M;
  const long e = 8 * j;
  if (e <= M) return taylor_cos(kTwoPi * (double)j / (double)M);
  if (e <= 2 * M) return taylor_sin(kTwoPi * (double)(M - 4 * j) / (4.0 * M));
  if (e <= 3 * M) return -taylor_sin(kTwoPi * (double)(4 * j - M) / (4.0 * M));
  if (e <= 4 * M) return -taylor_cos(kTwoPi * (double)(M - 2 * j) / (2.0 * M));
  return tcos(M - j, M);
}
constexpr double tsin(long j, long M) { return tcos(4 * j - M, 4 * M); }

struct Tw {
  float c, s;
};
template <int M>
struct TwTable {
  Tw w[M];
  constexpr TwTable() : w() {
    for (int j = 0; j < M; ++j) {
      w[j].c = (float)tcos(j, M);
      w[j].s = (float)tsin(j, M);
    }
  }
};
__constant__ TwTable<8> kTw8 = TwTable<8>();
__constant__ TwTable<16> kTw16 = TwTable<16>();
__constant__ TwTable<25> kTw25 = TwTable<25>();

template <int M>
__device__ __forceinline__ Tw tw_const(int e);
template <>
__device__ __forceinline__ Tw tw_const<8>(int e) { return kTw8.w[e]; }
template <>
__device__ __forceinline__ Tw tw_const<16>(int e) { return kTw16.w[e]; }
template <>
__device__ __forceinline__ Tw tw_const<25>(int e) { return kTw25.w[e]; }

// ---- complex helpers -------------------------------------------------------------------

// A complex value is a float2 (re, im): complex sums and differences, and products with a
// real constant, are one packed f32x2 instruction (sm_100 and later) instead of two.
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 pk(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 cmul(float2 a, float2 w) {
  return make_float2(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x);
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 w) {  // a * conj(w)
  return make_float2(a.x * w.x + a.y * w.y, a.y * w.x - a.x * w.y);
}
template <int SG>  // multiply by SG * i
__device__ __forceinline__ float2 mul_i(float2 a) {
  return SG > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// v * w_M^(SG e), e a compile-time constant after unrolling
template <int M, int SG>
__device__ __forceinline__ float2 twiddle(float2 v, int e) {
  e %= M;
  if (e == 0) return v;
  if (2 * e == M) return make_float2(-v.x, -v.y);
  if (4 * e == M) return mul_i<SG>(v);
  if (4 * e == 3 * M) return mul_i<-SG>(v);
  const Tw w = tw_const<M>(e);
  const float s = SG > 0 ? w.s : -w.s;
  const float2 t = __fmul2_rn(v, pk(w.c));  // (re c, im c)
  return make_float2(fmaf(-v.y, s, t.x), fmaf(v.x, s, t.y));
}

// ---- in-register DFTs, natural order in and out: v'[k] = sum_n v[n] w_R^(SG n k) -------

template <int R, int SG>
struct Dft;

template <int SG>
struct Dft<2, SG> {
  __device__ __forceinline__ static void run(float2* v) {
    const float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};

template <int SG>
struct Dft<4, SG> {
  __device__ __forceinline__ static void run(float2* v) {
    const float2 s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
    const float2 s13 = cadd(v[1], v[3]), t = csub(v[1], v[3]);
    v[0] = cadd(s02, s13);
    v[2] = csub(s02, s13);
    // d02 +- SG i t, with i t = (-t.y, t.x)
    const float2 plus = make_float2(d02.x - t.y, d02.y + t.x), minus = make_float2(d02.x + t.y, d02.y - t.x);
    v[1] = SG > 0 ? plus : minus;
    v[3] = SG > 0 ? minus : plus;
  }
};

template <int SG>
struct Dft<5, SG> {
  __device__ __forceinline__ static void run(float2* v) {
    // cos(2 pi / 5), cos(4 pi / 5), sin(2 pi / 5), sin(4 pi / 5)
    constexpr float c1 = (float)tcos(1, 5), c2 = (float)tcos(2, 5);
    constexpr float s1 = (float)(SG * tsin(1, 5)), s2 = (float)(SG * tsin(2, 5));
    const float2 t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
    const float2 d1 = csub(v[1], v[4]), d2 = csub(v[2], v[3]);
    const float2 a1 = __ffma2_rn(t2, pk(c2), __ffma2_rn(t1, pk(c1), v[0]));
    const float2 a2 = __ffma2_rn(t2, pk(c1), __ffma2_rn(t1, pk(c2), v[0]));
    // u1 = s1 d1 + s2 d2, u2 = s2 d1 - s1 d2; the outputs add and subtract i u
    const float2 u1 = __ffma2_rn(d2, pk(s2), __fmul2_rn(d1, pk(s1)));
    const float2 u2 = __ffma2_rn(d2, pk(-s1), __fmul2_rn(d1, pk(s2)));
    v[0] = cadd(v[0], cadd(t1, t2));
    v[1] = make_float2(a1.x - u1.y, a1.y + u1.x);
    v[4] = make_float2(a1.x + u1.y, a1.y - u1.x);
    v[2] = make_float2(a2.x - u2.y, a2.y + u2.x);
    v[3] = make_float2(a2.x + u2.y, a2.y - u2.x);
  }
};

// R = A * B: n = B n1 + n2, k = k1 + A k2;
// X[k1 + A k2] = sum_n2 w_B^(n2 k2) w_R^(n2 k1) sum_n1 x[B n1 + n2] w_A^(n1 k1)
template <int A, int B, int SG>
__device__ __forceinline__ void dft_composite(float2* x) {
  constexpr int R = A * B;
  float2 y[R];
#pragma unroll
  for (int n2 = 0; n2 < B; ++n2) {
    float2 t[A];
#pragma unroll
    for (int n1 = 0; n1 < A; ++n1) t[n1] = x[B * n1 + n2];
    Dft<A, SG>::run(t);
#pragma unroll
    for (int k1 = 0; k1 < A; ++k1) y[n2 * A + k1] = twiddle<R, SG>(t[k1], n2 * k1);
  }
#pragma unroll
  for (int k1 = 0; k1 < A; ++k1) {
    float2 t[B];
#pragma unroll
    for (int n2 = 0; n2 < B; ++n2) t[n2] = y[n2 * A + k1];
    Dft<B, SG>::run(t);
#pragma unroll
    for (int k2 = 0; k2 < B; ++k2) x[k1 + A * k2] = t[k2];
  }
}

template <int SG>
struct Dft<8, SG> {
  __device__ __forceinline__ static void run(float2* v) { dft_composite<2, 4, SG>(v); }
};
template <int SG>
struct Dft<16, SG> {
  __device__ __forceinline__ static void run(float2* v) { dft_composite<4, 4, SG>(v); }
};
template <int SG>
struct Dft<25, SG> {
  __device__ __forceinline__ static void run(float2* v) { dft_composite<5, 5, SG>(v); }
};

// ---- the kernel --------------------------------------------------------------------------

struct SqArgs {
  int L, nr, ntheta, npairs, N, nterms;
  int64_t sp, sj;         // F and G strides between problems mp and ring pairs jp (elements)
  int64_t gt_stride;      // elements between BF16 terms of G
  const float* F;         // [jp][mp][Cpad]
  __nv_bfloat16* GT;      // [term][jp][mp][Cpad]
  const float2* tw2;      // [N1][Q][P]: w_N^(k1 (c + Q d))
  const float2* tw1;      // [P][Q]:     w_PQ^(a c)
  const double* mu;       // [nr]
  const double* wgl;      // [npairs]
};

template <int T>
__device__ __forceinline__ void group_sync(int g) {
  if constexpr (T == 32) {
    __syncwarp();
  } else {
    asm volatile("bar.sync %0, %1;" ::"r"(g + 1), "r"(T) : "memory");
  }
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// BF16 terms of (x, y): term 0 = bf16(v), term t = bf16(v - sum of earlier terms)
__device__ __forceinline__ void store_pair_terms(__nv_bfloat16* p, int64_t stride, int nterms, float x, float y) {
  const __nv_bfloat162 h0 = __floats2bfloat162_rn(x, y);
  const float rx = x - __low2float(h0), ry = y - __high2float(h0);
  const __nv_bfloat162 h1 = __floats2bfloat162_rn(rx, ry);
  *(__nv_bfloat162*)p = h0;
  *(__nv_bfloat162*)(p + stride) = h1;
  if (nterms > 2) *(__nv_bfloat162*)(p + 2 * stride) = __floats2bfloat162_rn(rx - __low2float(h1), ry - __high2float(h1));
}

// Several instances of one ring length in one launch: instance n owns the work items
// [item0[n], item0[n + 1]); its arguments are inst[n].
struct SqMulti {
  const SqArgs* inst;
  const int* item0;  // [ninst + 1]
  int ninst, maxL;
};

template <int N1, int P, int Q, int PAD, int G, bool MULTI>
__global__ void __launch_bounds__(G * ((P * Q + 31) / 32 * 32), 1)
    k_ring_square(const __grid_constant__ SqArgs a, const __grid_constant__ SqMulti mi) {
  constexpr int T = P * Q;             // tasks of phase 2 (one (c, d) each)
  constexpr int TG = (T + 31) / 32 * 32;  // threads of one shell group (whole warps)
  constexpr int N = N1 * P * Q;
  constexpr int S = N1 * P + PAD;    // stride of the b|c index
  constexpr int NB = N1 * P + S * (Q - 1);  // buffer length per shell (complex)
  static_assert(NB >= N, "buffer");
  extern __shared__ __align__(16) unsigned char smem[];
  float2* buf = (float2*)smem;                  // [G][NB]
  float2* stg = buf + (size_t)G * NB;           // [2 L + 1][G]: staged F rows of the item
  const int Lmax = MULTI ? mi.maxL : a.L;
  float2* tw2 = stg + (size_t)(2 * Lmax + 1) * G;  // [N1][Q][P]
  float2* tw1 = tw2 + (size_t)N1 * T;              // [P][Q]
  for (int i = threadIdx.x; i < N1 * T; i += blockDim.x) tw2[i] = a.tw2[i];
  for (int i = threadIdx.x; i < T; i += blockDim.x) tw1[i] = a.tw1[i];

  const int items = MULTI ? mi.item0[mi.ninst] : (a.nr / G) * a.npairs;
  const int g = threadIdx.x / TG, u = threadIdx.x % TG;
  float2* B = buf + (size_t)g * NB;
  // instance of a work item (binary search over the item offsets)
  auto inst_of = [&](int item) -> int {
    int lo = 0, hi = mi.ninst - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (mi.item0[mid] <= item) lo = mid;
      else hi = mid - 1;
    }
    return lo;
  };

  auto prefetch = [&](int item) {
    int li = item, groups, nrows;  // nrows: problem (m = L, p = 1) is empty
    const float* Fp;
    int64_t sp, sj;
    if constexpr (MULTI) {
      const int n = inst_of(item);
      const SqArgs& pa = mi.inst[n];
      li = item - mi.item0[n];
      groups = pa.nr / G, nrows = 2 * pa.L + 1, Fp = pa.F, sp = pa.sp, sj = pa.sj;
    } else {
      groups = a.nr / G, nrows = 2 * a.L + 1, Fp = a.F, sp = a.sp, sj = a.sj;
    }
    const int jp = li / groups, s0 = (li % groups) * G;
    const float* src = Fp + (size_t)jp * sj + 2 * s0;
    for (int q = threadIdx.x; q < nrows * (G / 2); q += blockDim.x) {
      const int mp = q / (G / 2), h = q % (G / 2);
      cp_async16(stg + (size_t)mp * G + 2 * h, src + (size_t)mp * sp + 4 * h);
    }
    cp_async_commit();
  };

  int item = blockIdx.x;
  if (item < items) prefetch(item);
  SqArgs cur;
  for (; item < items; item += gridDim.x) {
    // this item's instance: the kernel parameters themselves when there is one
    int li = item;
    if constexpr (MULTI) {
      const int n = inst_of(item);
      cur = mi.inst[n];
      li = item - mi.item0[n];
    }
    const SqArgs& A = MULTI ? cur : a;
    const int L = A.L;
    const int groups = A.nr / G;
    const int jp = li / groups, s0 = (li % groups) * G;
    cp_async_wait_all();
    __syncthreads();  // staged rows visible; the previous item's buffers are free
    // spectrum Z of every shell of the item, natural order at k + PAD (k / (N1 P))
    for (int t = threadIdx.x; t < (L + 1) * G; t += blockDim.x) {
      const int gg = t % G, m = t / G;
      const float2 E = stg[(size_t)(2 * m) * G + gg];
      const float2 O = m < L ? stg[(size_t)(2 * m + 1) * G + gg] : make_float2(0.f, 0.f);
      const float2 FN = cadd(E, O), FS = csub(E, O);
      float2* Bg = buf + (size_t)gg * NB;
      if (m == 0) {
        Bg[0] = make_float2(FN.x, FS.x);
      } else {
        Bg[m + PAD * (m / (N1 * P))] = make_float2(FN.x - FS.y, FN.y + FS.x);
        const int k = N - m;
        Bg[k + PAD * (k / (N1 * P))] = make_float2(FN.x + FS.y, FS.x - FN.y);
      }
    }
    __syncthreads();  // the staging buffer is free: fetch the next item behind the transforms
    if (item + (int)gridDim.x < items) prefetch(item + gridDim.x);

    // phase 1a: DFT_Q over b (inverse), entries in l_max < k < N - l_max are zero
#pragma unroll 1
    for (int t = u; t < N1 * P; t += TG) {
      const int base = t;  // k1 + N1 a
      float2 v[Q];
#pragma unroll
      for (int b = 0; b < Q; ++b) {
        const int k = base + N1 * P * b;
        v[b] = (k > L && k < N - L) ? make_float2(0.f, 0.f) : B[base + S * b];
      }
      Dft<Q, 1>::run(v);
#pragma unroll
      for (int c = 0; c < Q; ++c) B[base + S * c] = v[c];
    }
    group_sync<TG>(g);
    // phase 1b: twiddle w_PQ^(a c), DFT_P over a (inverse)
#pragma unroll 1
    for (int t = u; t < N1 * Q; t += TG) {
      const int c = t % Q, k1 = t / Q;
      const int base = k1 + S * c;
      float2 v[P];
#pragma unroll
      for (int aa = 0; aa < P; ++aa) {
        const float2 x = B[base + N1 * aa];
        v[aa] = aa ? cmul(x, tw1[aa * Q + c]) : x;
      }
      Dft<P, 1>::run(v);
#pragma unroll
      for (int d = 0; d < P; ++d) B[base + N1 * d] = v[d];
    }
    group_sync<TG>(g);
    // phase 2: twiddle w_N^(k1 n2), DFT_N1 (inverse) -> ring values, square, DFT_N1 (forward),
    // twiddle w_N^(-k1 n2)
    if (u < T) {
      const int d = u % P, c = u / P;
      const int base = N1 * d + S * c;
      const float mu = (float)A.mu[s0 + g];
      const float2* w = tw2 + c * P + d;
      float2 v[N1];
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) {
        const float2 x = B[base + k1];
        v[k1] = k1 ? cmul(x, w[k1 * T]) : x;
      }
      Dft<N1, 1>::run(v);
#pragma unroll
      for (int n1 = 0; n1 < N1; ++n1) v[n1] = __ffma2_rn(v[n1], v[n1], pk(-mu));
      Dft<N1, -1>::run(v);
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) B[base + k1] = k1 ? cmulc(v[k1], w[k1 * T]) : v[k1];
    }
    group_sync<TG>(g);
    // phase 3a: DFT_P over d (forward), twiddle w_PQ^(-a c)
#pragma unroll 1
    for (int t = u; t < N1 * Q; t += TG) {
      const int c = t % Q, k1 = t / Q;
      const int base = k1 + S * c;
      float2 v[P];
#pragma unroll
      for (int d = 0; d < P; ++d) v[d] = B[base + N1 * d];
      Dft<P, -1>::run(v);
#pragma unroll
      for (int aa = 0; aa < P; ++aa) B[base + N1 * aa] = aa ? cmulc(v[aa], tw1[aa * Q + c]) : v[aa];
    }
    group_sync<TG>(g);
    // phase 3b: DFT_Q over c (forward); W_k at k + PAD (k / (N1 P)), kept for k <= l_max and
    // k >= N - l_max
#pragma unroll 1
    for (int t = u; t < N1 * P; t += TG) {
      const int base = t;
      float2 v[Q];
#pragma unroll
      for (int c = 0; c < Q; ++c) v[c] = B[base + S * c];
      Dft<Q, -1>::run(v);
#pragma unroll
      for (int b = 0; b < Q; ++b) {
        const int k = base + N1 * P * b;
        if (k <= L || k >= N - L) B[base + S * b] = v[b];
      }
    }
    __syncthreads();
    // S and D of every shell, as BF16 terms
    const int south = A.ntheta - 1 - jp;
    const bool equator = (south == jp);
    const float scale = (float)(6.28318530717958647692 / N * A.wgl[jp]);
    __nv_bfloat16* out = A.GT + (size_t)jp * A.sj + 2 * s0;
    for (int t = threadIdx.x; t < (L + 1) * G; t += blockDim.x) {
      const int gg = t % G, m = t / G;
      const float2* Bg = buf + (size_t)gg * NB;
      const float2 wm = Bg[m + PAD * (m / (N1 * P))];
      const int kc = m ? N - m : 0;
      const float2 wc = Bg[kc + PAD * (kc / (N1 * P))];
      const float gnx = (wm.x + wc.x) * 0.5f, gny = (wm.y - wc.y) * 0.5f;
      const float gsx = (wm.y + wc.y) * 0.5f, gsy = -(wm.x - wc.x) * 0.5f;
      float Sx, Sy, Dx, Dy;
      if (equator) {
        Sx = Dx = gnx * scale;
        Sy = Dy = gny * scale;
      } else {
        Sx = (gnx + gsx) * scale;
        Sy = (gny + gsy) * scale;
        Dx = (gnx - gsx) * scale;
        Dy = (gny - gsy) * scale;
      }
      __nv_bfloat16* o = out + (size_t)(2 * m) * A.sp + 2 * gg;
      store_pair_terms(o, A.gt_stride, A.nterms, Sx, Sy);
      if (m < L) store_pair_terms(o + A.sp, A.gt_stride, A.nterms, Dx, Dy);
    }
  }
  cp_async_wait_all();
}

// Rings of the cubic estimator (Sect. 5): work item = (ring pair, G / 2 shells).  Groups
// 0 .. G/2 - 1 hold the A spectra of the item's shells (columns 2 s of F), groups G/2 .. G - 1
// their B spectra (columns 2 (nsh + s)).  Phases 1a, 1b and the inverse half of phase 2 run as
// in the square and leave every field's ring values in its buffer, in the same permuted order;
// then the A group of each shell sums A B^2 over the ring pair (north rings in x, south in y,
// the equator once; FP32 products and per-thread sums, FP64 across threads) and writes the GL
// weight times the sum to part[s][jp].
struct CubeArgs {
  int L, nsh, ntheta, npairs;
  int64_t sp, sj;      // F strides between problems mp and ring pairs jp (floats)
  const float* F;      // [jp][mp][Cpad]
  const float2* tw2;   // as SqArgs
  const float2* tw1;
  const double* wgl;   // [npairs]
  double* part;        // [nsh][npairs]
};

template <int N1, int P, int Q, int PAD, int G>
__global__ void __launch_bounds__(G * ((P * Q + 31) / 32 * 32), 1) k_ring_cubic_sq(const __grid_constant__ CubeArgs a) {
  constexpr int T = P * Q;
  constexpr int TG = (T + 31) / 32 * 32;
  constexpr int N = N1 * P * Q;
  constexpr int S = N1 * P + PAD;
  constexpr int NB = N1 * P + S * (Q - 1);
  constexpr int H = G / 2;  // shells of an item
  static_assert(NB >= N && H % 2 == 0, "layout");
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[G][TG / 32];
  float2* buf = (float2*)smem;                       // [G][NB]
  float2* stg = buf + (size_t)G * NB;                // [2 L + 1][G]: A fields, then B fields
  float2* tw2 = stg + (size_t)(2 * a.L + 1) * G;     // [N1][Q][P]
  float2* tw1 = tw2 + (size_t)N1 * T;                // [P][Q]
  for (int i = threadIdx.x; i < N1 * T; i += blockDim.x) tw2[i] = a.tw2[i];
  for (int i = threadIdx.x; i < T; i += blockDim.x) tw1[i] = a.tw1[i];
  const int groups = a.nsh / H;
  const int items = groups * a.npairs;
  const int g = threadIdx.x / TG, u = threadIdx.x % TG;
  float2* B = buf + (size_t)g * NB;
  const int L = a.L;

  auto prefetch = [&](int item) {
    const int jp = item / groups, s0 = (item % groups) * H;
    const float* srcA = a.F + (size_t)jp * a.sj + 2 * s0;
    const float* srcB = a.F + (size_t)jp * a.sj + 2 * (a.nsh + s0);
    constexpr int Q4 = H / 2;  // 16-byte copies per row and field
    for (int q = threadIdx.x; q < (2 * L + 1) * 2 * Q4; q += blockDim.x) {
      const int mp = q / (2 * Q4), h = q % (2 * Q4);
      const bool isB = h >= Q4;
      const int hh = isB ? h - Q4 : h;
      cp_async16(stg + (size_t)mp * G + (isB ? H : 0) + 2 * hh, (isB ? srcB : srcA) + (size_t)mp * a.sp + 4 * hh);
    }
    cp_async_commit();
  };

  int item = blockIdx.x;
  if (item < items) prefetch(item);
  for (; item < items; item += gridDim.x) {
    const int jp = item / groups, s0 = (item % groups) * H;
    cp_async_wait_all();
    __syncthreads();  // staged rows visible; the previous item's buffers are free
    for (int t = threadIdx.x; t < (L + 1) * G; t += blockDim.x) {
      const int gg = t % G, m = t / G;
      const float2 E = stg[(size_t)(2 * m) * G + gg];
      const float2 O = m < L ? stg[(size_t)(2 * m + 1) * G + gg] : make_float2(0.f, 0.f);
      const float2 FN = cadd(E, O), FS = csub(E, O);
      float2* Bg = buf + (size_t)gg * NB;
      if (m == 0) {
        Bg[0] = make_float2(FN.x, FS.x);
      } else {
        Bg[m + PAD * (m / (N1 * P))] = make_float2(FN.x - FS.y, FN.y + FS.x);
        const int k = N - m;
        Bg[k + PAD * (k / (N1 * P))] = make_float2(FN.x + FS.y, FS.x - FN.y);
      }
    }
    __syncthreads();
    if (item + (int)gridDim.x < items) prefetch(item + gridDim.x);
    // phase 1a: DFT_Q over b (inverse)
#pragma unroll 1
    for (int t = u; t < N1 * P; t += TG) {
      const int base = t;
      float2 v[Q];
#pragma unroll
      for (int b = 0; b < Q; ++b) {
        const int k = base + N1 * P * b;
        v[b] = (k > L && k < N - L) ? make_float2(0.f, 0.f) : B[base + S * b];
      }
      Dft<Q, 1>::run(v);
#pragma unroll
      for (int c = 0; c < Q; ++c) B[base + S * c] = v[c];
    }
    group_sync<TG>(g);
    // phase 1b: twiddle w_PQ^(a c), DFT_P over a (inverse)
#pragma unroll 1
    for (int t = u; t < N1 * Q; t += TG) {
      const int c = t % Q, k1 = t / Q;
      const int base = k1 + S * c;
      float2 v[P];
#pragma unroll
      for (int aa = 0; aa < P; ++aa) {
        const float2 x = B[base + N1 * aa];
        v[aa] = aa ? cmul(x, tw1[aa * Q + c]) : x;
      }
      Dft<P, 1>::run(v);
#pragma unroll
      for (int d = 0; d < P; ++d) B[base + N1 * d] = v[d];
    }
    group_sync<TG>(g);
    // phase 2 (inverse half): twiddle w_N^(k1 n2), DFT_N1 -> ring values.  The B groups leave
    // theirs in shared memory; each A group keeps its own in registers and, once the B values
    // have landed, sums A B^2 over the ring points it holds.
    const int base2 = N1 * (u % P) + S * (u / P);
    float2 v[N1];
    if (u < T) {
      const float2* w = tw2 + (u / P) * P + u % P;
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) {
        const float2 x = B[base2 + k1];
        v[k1] = k1 ? cmul(x, w[k1 * T]) : x;
      }
      Dft<N1, 1>::run(v);
      if (g >= H) {
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) B[base2 + n1] = v[n1];
      }
    }
    __syncthreads();  // the B ring values of every shell in place
    if (g < H) {
      const float2* BB = buf + (size_t)(g + H) * NB;
      const bool equator = (a.ntheta - 1 - jp == jp);
      float accf = 0.f;  // N1 terms per thread in FP32, the block sums in FP64
      if (u < T) {
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) {
          const float2 y = BB[base2 + n1];
          accf += v[n1].x * y.x * y.x;
          if (!equator) accf += v[n1].y * y.y * y.y;
        }
      }
      double acc = (double)accf;
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
      if ((u & 31) == 0) red[g][u >> 5] = acc;
      group_sync<TG>(g);
      if (u == 0) {
        double t = 0.0;
#pragma unroll
        for (int w = 0; w < TG / 32; ++w) t += red[g][w];
        a.part[(size_t)(s0 + g) * a.npairs + jp] = t * a.wgl[jp];
      }
    }
  }
  cp_async_wait_all();
}

// Rings of the adjoint (differentiation form) in the tensor-core forms: per (ring pair, shell)
// the spectra of f (F1) and of s (F2) go to their ring values z1, z2 (north + i south), the
// product w = 2 Re z1 Re z2 + i 2 Im z1 Im z2 (the square's adjoint, 2 f s) goes back by the
// forward DFT, and S and D are written as BF16 terms with the square's scale and equator rule.
// Work item = (ring pair, G / 2 shells): groups 0 .. G/2 - 1 transform the f spectra of the
// item's shells, groups G/2 .. G - 1 their s spectra; after the inverse half of phase 2 the s
// groups leave their ring values in shared memory, and each f group multiplies them into its
// own (still in registers) and runs the forward half and phases 3a, 3b alone.
struct ProdArgs {
  int L, nr, ntheta, npairs, N, nterms;
  int64_t sp, sj;      // F1, F2 and G strides between problems mp and ring pairs jp (elements)
  int64_t gt_stride;   // elements between BF16 terms of G
  const float* F1;     // [jp][mp][Cpad]: spectra of f
  const float* F2;     // [jp][mp][Cpad]: spectra of s
  __nv_bfloat16* GT;   // [term][jp][mp][Cpad]
  const float2* tw2;
  const float2* tw1;
  const double* wgl;   // [npairs]
};

template <int N1, int P, int Q, int PAD, int G>
__global__ void __launch_bounds__(G * ((P * Q + 31) / 32 * 32), 1) k_ring_product_sq(const __grid_constant__ ProdArgs a) {
  constexpr int T = P * Q;
  constexpr int TG = (T + 31) / 32 * 32;
  constexpr int N = N1 * P * Q;
  constexpr int S = N1 * P + PAD;
  constexpr int NB = N1 * P + S * (Q - 1);
  constexpr int H = G / 2;  // shells of an item
  static_assert(NB >= N && H % 2 == 0, "layout");
  extern __shared__ __align__(16) unsigned char smem[];
  float2* buf = (float2*)smem;                    // [G][NB]
  float2* stg = buf + (size_t)G * NB;             // [2 L + 1][G]: f fields, then s fields
  float2* tw2 = stg + (size_t)(2 * a.L + 1) * G;  // [N1][Q][P]
  float2* tw1 = tw2 + (size_t)N1 * T;             // [P][Q]
  for (int i = threadIdx.x; i < N1 * T; i += blockDim.x) tw2[i] = a.tw2[i];
  for (int i = threadIdx.x; i < T; i += blockDim.x) tw1[i] = a.tw1[i];
  const int groups = a.nr / H;
  const int items = groups * a.npairs;
  const int g = threadIdx.x / TG, u = threadIdx.x % TG;
  const bool is_f = g < H;
  float2* B = buf + (size_t)g * NB;
  const int L = a.L;

  auto prefetch = [&](int item) {
    const int jp = item / groups, s0 = (item % groups) * H;
    const float* src1 = a.F1 + (size_t)jp * a.sj + 2 * s0;
    const float* src2 = a.F2 + (size_t)jp * a.sj + 2 * s0;
    constexpr int Q4 = H / 2;  // 16-byte copies per row and field
    for (int q = threadIdx.x; q < (2 * L + 1) * 2 * Q4; q += blockDim.x) {
      const int mp = q / (2 * Q4), h = q % (2 * Q4);
      const bool second = h >= Q4;
      const int hh = second ? h - Q4 : h;
      cp_async16(stg + (size_t)mp * G + (second ? H : 0) + 2 * hh, (second ? src2 : src1) + (size_t)mp * a.sp + 4 * hh);
    }
    cp_async_commit();
  };

  int item = blockIdx.x;
  if (item < items) prefetch(item);
  for (; item < items; item += gridDim.x) {
    const int jp = item / groups, s0 = (item % groups) * H;
    const double wgl = a.wgl[jp];
    cp_async_wait_all();
    __syncthreads();  // staged rows visible; the previous item's buffers are free
    for (int t = threadIdx.x; t < (L + 1) * G; t += blockDim.x) {
      const int gg = t % G, m = t / G;
      const float2 E = stg[(size_t)(2 * m) * G + gg];
      const float2 O = m < L ? stg[(size_t)(2 * m + 1) * G + gg] : make_float2(0.f, 0.f);
      const float2 FN = cadd(E, O), FS = csub(E, O);
      float2* Bg = buf + (size_t)gg * NB;
      if (m == 0) {
        Bg[0] = make_float2(FN.x, FS.x);
      } else {
        Bg[m + PAD * (m / (N1 * P))] = make_float2(FN.x - FS.y, FN.y + FS.x);
        const int k = N - m;
        Bg[k + PAD * (k / (N1 * P))] = make_float2(FN.x + FS.y, FS.x - FN.y);
      }
    }
    __syncthreads();
    if (item + (int)gridDim.x < items) prefetch(item + gridDim.x);
    // phase 1a: DFT_Q over b (inverse), entries in l_max < k < N - l_max are zero
#pragma unroll 1
    for (int t = u; t < N1 * P; t += TG) {
      float2 v[Q];
#pragma unroll
      for (int b = 0; b < Q; ++b) {
        const int k = t + N1 * P * b;
        v[b] = (k > L && k < N - L) ? make_float2(0.f, 0.f) : B[t + S * b];
      }
      Dft<Q, 1>::run(v);
#pragma unroll
      for (int c = 0; c < Q; ++c) B[t + S * c] = v[c];
    }
    group_sync<TG>(g);
    // phase 1b: twiddle w_PQ^(a c), DFT_P over a (inverse)
#pragma unroll 1
    for (int t = u; t < N1 * Q; t += TG) {
      const int c = t % Q, k1 = t / Q;
      const int base = k1 + S * c;
      float2 v[P];
#pragma unroll
      for (int aa = 0; aa < P; ++aa) {
        const float2 x = B[base + N1 * aa];
        v[aa] = aa ? cmul(x, tw1[aa * Q + c]) : x;
      }
      Dft<P, 1>::run(v);
#pragma unroll
      for (int d = 0; d < P; ++d) B[base + N1 * d] = v[d];
    }
    group_sync<TG>(g);
    // phase 2: twiddle w_N^(k1 n2), DFT_N1 (inverse) -> ring values; the s groups leave theirs in
    // shared memory, the f groups keep theirs in registers, multiply, and go back (forward)
    {
      const int d = u % P, c = u / P;
      const int base = N1 * d + S * c;
      const float2* w = tw2 + c * P + d;
      float2 v[N1];
      if (u < T) {
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) {
          const float2 x = B[base + k1];
          v[k1] = k1 ? cmul(x, w[k1 * T]) : x;
        }
        Dft<N1, 1>::run(v);
        if (!is_f) {
#pragma unroll
          for (int n1 = 0; n1 < N1; ++n1) B[base + n1] = v[n1];
        }
      }
      __syncthreads();  // the s ring values are in place
      if (is_f && u < T) {
        const float2* Bs = buf + (size_t)(g + H) * NB;
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) {
          const float2 y = Bs[base + n1];
          v[n1] = make_float2(2.f * v[n1].x * y.x, 2.f * v[n1].y * y.y);
        }
        Dft<N1, -1>::run(v);
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) B[base + k1] = k1 ? cmulc(v[k1], w[k1 * T]) : v[k1];
      }
    }
    if (is_f) {
      group_sync<TG>(g);
      // phase 3a: DFT_P over d (forward), twiddle w_PQ^(-a c)
#pragma unroll 1
      for (int t = u; t < N1 * Q; t += TG) {
        const int c = t % Q, k1 = t / Q;
        const int base = k1 + S * c;
        float2 v[P];
#pragma unroll
        for (int d = 0; d < P; ++d) v[d] = B[base + N1 * d];
        Dft<P, -1>::run(v);
#pragma unroll
        for (int aa = 0; aa < P; ++aa) B[base + N1 * aa] = aa ? cmulc(v[aa], tw1[aa * Q + c]) : v[aa];
      }
      group_sync<TG>(g);
      // phase 3b: DFT_Q over c (forward); W_k kept for k <= l_max and k >= N - l_max
#pragma unroll 1
      for (int t = u; t < N1 * P; t += TG) {
        float2 v[Q];
#pragma unroll
        for (int c = 0; c < Q; ++c) v[c] = B[t + S * c];
        Dft<Q, -1>::run(v);
#pragma unroll
        for (int b = 0; b < Q; ++b) {
          const int k = t + N1 * P * b;
          if (k <= L || k >= N - L) B[t + S * b] = v[b];
        }
      }
    }
    __syncthreads();
    // S and D of every shell of the item, as BF16 terms
    const int south = a.ntheta - 1 - jp;
    const bool equator = (south == jp);
    const float scale = (float)(6.28318530717958647692 / N * wgl);
    __nv_bfloat16* out = a.GT + (size_t)jp * a.sj + 2 * s0;
    for (int t = threadIdx.x; t < (L + 1) * H; t += blockDim.x) {
      const int gg = t % H, m = t / H;
      const float2* Bg = buf + (size_t)gg * NB;
      const float2 wm = Bg[m + PAD * (m / (N1 * P))];
      const int kc = m ? N - m : 0;
      const float2 wc = Bg[kc + PAD * (kc / (N1 * P))];
      const float gnx = (wm.x + wc.x) * 0.5f, gny = (wm.y - wc.y) * 0.5f;
      const float gsx = (wm.y + wc.y) * 0.5f, gsy = -(wm.x - wc.x) * 0.5f;
      float Sx, Sy, Dx, Dy;
      if (equator) {
        Sx = Dx = gnx * scale;
        Sy = Dy = gny * scale;
      } else {
        Sx = (gnx + gsx) * scale;
        Sy = (gny + gsy) * scale;
        Dx = (gnx - gsx) * scale;
        Dy = (gny - gsy) * scale;
      }
      __nv_bfloat16* o = out + (size_t)(2 * m) * a.sp + 2 * gg;
      store_pair_terms(o, a.gt_stride, a.nterms, Sx, Sy);
      if (m < L) store_pair_terms(o + a.sp, a.gt_stride, a.nterms, Dx, Dy);
    }
  }
  cp_async_wait_all();
}

struct SqConfig {
  int N, N1, P, Q, G;
};

// Sizes with a specialised kernel: N = 25 P Q.
constexpr SqConfig kSqConfigs[] = {{3200, 25, 16, 8, 4}, {3125, 25, 25, 5, 4}, {1600, 25, 8, 8, 8}, {800, 25, 8, 4, 8},
                                   {400, 25, 4, 4, 8}};

template <int N1, int P, int Q, int PAD, int G>
void launch_sq(const SqArgs& a, int sms, cudaStream_t st, const SqMulti* multi = nullptr, int items_multi = 0) {
  constexpr int T = P * Q, TG = (T + 31) / 32 * 32, N = N1 * P * Q, S = N1 * P + PAD, NB = N1 * P + S * (Q - 1);
  const int Lmax = multi ? multi->maxL : a.L;
  const size_t smem = sizeof(float2) * ((size_t)G * NB + (size_t)(2 * Lmax + 1) * G + (size_t)N1 * T + T);
  if (smem > 227 * 1024) throw Error(FNL_EUNSUPPORTED, "ring square staging exceeds shared memory");
  (void)N;
  auto run = [&](auto kern, int items) {
    FNL_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    FNL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, G * TG, smem));
    const int grid = std::max(1, std::min(items, sms * std::max(per_sm, 1)));
    kern<<<grid, G * TG, smem, st>>>(a, multi ? *multi : SqMulti{});
    FNL_CUDA(cudaGetLastError());
  };
  if (multi) run(k_ring_square<N1, P, Q, PAD, G, true>, items_multi);
  else run(k_ring_square<N1, P, Q, PAD, G, false>, (a.nr / G) * a.npairs);
}

template <int N1, int P, int Q, int PAD, int G>
void launch_cube(const CubeArgs& a, int sms, cudaStream_t st) {
  constexpr int T = P * Q, TG = (T + 31) / 32 * 32, S = N1 * P + PAD, NB = N1 * P + S * (Q - 1);
  const size_t smem = sizeof(float2) * ((size_t)G * NB + (size_t)(2 * a.L + 1) * G + (size_t)N1 * T + T);
  if (smem > 227 * 1024 - sizeof(double) * G * (TG / 32))
    throw Error(FNL_EUNSUPPORTED, "estimator ring staging exceeds shared memory");
  auto kern = k_ring_cubic_sq<N1, P, Q, PAD, G>;
  FNL_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  FNL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, G * TG, smem));
  const int items = (a.nsh / (G / 2)) * a.npairs;
  const int grid = std::max(1, std::min(items, sms * std::max(per_sm, 1)));
  kern<<<grid, G * TG, smem, st>>>(a);
  FNL_CUDA(cudaGetLastError());
}

template <int N1, int P, int Q, int PAD, int G>
void launch_prod(const ProdArgs& a, int sms, cudaStream_t st) {
  constexpr int T = P * Q, TG = (T + 31) / 32 * 32, S = N1 * P + PAD, NB = N1 * P + S * (Q - 1);
  const size_t smem = sizeof(float2) * ((size_t)G * NB + (size_t)(2 * a.L + 1) * G + (size_t)N1 * T + T);
  if (smem > 227 * 1024) throw Error(FNL_EUNSUPPORTED, "adjoint ring staging exceeds shared memory");
  auto kern = k_ring_product_sq<N1, P, Q, PAD, G>;
  FNL_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  FNL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, G * TG, smem));
  const int items = (a.nr / (G / 2)) * a.npairs;
  const int grid = std::max(1, std::min(items, sms * std::max(per_sm, 1)));
  kern<<<grid, G * TG, smem, st>>>(a);
  FNL_CUDA(cudaGetLastError());
}

}  // namespace

// Twiddle tables of the specialised ring kernel for N = nphi (empty if none applies).
void ring_square_tables(int nphi, std::vector<float>& tw2, std::vector<float>& tw1) {
  tw2.clear();
  tw1.clear();
  for (const SqConfig& c : kSqConfigs) {
    if (c.N != nphi) continue;
    const int T = c.P * c.Q;
    tw2.resize(2 * (size_t)c.N1 * T);
    for (int k1 = 0; k1 < c.N1; ++k1)
      for (int cc = 0; cc < c.Q; ++cc)
        for (int d = 0; d < c.P; ++d) {
          const long e = (long)k1 * (cc + c.Q * d);
          const size_t i = ((size_t)k1 * c.Q + cc) * c.P + d;
          tw2[2 * i] = (float)tcos(e, c.N);
          tw2[2 * i + 1] = (float)tsin(e, c.N);
        }
    tw1.resize(2 * (size_t)T);
    for (int aa = 0; aa < c.P; ++aa)
      for (int cc = 0; cc < c.Q; ++cc) {
        const size_t i = (size_t)aa * c.Q + cc;
        tw1[2 * i] = (float)tcos((long)aa * cc, T);
        tw1[2 * i + 1] = (float)tsin((long)aa * cc, T);
      }
  }
}

namespace {

SqArgs sq_args_of(const fnl_shells* sh) {
  SqArgs a;
  a.L = sh->lmax;
  a.nr = sh->nr;
  a.ntheta = sh->ntheta;
  a.npairs = sh->npairs;
  a.N = sh->nphi;
  a.nterms = sh->nterms;
  a.sp = sh->Cpad;
  a.sj = (int64_t)2 * (sh->lmax + 1) * sh->Cpad;
  a.gt_stride = sh->gt_stride;
  a.F = (const float*)sh->d_F;
  a.GT = (__nv_bfloat16*)sh->d_GT;
  a.tw2 = (const float2*)sh->d_sqtw2;
  a.tw1 = (const float2*)sh->d_sqtw1;
  a.mu = sh->d_mu;
  a.wgl = sh->d_wgl;
  return a;
}

}  // namespace

int ring_square_group(const fnl_shells* sh) {
  if (!sh->nterms || !sh->d_sqtw2) return 0;
  for (const SqConfig& c : kSqConfigs)
    if (c.N == sh->nphi) return (sh->nr % c.G || 2 * sh->lmax + 2 > c.N) ? 0 : c.G;
  return 0;
}

size_t ring_square_args_size() { return sizeof(SqArgs); }

void ring_square_args(const fnl_shells* sh, void* out) {
  const SqArgs a = sq_args_of(sh);
  std::memcpy(out, &a, sizeof(a));
}

// Specialised steps (ii)-(iv) ring kernel of the tensor-core forms; false if this
// configuration has none (the caller then runs the general kernel).
bool launch_ring_square(const fnl_shells* sh, cudaStream_t st) {
  if (!ring_square_group(sh)) return false;
  const SqArgs a = sq_args_of(sh);
  switch (sh->nphi) {
    case 3200: launch_sq<25, 16, 8, 2, 4>(a, sh->sms_ring ? sh->sms_ring : sh->sms, st); return true;
    case 3125: launch_sq<25, 25, 5, 2, 4>(a, sh->sms_ring ? sh->sms_ring : sh->sms, st); return true;
    case 1600: launch_sq<25, 8, 8, 2, 8>(a, sh->sms_ring ? sh->sms_ring : sh->sms, st); return true;
    case 800: launch_sq<25, 8, 4, 4, 8>(a, sh->sms_ring ? sh->sms_ring : sh->sms, st); return true;
    case 400: launch_sq<25, 4, 4, 2, 8>(a, sh->sms_ring ? sh->sms_ring : sh->sms, st); return true;
    default: return false;
  }
}

// One launch over several instances of the ring length of `proto` (whose twiddle tables
// serve all of them): d_inst holds their ring_square_args, d_item0 the item offsets.
void launch_ring_square_multi(const fnl_shells* proto, const void* d_inst, const int* d_item0, int ninst, int maxL,
                              int items, cudaStream_t st) {
  const SqArgs a = sq_args_of(proto);
  const SqMulti m{(const SqArgs*)d_inst, d_item0, ninst, maxL};
  switch (proto->nphi) {
    case 3200: launch_sq<25, 16, 8, 2, 4>(a, proto->sms, st, &m, items); return;
    case 3125: launch_sq<25, 25, 5, 2, 4>(a, proto->sms, st, &m, items); return;
    case 1600: launch_sq<25, 8, 8, 2, 8>(a, proto->sms, st, &m, items); return;
    case 800: launch_sq<25, 8, 4, 4, 8>(a, proto->sms, st, &m, items); return;
    case 400: launch_sq<25, 4, 4, 2, 8>(a, proto->sms, st, &m, items); return;
    default: throw Error(FNL_EUNSUPPORTED, "no specialised ring kernel for this ring length");
  }
}

// Specialised rings of the estimator for an object of 2 nsh fields (A, then B); false if this
// configuration has none (the caller then runs the general kernel).
bool launch_ring_cubic_sq(const fnl_shells* sh, int nsh, double* part, cudaStream_t st) {
  const int G = ring_square_group(sh);
  if (!G || sh->nr != 2 * nsh || nsh % (G / 2) || nsh % 2) return false;
  CubeArgs a;
  a.L = sh->lmax;
  a.nsh = nsh;
  a.ntheta = sh->ntheta;
  a.npairs = sh->npairs;
  a.sp = sh->Cpad;
  a.sj = (int64_t)2 * (sh->lmax + 1) * sh->Cpad;
  a.F = (const float*)sh->d_F;
  a.tw2 = (const float2*)sh->d_sqtw2;
  a.tw1 = (const float2*)sh->d_sqtw1;
  a.wgl = sh->d_wgl;
  a.part = part;
  switch (sh->nphi) {
    case 3200: launch_cube<25, 16, 8, 2, 4>(a, sh->sms, st); return true;
    case 3125: launch_cube<25, 25, 5, 2, 4>(a, sh->sms, st); return true;
    case 1600: launch_cube<25, 8, 8, 2, 8>(a, sh->sms, st); return true;
    case 800: launch_cube<25, 8, 4, 4, 8>(a, sh->sms, st); return true;
    case 400: launch_cube<25, 4, 4, 2, 8>(a, sh->sms, st); return true;
    default: return false;
  }
}

// Specialised adjoint rings of the tensor-core forms (f spectra in d_F, s spectra in d_F2, 2 f s
// as BF16 terms in d_GT); false if this configuration has none (the caller then runs the general
// kernel).  The shells of an item are half the square kernel's group, since every shell holds
// two fields.
bool launch_ring_product_sq(const fnl_shells* sh, cudaStream_t st) {
  const int G = ring_square_group(sh);
  if (!G || !sh->d_F2 || sh->nr % (G / 2) || (G / 2) % 2) return false;
  ProdArgs a;
  a.L = sh->lmax;
  a.nr = sh->nr;
  a.ntheta = sh->ntheta;
  a.npairs = sh->npairs;
  a.N = sh->nphi;
  a.nterms = sh->nterms;
  a.sp = sh->Cpad;
  a.sj = (int64_t)2 * (sh->lmax + 1) * sh->Cpad;
  a.gt_stride = sh->gt_stride;
  a.F1 = (const float*)sh->d_F;
  a.F2 = (const float*)sh->d_F2;
  a.GT = (__nv_bfloat16*)sh->d_GT;
  a.tw2 = (const float2*)sh->d_sqtw2;
  a.tw1 = (const float2*)sh->d_sqtw1;
  a.wgl = sh->d_wgl;
  switch (sh->nphi) {
    case 3200: launch_prod<25, 16, 8, 2, 4>(a, sh->sms, st); return true;
    case 3125: launch_prod<25, 25, 5, 2, 4>(a, sh->sms, st); return true;
    case 1600: launch_prod<25, 8, 8, 2, 8>(a, sh->sms, st); return true;
    case 800: launch_prod<25, 8, 4, 4, 8>(a, sh->sms, st); return true;
    case 400: launch_prod<25, 4, 4, 2, 8>(a, sh->sms, st); return true;
    default: return false;
  }
}

}  // namespace fnl
