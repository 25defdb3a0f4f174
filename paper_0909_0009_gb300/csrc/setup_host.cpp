// Host-side set-up of libfnl (Sect. 3: auxiliary data computed once per configuration):
// Gauss-Legendre rule, radial covariance of Eq. 7 and its Cholesky filters (Eq. 9),
// FFT factorisation.  Plain C++ (OpenMP over independent items), FP64 throughout.
#include <cmath>
#include <cstring>
#include <vector>

#include "fnl_internal.cuh"

namespace fnl {

// n-point Gauss-Legendre rule by Newton's method on P_n (Bonnet recurrence for P_n and
// P_{n-1}, P_n' = n (x P_n - P_{n-1}) / (x^2 - 1)); nodes north to south.  The rule is
// symmetrised: x_{n-1-j} = -x_j, and the middle node of an odd rule is exactly 0.
void gauss_legendre(int n, double* x, double* w) {
  const double pi = 3.14159265358979323846;
  std::vector<double> xs(n), ws(n);
#pragma omp parallel for schedule(static)
  for (int j = 0; j < n; ++j) {
    double z = std::cos(pi * (j + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) { p0 = 1.0; p1 = z; }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    xs[j] = z;
  }
  for (int j = 0; j < n; ++j) x[j] = 0.5 * (xs[j] - xs[n - 1 - j]);
  if (n % 2 == 1) x[n / 2] = 0.0;
#pragma omp parallel for schedule(static)
  for (int j = 0; j < n; ++j) {
    double z = x[j], p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) {
      double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    if (n == 1) { p0 = 1.0; p1 = z; }
    double dp = n * (z * p1 - p0) / (z * z - 1.0);
    ws[j] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
  for (int j = 0; j < n; ++j) w[j] = 0.5 * (ws[j] + ws[n - 1 - j]);
}

// Spherical Bessel j_l(x), l = 0..L, into out[l * stride].
//  x > L + 60: upward recurrence from j_0, j_1 (stable while l < x).
//  otherwise:  Miller's downward recurrence from N = L + 200 + x with j_{N+1} = 0, j_N = 1,
//              rescaled by 2^-400 whenever it passes 2^400, normalised by
//              sum_l (2l+1) j_l^2 = 1 and signed by j_0 (or j_1 where j_0 is small).
static void sph_bessel(int L, double x, double* out, size_t stride, std::vector<double>& mant,
                       std::vector<int>& ex) {
  const double s = std::sin(x), c = std::cos(x);
  const double j0 = s / x, j1 = s / (x * x) - c / x;
  if (x > L + 60.0) {
    out[0] = j0;
    if (L >= 1) out[stride] = j1;
    double a = j0, b = j1;
    for (int l = 1; l < L; ++l) {
      double nb = (2.0 * l + 1.0) / x * b - a;
      a = b;
      b = nb;
      out[(size_t)(l + 1) * stride] = b;
    }
    return;
  }
  const int N = L + 200 + (int)x;
  mant.assign(L + 1, 0.0);
  ex.assign(L + 1, 0);
  double yn = 0.0, y = 1.0, sum = 0.0;
  int e = 0;
  for (int l = N; l >= 1; --l) {
    if (l <= L) { mant[l] = y; ex[l] = e; }
    sum += (2.0 * l + 1.0) * y * y;
    double yp = (2.0 * l + 1.0) / x * y - yn;
    yn = y;
    y = yp;
    if (std::fabs(y) > 0x1p400) {
      y *= 0x1p-400;
      yn *= 0x1p-400;
      sum *= 0x1p-800;
      e += 400;
    }
  }
  mant[0] = y;
  ex[0] = e;
  sum += y * y;
  const double norm = 1.0 / std::sqrt(sum);
  double ref_true, ref_num;
  if (std::fabs(j0) > 0.1 * std::fabs(j1) || L < 1) {
    ref_true = j0;
    ref_num = mant[0] * norm;
  } else {
    ref_true = j1;
    ref_num = std::ldexp(mant[1] * norm, ex[1] - e);
  }
  const double sign = ((ref_true >= 0) == (ref_num >= 0)) ? 1.0 : -1.0;
  for (int l = 0; l <= L; ++l) {
    double v = sign * std::ldexp(mant[l] * norm, ex[l] - e);
    out[(size_t)l * stride] = std::fabs(v) < 1e-290 ? 0.0 : v;
  }
}

// C_l(r_i, r_j) = (2/pi) sum_k wk k^2 A k^(ns-4) j_l(k r_i) j_l(k r_j) on the uniform trapezoid
// rule with nk points over [kmin, kmax] (Eq. 7 with Eq. 8 and P(k) = A k^(ns-4)).
void covariance(int L, int nr, const double* r, double A, double ns, double kmin, double kmax,
                int nk, double* C) {
  const double pi = 3.14159265358979323846;
  const double h = (kmax - kmin) / (nk - 1);
  const int KC = 128;
  std::memset(C, 0, sizeof(double) * (size_t)(L + 1) * nr * nr);
  std::vector<double> J((size_t)(L + 1) * KC * nr);  // [l][k in chunk][i]
  std::vector<double> pk(KC);
  for (int k0 = 0; k0 < nk; k0 += KC) {
    const int kc = std::min(KC, nk - k0);
    for (int q = 0; q < kc; ++q) {
      const int kk = k0 + q;
      const double k = (kk == nk - 1) ? kmax : kmin + kk * h;
      const double wk = (kk == 0 || kk == nk - 1) ? 0.5 * h : h;
      pk[q] = (2.0 / pi) * wk * k * k * A * std::pow(k, ns - 4.0);
    }
#pragma omp parallel
    {
      std::vector<double> mant;
      std::vector<int> ex;
#pragma omp for schedule(dynamic, 16)
      for (int t = 0; t < kc * nr; ++t) {
        const int q = t / nr, i = t % nr;
        const int kk = k0 + q;
        const double k = (kk == nk - 1) ? kmax : kmin + kk * h;
        sph_bessel(L, k * r[i], &J[(size_t)q * nr + i], (size_t)KC * nr, mant, ex);
      }
    }
#pragma omp parallel for schedule(dynamic, 4)
    for (int l = 0; l <= L; ++l) {
      double* Cl = C + (size_t)l * nr * nr;
      const double* Jl = &J[(size_t)l * KC * nr];
      for (int q = 0; q < kc; ++q) {
        const double* v = Jl + (size_t)q * nr;
        for (int i = 0; i < nr; ++i) {
          const double s = pk[q] * v[i];
          if (s == 0.0) continue;
          double* row = Cl + (size_t)i * nr;
          for (int j = 0; j <= i; ++j) row[j] += s * v[j];
        }
      }
    }
  }
#pragma omp parallel for schedule(static)
  for (int l = 0; l <= L; ++l) {
    double* Cl = C + (size_t)l * nr * nr;
    for (int i = 0; i < nr; ++i)
      for (int j = i + 1; j < nr; ++j) Cl[(size_t)i * nr + j] = Cl[(size_t)j * nr + i];
  }
}

// K_l = chol(C_l + eps_l I), eps_l = jitter_rel * mean(diag C_l): lower triangular,
// upper triangle set to zero.  Throws FNL_EINVAL if a pivot is not positive.
void cholesky_filters(int L, int nr, const double* C, double jitter_rel, double* K) {
  int bad = -1;
#pragma omp parallel for schedule(dynamic, 4)
  for (int l = 0; l <= L; ++l) {
    const double* Cl = C + (size_t)l * nr * nr;
    double* Kl = K + (size_t)l * nr * nr;
    double tr = 0.0;
    for (int i = 0; i < nr; ++i) tr += Cl[(size_t)i * nr + i];
    const double eps = jitter_rel * tr / nr;
    for (int i = 0; i < nr; ++i) {
      for (int j = 0; j <= i; ++j) {
        double s = Cl[(size_t)i * nr + j] + (i == j ? eps : 0.0);
        for (int k = 0; k < j; ++k) s -= Kl[(size_t)i * nr + k] * Kl[(size_t)j * nr + k];
        if (i == j) {
          if (!(s > 0.0)) {
#pragma omp critical
            bad = l;
            s = 1.0;
          }
          Kl[(size_t)i * nr + i] = std::sqrt(s);
        } else {
          Kl[(size_t)i * nr + j] = s / Kl[(size_t)j * nr + j];
        }
      }
      for (int j = i + 1; j < nr; ++j) Kl[(size_t)i * nr + j] = 0.0;
    }
  }
  if (bad >= 0)
    throw Error(FNL_EINVAL, "covariance of l = " + std::to_string(bad) +
                                " is not positive definite (raise jitter_rel)");
}

FftPlan make_fft_plan(int n) {
  FftPlan p;
  p.n = n;
  int v = n;
  while (v % 8 == 0 && p.nrad < kMaxRadix) { p.rad[p.nrad++] = 8; v /= 8; }
  while (v % 4 == 0 && p.nrad < kMaxRadix) { p.rad[p.nrad++] = 4; v /= 4; }
  while (v % 2 == 0 && p.nrad < kMaxRadix) { p.rad[p.nrad++] = 2; v /= 2; }
  while (v % 3 == 0 && p.nrad < kMaxRadix) { p.rad[p.nrad++] = 3; v /= 3; }
  while (v % 5 == 0 && p.nrad < kMaxRadix) { p.rad[p.nrad++] = 5; v /= 5; }
  if (v != 1) throw Error(FNL_EINVAL, "nphi = " + std::to_string(n) + " is not 2/3/5-smooth");
  int ns = 1, off = 0;
  for (int i = 0; i < p.nrad; ++i) {
    p.toff[i] = off;
    off += (p.rad[i] - 1) * ns;
    ns *= p.rad[i];
  }
  p.ttotal = off;
  return p;
}

}  // namespace fnl
