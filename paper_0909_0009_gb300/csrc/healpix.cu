// HEALPix ring grid (Gorski et al. 2005), the grid of the paper's maps (Sect. 3), for the FP64
// and FP32 forms of the generator.  N_pix = 12 nside^2 equal-area pixels on 4 nside - 1 rings:
//   north cap, i < nside:          z = 1 - i^2 / (3 nside^2),  n_i = 4 i,      phi_0 = pi / (4 i)
//   belt, nside <= i <= 3 nside:   z = 4/3 - 2 i / (3 nside),  n_i = 4 nside,  phi_0 = s pi / (4 nside),
//                                  s = (i - nside + 1) mod 2
//   south cap, i > 3 nside:        the mirror of ring 4 nside - i
// Pixel k of ring i sits at phi_0 + 2 pi k / n_i; sphere integrals use the equal weight 4 pi / N_pix.
// Ring pair j (0 <= j < 2 nside) is ring j + 1 and its mirror (the equator, j = 2 nside - 1, pairs
// with itself), so the Legendre GEMMs are the Gauss-Legendre ones at other nodes.
//
// The ring transforms have lengths n = 4 i that need not be 2/3/5-smooth, so the ring kernel
// takes each ring's DFT by Bluestein's chirp-z algorithm (X_m = c_m sum_k (x_k c_k) conj(c_{m-k}),
// c_k = e^{-i pi k^2 / n}, a circular convolution of length M_j, the ring's own power of two
// >= 2 n - 1, by FFTs); the belt rings (n = 4 nside, a power of two) need none of it.
// Tables per ring pair: the chirp c_k (k < n), the M-point DFT of the filter b (b_j = conj(c_j) for
// 0 <= j < n and b_{M-j} = conj(c_j) for 0 < j < n, else 0), and e^{i m phi_0} for m <= l_max; all
// built in FP64 on the host (k^2 reduced modulo 2 n exactly before the angle is formed).
#include <cmath>
#include <complex>
#include <vector>

#include "fnl_internal.cuh"

namespace fnl {

namespace {

// In-place radix-2 DFT of a power-of-two length, X_m = sum_k x_k e^{-2 pi i m k / M}.
void host_fft(std::vector<std::complex<double>>& a) {
  const size_t M = a.size();
  for (size_t i = 1, j = 0; i < M; ++i) {
    size_t bit = M >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) std::swap(a[i], a[j]);
  }
  for (size_t len = 2; len <= M; len <<= 1) {
    const double ang = -2.0 * M_PI / (double)len;
    for (size_t i = 0; i < M; i += len)
      for (size_t k = 0; k < len / 2; ++k) {
        const std::complex<double> w(std::cos(ang * (double)k), std::sin(ang * (double)k));
        const std::complex<double> u = a[i + k], v = a[i + k + len / 2] * w;
        a[i + k] = u + v;
        a[i + k + len / 2] = u - v;
      }
  }
}

template <typename T>
void* upload_complex(fnl_shells* sh, const std::vector<std::complex<double>>& v) {
  std::vector<T> h(2 * v.size());
  for (size_t i = 0; i < v.size(); ++i) {
    h[2 * i] = (T)v[i].real();
    h[2 * i + 1] = (T)v[i].imag();
  }
  void* p = device_malloc(sizeof(T) * (h.size() ? h.size() : 1));
  sh->allocations.push_back(p);
  sh->device_bytes += sizeof(T) * h.size();
  FNL_CUDA(cudaMemcpy(p, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice));
  return p;
}

template <typename V>
V* upload_vec(fnl_shells* sh, const std::vector<V>& v) {
  void* p = device_malloc(sizeof(V) * (v.size() ? v.size() : 1));
  sh->allocations.push_back(p);
  sh->device_bytes += sizeof(V) * v.size();
  FNL_CUDA(cudaMemcpy(p, v.data(), sizeof(V) * v.size(), cudaMemcpyHostToDevice));
  return (V*)p;
}

template <typename T>
void build_tables(fnl_shells* sh) {
  const int nside = sh->nside, np = sh->npairs, L = sh->lmax, nmax = sh->hp_nmax;
  std::vector<double> z, phi0;
  std::vector<int> n;
  healpix_rings(nside, z, n, phi0);
  std::vector<int64_t> off(sh->ntheta + 1, 0);
  for (int i = 0; i < sh->ntheta; ++i) off[i + 1] = off[i] + n[i];
  sh->npix = off[sh->ntheta];
  std::vector<int> npair(n.begin(), n.begin() + np), e(np);
  std::vector<int64_t> bfoff(np);
  int64_t bftotal = 0;
  for (int j = 0; j < np; ++j) {
    int ej = 0;
    while ((1 << ej) < 2 * n[j] - 1) ++ej;
    e[j] = ej;
    bfoff[j] = bftotal;
    bftotal += (int64_t)1 << ej;
  }
  std::vector<std::complex<double>> rot((size_t)np * (L + 1)), chirp((size_t)np * nmax), bf((size_t)bftotal);
  for (int j = 0; j < np; ++j) {
    const int nj = n[j], M = 1 << e[j];
    for (int m = 0; m <= L; ++m) rot[(size_t)j * (L + 1) + m] = std::polar(1.0, (double)m * phi0[j]);
    for (int k = 0; k < nj; ++k) {
      const long long ee = ((long long)k * k) % (2LL * nj);
      chirp[(size_t)j * nmax + k] = std::polar(1.0, -M_PI * (double)ee / (double)nj);
    }
    std::vector<std::complex<double>> b(M, std::complex<double>(0.0, 0.0));
    for (int k = 0; k < nj; ++k) {
      const std::complex<double> c = std::conj(chirp[(size_t)j * nmax + k]);
      b[k] = c;
      if (k) b[M - k] = c;
    }
    host_fft(b);
    for (int k = 0; k < M; ++k) bf[(size_t)bfoff[j] + k] = b[k];
  }
  // twiddles of every power of two up to the longest Bluestein length
  std::vector<std::complex<double>> tw;
  for (int ee = 0; ee < fnl_shells::kHpPlans && (1 << ee) <= sh->hp_M; ++ee) {
    const int M = 1 << ee;
    sh->hp_twoff[ee] = (int64_t)tw.size();
    if (ee >= 1) sh->hp_plans[ee] = make_fft_plan(M);
    for (int k = 0; k < M; ++k) tw.push_back(std::polar(1.0, -2.0 * M_PI * (double)k / (double)M));
  }
  sh->d_hp_n = upload_vec(sh, npair);
  sh->d_hp_e = upload_vec(sh, e);
  sh->d_hp_bfoff = upload_vec(sh, bfoff);
  sh->d_hp_off = upload_vec(sh, off);
  sh->d_hp_rot = upload_complex<T>(sh, rot);
  sh->d_hp_chirp = upload_complex<T>(sh, chirp);
  sh->d_hp_bf = upload_complex<T>(sh, bf);
  sh->d_hp_tw = upload_complex<T>(sh, tw);
}

}  // namespace

void healpix_rings(int nside, std::vector<double>& z, std::vector<int>& n, std::vector<double>& phi0) {
  const int nr = 4 * nside - 1;
  z.resize(nr);
  n.resize(nr);
  phi0.resize(nr);
  for (int idx = 0; idx < nr; ++idx) {
    const int i = idx + 1;
    const int ii = i <= 2 * nside ? i : 4 * nside - i;  // the mirror ring of the south
    double zz, p0;
    int nn;
    if (ii < nside) {
      zz = 1.0 - (double)ii * ii / (3.0 * nside * nside);
      nn = 4 * ii;
      p0 = M_PI / (4.0 * ii);
    } else {
      const int s = (ii - nside + 1) % 2;
      zz = 4.0 / 3.0 - 2.0 * ii / (3.0 * nside);
      nn = 4 * nside;
      p0 = s * M_PI / (4.0 * nside);
    }
    z[idx] = i <= 2 * nside ? zz : -zz;
    n[idx] = nn;
    phi0[idx] = p0;
  }
}

void setup_healpix(fnl_shells* sh) {
  sh->hp_nmax = 4 * sh->nside;
  int M = 1;
  while (M < 2 * sh->hp_nmax - 1) M <<= 1;
  sh->hp_M = M;
  FNL_REQUIRE(M < (1 << fnl_shells::kHpPlans), "nside too large for the HEALPix ring kernel");
  const size_t ts = sh->real_is_double ? 16 : 8;
  FNL_REQUIRE(2 * ts * (size_t)M <= 227 * 1024, "nside too large for the HEALPix ring kernel's shared memory");
  if (sh->real_is_double) build_tables<double>(sh);
  else build_tables<float>(sh);
}

}  // namespace fnl
