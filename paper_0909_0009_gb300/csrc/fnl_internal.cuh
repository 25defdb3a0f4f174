// Internal declarations of libfnl (not part of the C ABI).
//
// Index conventions used by every kernel:
//   L = lmax, nr shells, C = 2 nr real columns (column c = 2 i + {0: re, 1: im} of shell i).
//   Legendre problems are indexed by mp = 2 m + p, p = parity of (l - m); problem (m, p)
//   holds the K_mp = max(0, (L - m - p + 2) / 2) degrees l = m + p + 2 k, k < K_mp.
//   Ring pairs jp < npairs = (ntheta + 1) / 2: north ring jp at x_jp >= 0, south ring
//   ntheta - 1 - jp at -x_jp (the same ring for the equator of an odd grid).
//   lambda_lm(-x) = (-1)^(l-m) lambda_lm(x) turns every transform into two half-size
//   contractions per m: even (p = 0) and odd (p = 1) degrees over the northern rings.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <functional>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

#include "fnl.h"
#include "tc_gemm.cuh"

namespace fnl {

// Ring pairs of an order m where every |lambda_lm| (l = m .. l_max) stays below this bound lie in
// the polar cap where the associated Legendre functions of that order decay; the tensor-core
// GEMMs leave them out.  The dropped terms change F_m by at most 2^-30 sum_l |a_lm| and the
// analysis by at most 2^-30 sum_j w_j |G_m(theta_j)|: below 1e-7 of either result, far under the
// BF16 split's 4e-6.
constexpr double kLambdaSkip = 0x1p-30;

// ---- error handling -----------------------------------------------------------------

struct Error : std::runtime_error {
  fnl_status code;
  Error(fnl_status c, const std::string& m) : std::runtime_error(m), code(c) {}
};

void set_last_error(const std::string& msg);

#define FNL_CUDA(call)                                                                  \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) {                                                            \
      throw ::fnl::Error(e_ == cudaErrorMemoryAllocation ? FNL_ENOMEM : FNL_ECUDA,      \
                         std::string(#call) + ": " + cudaGetErrorString(e_));           \
    }                                                                                   \
  } while (0)

#define FNL_REQUIRE(cond, msg)                                   \
  do {                                                           \
    if (!(cond)) throw ::fnl::Error(FNL_EINVAL, (msg));          \
  } while (0)

// ---- device memory of the set-up paths ---------------------------------------------------

// cudaMalloc of `bytes` (at least 1), throwing FNL_ENOMEM / FNL_ECUDA; when the allocation-failure
// test hook (fnl_test_fail_alloc) is armed, the chosen allocation fails instead, without calling
// cudaMalloc, so that the unwinding of every set-up path can be tested.
void* device_malloc(size_t bytes);

// A temporary device buffer of a set-up step, freed when it goes out of scope (also when the
// step throws).
struct TempDev {
  void* p = nullptr;
  explicit TempDev(size_t bytes) : p(device_malloc(bytes)) {}
  ~TempDev() {
    if (p) cudaFree(p);
  }
  TempDev(const TempDev&) = delete;
  TempDev& operator=(const TempDev&) = delete;
  template <typename T>
  T* as() const {
    return (T*)p;
  }
};

// ---- small helpers --------------------------------------------------------------------

template <typename T>
struct cplx {
  T x, y;
};

inline int64_t n_alm(int L) { return (int64_t)(L + 1) * (L + 2) / 2; }
__host__ __device__ inline int64_t alm_idx(int l, int m, int L) {
  return (int64_t)m * (2 * L + 1 - m) / 2 + l;
}
__host__ __device__ inline int k_of(int L, int m, int p) {
  int v = (L - m - p + 2) / 2;
  return v > 0 ? v : 0;
}
inline int round_up(int v, int q) { return (v + q - 1) / q * q; }

// Maximum number of FFT passes and the radices used.
constexpr int kMaxRadix = 24;

struct FftPlan {
  int n = 0;
  int nrad = 0;
  int rad[kMaxRadix];
  int toff[kMaxRadix];  // offset of pass p in the per-pass twiddle table
  int ttotal = 0;       // sum over passes of (R_p - 1) Ns_p
};

// Tile of a SIMT grouped GEMM: problem mp, row tile, column tile.
// Output tiles of the SIMT Legendre GEMMs: kSimtBM rows (ring pairs or degrees; kSimtBM64 in
// the FP64 form) x kSimtBN columns, kSimtBK-deep k steps; a tile's first k is a multiple of 16.
constexpr int kSimtBM = 128, kSimtBM64 = 64, kSimtBN = 64, kSimtBK = 8;
struct Tile {
  int mp, rt, ct;
  int q0;  // first k of the tile's k loop: the analysis's first ring pair (a multiple of 16), past
           // which the polar ring pairs of negligible lambda lie; a synthesis tile whose ring pairs
           // all lie there gets the padded depth, runs no k step and writes zeros
};

// ---- the shells object ---------------------------------------------------------------

// Host copies of a shells object's set-up data in FP64 (shared by its scratch clones):
// K_l [L+1][nr][nr] (lower; empty for a synthesis-only object), r, w [nr], alpha^T, alpha^E
// [L+1][nr] and v^X_l = K_l^T q^X_l [L+1][nr].
struct HostSetup {
  std::vector<double> K, r, w, alphaT, alphaE, vT, vE;
};

struct DeviceBuffer {
  void* p = nullptr;
  size_t bytes = 0;
};

}  // namespace fnl

struct fnl_shells {
  int device = 0;
  int lmax = 0, nr = 0, ntheta = 0, nphi = 0, prec = 0;
  int npairs = 0, C = 0;
  // shell shard: the object's nr shells are shells j0 .. j0 + nr - 1 of a configuration of
  // nr_total shells (j0 = 0 and nr_total = nr for a whole configuration)
  int j0 = 0, nr_total = 0;
  int64_t nalm = 0;
  bool real_is_double = true;  // SIMT real type: double (FP64) or float (FP32 and mixed)
  size_t device_bytes = 0;
  std::vector<void*> allocations;

  std::shared_ptr<const fnl::HostSetup> host;
  bool synth_only = false;     // internal object without filters (the estimator's synthesis)

  // problem geometry
  std::vector<int> K;          // [2(L+1)]
  std::vector<int> jmin;       // [L+1] tensor-core forms: first ring pair (from the pole) where some
                               // |lambda_lm| >= kLambdaSkip; the GEMMs leave out the ring pairs below
  std::vector<int> KP;         // K rounded up to 16
  std::vector<int64_t> row0;   // first row of problem mp in the [rows][C] phi buffer (SIMT)
  std::vector<int64_t> lam0;   // first element of problem mp in the SIMT lambda table
  int64_t rows_total = 0, lam_total = 0;
  int* d_K = nullptr;
  int64_t* d_row0 = nullptr;
  int64_t* d_lam0 = nullptr;

  // host copies of set-up data
  std::vector<double> x, wgl;      // [npairs] northern GL nodes and weights
  std::vector<double> mu;          // [nr]

  // device tables
  double* d_x = nullptr;           // [npairs]
  double* d_wgl = nullptr;         // [npairs]
  void* d_lam = nullptr;           // SIMT table, real type, [lam_total]
  void* d_Kf = nullptr;            // [L+1][nr][ncol] real type: row i holds K_l[j0 + i][0 .. ncol),
                                   // ncol = j0 + nr (the noise shells the object's rows need)
  void* d_Kterm = nullptr;         // tensor-core forms: BF16 [3 terms][L+1][128 j][128 i] of K_l[j0 + i][j]
  CUtensorMap tmK{};               // its tensor map (one box per degree: every term, both halves of i)
  double* d_vT = nullptr;          // [L+1][ncol]  v^X_l[j] = sum_i K_l[j0 + i][j] q^X_l[i]
  double* d_vE = nullptr;
  double* d_qT = nullptr;          // [L+1][nr]  q^X_l[i] = w_i r_i^2 alpha^X_l(r_i)
  double* d_qE = nullptr;
  float* d_qT32 = nullptr;         // FP32 copies of q^T, q^E (the adjoint's FP32 and tensor-core forms)
  float* d_qE32 = nullptr;
  double* d_mu = nullptr;          // [nr]
  void* d_tw = nullptr;            // [nphi] complex real type, e^{-2 pi i k / nphi}
  void* d_twp = nullptr;           // per-pass twiddles: pass p, [(r - 1) Ns_p + k] = e^{-2 pi i r k / (Ns_p R_p)}
  fnl::FftPlan fft;

  // scratch of the path
  void* d_phi = nullptr;           // [rows_total][C] real type
  void* d_F = nullptr;             // SIMT: [2(L+1)][npairs][C]; tensor-core forms: float [npairs][2(L+1)][Cpad]
  void* d_G = nullptr;             // [2(L+1)][npairs][C] real type
  double* d_aL = nullptr;          // [2][nalm][2]  a^T_L, a^E_L when the caller passes NULL
  double* d_aNL = nullptr;         // [2][nalm][2]
  double* d_aOut = nullptr;        // [2][nalm][2]  a^T, a^E of fnl_generate_host

  // per-stage timing of fnl_generate
  int ring_slots = 0;                 // 0: profiling off
  int ring_head = 0, ring_count = 0;  // next slot, profiled calls since the last read
  std::vector<cudaEvent_t> ring;      // [ring_slots][FNL_NSTAGES + 1]

  // mixed (tensor-core) forms
  int nterms = 0;                  // BF16 terms per operand (0: SIMT forms)
  int Cpad = 0;                    // columns padded to a multiple of 128
  int npj = 0;                     // ring pairs padded to a multiple of 32 (row stride of Lambda_ana)
  int nsyn = 0;                    // synthesis tile width (ring pairs)
  int nana = 0;                    // analysis tile width cap (degrees)
  int tc_split = 1;                // separate accumulators for leading and correction products
  int sms = 0;
  int sms_gemm = 0, sms_ring = 0;  // SMs the persistent GEMM and ring kernels may occupy (0: all)
  std::vector<int64_t> row32;      // first Phi row of problem mp (rows padded to 32)
  int64_t* d_row32 = nullptr;
  void* d_phiT = nullptr;          // bf16 [nterms][rows32][Cpad]
  int64_t phiT_stride = 0;
  void* d_lsyn = nullptr;          // bf16 [nterms][slabs][npairs][32]
  int64_t lsyn_stride = 0;
  void* d_lana = nullptr;          // bf16 [nterms][rows16][npj]
  int64_t lana_stride = 0;
  void* d_GT = nullptr;            // bf16 [nterms][npairs][2(L+1)][Cpad] (ring-pair-major)
  void* d_sqtw2 = nullptr;         // float2 twiddles of the specialised ring kernel (NULL: none for nphi)
  void* d_sqtw1 = nullptr;
  int64_t gt_stride = 0;
  void* d_part = nullptr;          // double2 [Cpad / 128][nalm][2]: quadrature partials per column tile
  float2* d_q2 = nullptr;          // [L+1][2][nre]  q^T, q^E as FP32 pairs (hi, lo), nre = nr rounded up to even
  void* d_F2 = nullptr;            // adjoint: the spectra of s, float as d_F (owner objects only)
  float* d_adjA = nullptr;         // adjoint: analysis of 2 f s per shell, [nalm][nr][2] (FP32 accumulators)
  CUtensorMap tmF2{};              // adjoint: tensor map of d_F2 for the synthesis's tensor stores
  int* d_err = nullptr;            // device error word of the tensor-core kernels
  double* d_psum = nullptr;        // [nr] sum_lm w_m |Phi_L,lm(r_i)|^2 (Parseval monopole)
  double* d_psum_part = nullptr;   // [(L+1) * 2][nr] the filter's partials of d_psum
  fnl::TcTile* d_tc_syn = nullptr;
  fnl::TcTile* d_tc_ana = nullptr;
  fnl::TcArgs tc_syn{}, tc_ana{};
  fnl::TcInst tci[2] = {};         // per-configuration GEMM arguments: synthesis, analysis
  fnl::TcInst* d_tci = nullptr;    // their device copy (TcArgs::insts)
  std::vector<fnl::TcTile> tiles_syn_h, tiles_ana_h;  // host copies of the tile lists
  int tiles_version = 0;           // incremented whenever the tile shape changes
  const fnl_shells* owner = nullptr;  // set on scratch clones: the object whose tables they use

  // Stokes maps (fnl_maps): lambda, W, X in the SIMT table layout (real type) and the ring
  // sums F [2(L+1)][npairs][6] of I, Q, U; allocated by fnl_maps_prepare
  bool maps_ready = false;
  void* d_mapL = nullptr;
  void* d_mapW = nullptr;
  void* d_mapX = nullptr;
  void* d_Fiqu = nullptr;
  int* d_maps_jmin = nullptr;      // [L+1] first ring pair where some |lambda|, |W|, |X| of order m
                                   // reaches the maps' bound (2^-30 FP32 tables, 2^-60 FP64)

  // HEALPix ring grid (nside > 0; FP64 and FP32 forms): ring pair j = ring j + 1 and its mirror
  int nside = 0;
  int hp_M = 0;                    // longest Bluestein FFT: a power of two >= 2 (4 nside) - 1
  int hp_nmax = 0;                 // longest ring, 4 nside
  int64_t npix = 0;                // 12 nside^2
  static constexpr int kHpPlans = 14;
  fnl::FftPlan hp_plans[kHpPlans]; // plan of the power-of-two length 2^e
  int64_t hp_twoff[kHpPlans] = {}; // offset of the twiddles of 2^e in d_hp_tw
  int* d_hp_n = nullptr;           // [npairs] ring lengths
  int* d_hp_e = nullptr;           // [npairs] log2 of the ring's Bluestein length M_j >= 2 n_j - 1
  int64_t* d_hp_bfoff = nullptr;   // [npairs] offset of the ring's filter DFT in d_hp_bf
  int64_t* d_hp_off = nullptr;     // [ntheta + 1] first pixel of each ring (RING order)
  void* d_hp_rot = nullptr;        // [npairs][L+1] complex: e^{i m phi_0}
  void* d_hp_chirp = nullptr;      // [npairs][hp_nmax] complex: e^{-i pi k^2 / n}
  void* d_hp_bf = nullptr;         // per ring pair, M_j complex: DFT_{M_j} of the chirp filter
  void* d_hp_tw = nullptr;         // per power of two 2^e: e^{-2 pi i k / 2^e}, k < 2^e

  // SIMT tile lists
  fnl::Tile* d_tiles_syn = nullptr;
  int n_tiles_syn = 0;
  fnl::Tile* d_tiles_ana = nullptr;
  int n_tiles_ana = 0;
};

namespace fnl {

// ---- entry-point plumbing (fnl_api.cu) -----------------------------------------------------
// Runs `body`, turning exceptions into a status and the thread's last-error message.
fnl_status guard(const std::function<void()>& body);
// Makes `dev` current for the scope and restores the caller's device on exit.
struct DeviceScope {
  int prev = -1;
  explicit DeviceScope(int dev);
  ~DeviceScope();
};
void check_dev_ptr(const void* p, const char* name, bool nullable);
void check_shells(const fnl_shells* sh);
// Steps (i)-(v) of one realisation; NULL outputs go to the object's scratch.  `mark` records
// the per-stage profiling events when profiling is on.
void run_generate(const fnl_shells* sh, uint64_t seed, uint64_t realisation, double fnl, const double* noise,
                  double* aT, double* aE, double* aLT, double* aLE, double* aNLT, double* aNLE, cudaStream_t st,
                  bool mark = true);
// Tile shapes of the tensor-core GEMMs (mixed forms): widths capped at syn_cap ring pairs and
// ana_cap degrees, multiples of 16 in [kTcMinWidth, 256].
constexpr int kTcMinWidth = 64;
void configure_tc(fnl_shells* sh, int syn_cap, int ana_cap, bool exact = false);
// A shells object of the tensor-core forms that shares src's tables and tile lists but owns
// its scratch (so that several realisations of one configuration can run at once), and the
// step that copies src's current tile shape into it.  Freed with destroy_clone.
fnl_shells* clone_scratch(const fnl_shells* src);
void refresh_clone(fnl_shells* c, const fnl_shells* src);
void destroy_clone(fnl_shells* c);
void build_tc_inst_a(fnl_shells* sh);
// fnl_make_shells; with synth_only, an object without filters (K, mu, q and v zero) of up to
// 256 fields, used for the synthesis of other fields (the estimator's A and B maps).
// j0, j1: the shell shard [j0, j1) of the configuration (j1 < 0: every shell).
fnl_shells* make_shells_core(const fnl_shell_desc* d, int device, bool synth_only, int nside = 0, int j0 = 0,
                             int j1 = -1);
// HEALPix rings (healpix.cu): z, ring length and phi offset of rings 1 .. 4 nside - 1 (north to
// south); the per-ring-pair tables of the HEALPix ring kernel.
void healpix_rings(int nside, std::vector<double>& z, std::vector<int>& n, std::vector<double>& phi0);
void setup_healpix(fnl_shells* sh);
// Frees an object made by make_shells_core (its device memory and the object).
void release_shells(fnl_shells* sh);
// Step (ii) Legendre GEMM of the object's own Phi rows (tensor-core or SIMT form) into F.
void launch_synthesis_gemm(const fnl_shells* sh, cudaStream_t st);
void build_tc_inst_b(fnl_shells* sh);

// ---- host set-up (setup_host.cpp) -------------------------------------------------------
void gauss_legendre(int n, double* x, double* w);
void covariance(int lmax, int nr, const double* r, double A, double ns, double kmin, double kmax,
                int nk, double* C);
void cholesky_filters(int lmax, int nr, const double* C, double jitter_rel, double* K);
FftPlan make_fft_plan(int n);

// ---- kernel launchers (simt_path.cu, ring_fft.cu, tables.cu) ---------------------------
void build_lambda_tables(fnl_shells* sh, cudaStream_t st);
void launch_filter(const fnl_shells* sh, uint64_t seed, uint64_t real, const double* noise,
                   double* aLT, double* aLE, double* phi_api, cudaStream_t st);
void launch_synth_gemm(const fnl_shells* sh, cudaStream_t st);
void launch_synth_gemm_to(const fnl_shells* sh, void* out, cudaStream_t st);  // SIMT: phi rows -> out
void launch_analysis_gemm(const fnl_shells* sh, cudaStream_t st);
enum FftMode { FFT_SQUARE = 0, FFT_SYNTH_MAP = 1, FFT_ANALYSE_MAP = 2 };
bool launch_ring_square(const fnl_shells* sh, cudaStream_t st);
void ring_square_tables(int nphi, std::vector<float>& tw2, std::vector<float>& tw1);
void launch_ring_fft(const fnl_shells* sh, int mode, const double* maps_in, double* maps_out,
                     cudaStream_t st);
void launch_alm_to_phi(const fnl_shells* sh, const double* alm, cudaStream_t st);
void launch_phi_to_alm(const fnl_shells* sh, double* alm, cudaStream_t st);
void launch_quadrature(const fnl_shells* sh, const double* phi_api, int from_internal, double fnl,
                       const double* aLT, const double* aLE, double* aT, double* aE,
                       double* aNLT, double* aNLE, int accumulate_into_L, cudaStream_t st);
void launch_combine(const fnl_shells* sh, double fnl, const double* aLT, const double* aLE,
                    const double* aNLT, const double* aNLE, double* aT, double* aE,
                    cudaStream_t st);
// Ring synthesis of nf complex fields F [2(L+1)][npairs][2 nf] (problem 2 m + parity; the
// odd problem of m = L included) into maps [nf][ntheta][nphi].
void launch_ring_synth_fields(const fnl_shells* sh, const void* F, int nf, double* maps, cudaStream_t st);
// Estimator rings (ring_fft.cu): fields 0..nsh-1 (A) and nsh..2nsh-1 (B) of the object's F;
// part [nsh][npairs] = w^GL_j sum_k A B^2 on ring pair j (both rings).
void launch_ring_cubic(const fnl_shells* sh, int nsh, double* part, cudaStream_t st);
// The same with the specialised ring kernel of the tensor-core forms (ring_square.cu); false if
// the object's ring length has none.
bool launch_ring_cubic_sq(const fnl_shells* sh, int nsh, double* part, cudaStream_t st);
// Specialised adjoint rings of the tensor-core forms (ring_square.cu): 2 f s from the spectra of f
// (d_F) and s (d_F2) into d_GT; false if the object's ring length has none.
bool launch_ring_product_sq(const fnl_shells* sh, cudaStream_t st);
// Stokes maps (maps.cu): tables once, then I, Q, U of one set of a_lm.
void maps_prepare(fnl_shells* sh);
void launch_maps(const fnl_shells* sh, const double* aT, const double* aE, const double* aB, double* maps,
                 cudaStream_t st);
void launch_lambda_mm(const double* x, const double* fac, int npairs, int L, double* mant, int* expo,
                      cudaStream_t st);

// ---- adjoint of the SIMT forms (adjoint.cu, ring_fft.cu) -------------------------------------
void launch_adjoint_source(const fnl_shells* sh, double fnl, const double* gT, const double* gE, cudaStream_t st);
void launch_ring_product(const fnl_shells* sh, cudaStream_t st);
void launch_adjoint_filter(const fnl_shells* sh, const double* gT, const double* gE, double* grad_noise,
                           cudaStream_t st);
void launch_dot_fnl(const fnl_shells* sh, const double* gT, const double* gE, const double* aNLT,
                    const double* aNLE, double* out, cudaStream_t st);

// ---- several instances (configurations or realisations) in one launch (batch.cu) ----------

// Per-launch outputs of up to kTcMaxInst instances (kernel parameters).
struct MultiOut {
  double fnl[kTcMaxInst];
  double2* aT[kTcMaxInst];
  double2* aE[kTcMaxInst];
};
// Step (v) of one instance.
struct CombineInst {
  int64_t nalm;
  int nct, nr;
  const double2* part;  // [nct][nalm][2]
  const double* psum;
  const double* mu;
  const double* qT;
  const double* qE;
  const double2* aLT;
  const double2* aLE;
  double2* aNLT;
  double2* aNLE;
};
// Specialised ring kernel (ring_square.cu): shell-group size if this configuration has one
// (else 0), the size and contents of its argument block, and one launch over instances.
int ring_square_group(const fnl_shells* sh);
size_t ring_square_args_size();
void ring_square_args(const fnl_shells* sh, void* out);
void launch_ring_square_multi(const fnl_shells* proto, const void* d_inst, const int* d_item0, int ninst, int maxL,
                              int items, cudaStream_t st);
void launch_combine_multi(const CombineInst* inst, int64_t max_nalm, int ninst, const MultiOut& out, cudaStream_t st);

// ---- mixed-precision forms (mixed_path.cu, tc_gemm.cu) -------------------------------------
void build_lambda_tables_mixed(fnl_shells* sh, cudaStream_t st);
// Tensor-core filter (filter_tc.cu): the BF16 terms of K_l and their tensor map (set-up; Kf is
// [L+1][nr][ncol] as d_Kf), and step (i) with monopole partials psum_part [L+1][2][nr].
void build_filter_terms(fnl_shells* sh, const std::vector<double>& Kf);
void launch_filter_tc(const fnl_shells* sh, uint64_t seed, uint64_t real, const double* noise, double* aLT,
                      double* aLE, double* phi_api, double* psum_part, cudaStream_t st);
void launch_filter_mixed(const fnl_shells* sh, uint64_t seed, uint64_t real, const double* noise, double* aLT,
                         double* aLE, double* phi_api, double* psum, cudaStream_t st);
void launch_alm_to_terms(const fnl_shells* sh, const double* alm, cudaStream_t st);
void launch_combine_mixed(const fnl_shells* sh, double fnl, const double* aLT, const double* aLE, double* aNLT,
                          double* aNLE, double* aT, double* aE, const double* psum, cudaStream_t st);

}  // namespace fnl
