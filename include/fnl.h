/*
 * fnl.h -- C ABI of libfnl: the local-f_NL a_lm generator of Elsner & Wandelt,
 * "Improved simulation of non-Gaussian temperature and polarization CMB maps",
 * run on one NVIDIA GB300 (sm_103a).
 *
 * The method (Sect. 2, recipe steps (i)-(v)):
 *   (i)   Phi_L,lm(r_i) = sum_j K_l[i,j] n_lm(r_j)                 Eq. 9, K_l K_l^T = P_Phi,l (Eq. 7)
 *   (ii)  per shell r_i, synthesis of Phi_L on a Gauss-Legendre ring grid
 *   (iii) Phi_NL = Phi_L^2 - <Phi_L^2>                              Eq. 2
 *   (iv)  per shell, analysis of Phi_NL back to harmonic space
 *   (v)   a^X_lm = sum_i w_i r_i^2 alpha^X_l(r_i) Phi_lm(r_i)       Eq. 5, X in {T, E}
 *         a^X = a^X_L + f_NL a^X_NL                                  Eq. 3
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Spherical harmonics Y_lm(theta, phi) = lambda_lm(cos theta) e^{i m phi}, orthonormal,
 *    Condon-Shortley phase.  Fields are real, so only m >= 0 is stored.
 *  - a_lm layout ("m-major triangle"): entry (l, m), 0 <= m <= l <= lmax, sits at
 *        idx(l, m) = m (2 lmax + 1 - m) / 2 + l,   nalm = (lmax + 1)(lmax + 2) / 2,
 *    each entry a complex128 stored as two doubles (re, im).
 *  - Per-shell coefficient arrays ("phi" arrays) are [nalm][nr][2] doubles: shell index
 *    innermost.  Noise arrays are [nr][nalm][2] doubles (shell outermost).
 *  - Maps are [nr][ntheta][nphi] doubles: ring j at x_j = cos theta_j, Gauss-Legendre nodes
 *    ordered north to south, phi_k = 2 pi k / nphi.
 *  - Pointers documented "device" must be device memory of the device the shells object
 *    was made on; "host" pointers are ordinary host memory.  The caller owns every buffer
 *    it passes.  The library owns only what fnl_make_shells allocates (tables and the
 *    scratch used by the path), freed by fnl_shells_destroy.
 *  - Every call except fnl_make_shells and fnl_shells_destroy is asynchronous on the
 *    caller's CUDA stream (`stream`, a cudaStream_t; NULL = legacy default stream),
 *    allocates nothing and does not synchronise.  Calls that share one shells object
 *    share its scratch: they must not overlap on the GPU (use one stream, or order them).
 *  - Errors: every call returns an fnl_status; on failure fnl_last_error() returns a
 *    message (thread-local, valid until the next call on that thread).  Argument
 *    errors are detected on the host before anything is launched.  No C++ exception
 *    crosses this boundary.
 */
#ifndef FNL_H
#define FNL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fnl_shells fnl_shells; /* opaque: device tables + scratch for one configuration */

typedef enum {
  FNL_OK = 0,
  FNL_EINVAL = 1,       /* invalid argument (size, pointer, grid) */
  FNL_ENOMEM = 2,       /* device or host allocation failed */
  FNL_ECUDA = 3,        /* a CUDA runtime/driver call failed */
  FNL_EUNSUPPORTED = 4, /* valid request this build or device cannot run */
  FNL_ETIMEOUT = 5      /* a bounded device-side wait expired */
} fnl_status;

typedef enum {
  FNL_FP64 = 0,   /* every step in FP64 (SIMT DFMA) */
  FNL_FP32 = 1,   /* Legendre, filter and FFT in FP32 (SIMT); tables and quadrature in FP64 */
  FNL_BF16X2 = 2, /* Legendre GEMMs on tcgen05 tensor cores, operands split into 2 BF16 terms
                     (3 products), FP32 accumulation; FFT and filter in FP32; tables and
                     quadrature in FP64 */
  FNL_BF16X3 = 3  /* as FNL_BF16X2 with 3 BF16 terms (6 products) */
} fnl_precision;

/* Description of one configuration (host memory; read during fnl_make_shells only). */
typedef struct {
  int lmax;    /* band limit, 1 <= lmax <= 4096 */
  int nr;      /* number of radial shells, 1 <= nr <= 128 */
  int ntheta;  /* Gauss-Legendre rings, ntheta >= lmax + 1 (exact square needs (3 lmax + 2) / 2) */
  int nphi;    /* points per ring, 2/3/5-smooth, nphi >= 2 lmax + 2 (exact square needs 3 lmax + 1) */
  const double* r;      /* host [nr]: radial nodes r_i (Mpc) */
  const double* w;      /* host [nr]: radial quadrature weights w_i */
  const double* K;      /* host [lmax+1][nr][nr] row-major filters K_l (lower triangle used), or
                           NULL: K_l = chol(C_l + eps_l I) built from the covariance below */
  double A, ns;         /* P(k) = A k^(ns - 4) (Eq. 7 with Eq. 8) */
  double kmin, kmax;    /* k range of the trapezoid rule (Mpc^-1) */
  int nk;               /* number of k points (>= 2) */
  double jitter_rel;    /* eps_l = jitter_rel * mean(diag C_l) */
  const double* alphaT; /* host [lmax+1][nr]: alpha^T_l(r_i) (Eq. 6 kernel for temperature) */
  const double* alphaE; /* host [lmax+1][nr]: alpha^E_l(r_i) (E-mode polarization) */
  const double* mu;     /* host [nr]: <Phi_L^2(r_i)> of Eq. 2, or NULL: the ensemble value
                           mu_i = sum_l (2l+1)/(4 pi) (K_l K_l^T)_ii */
  int prec;             /* fnl_precision */
} fnl_shell_desc;

/* The same on the HEALPix grid of the paper's maps (Sect. 3; Gorski et al. 2005): 12 nside^2
 * equal-area pixels on 4 nside - 1 iso-latitude rings (ring i < nside at z = 1 - i^2/(3 nside^2)
 * with 4 i pixels, belt rings at z = 4/3 - 2 i/(3 nside) with 4 nside pixels, pixel k at
 * phi_0 + 2 pi k / n_i, phi_0 = pi/(4 i) in the caps and alternately pi/(4 nside) and 0 in the
 * belt), sphere integrals by the equal weight 4 pi / N_pix (approximate: the analysis of a
 * synthesis returns a_lm up to an error falling as nside^-2).  desc->ntheta and desc->nphi are
 * ignored; any lmax is allowed (the short polar rings alias m > n_i / 2).  nside a power of two;
 * FNL_FP64 and FNL_FP32 only (FNL_EINVAL otherwise).  fnl_synth / fnl_analyse maps are
 * [nr][12 nside^2] in RING order.  The Stokes maps, the estimator and the adjoint run on the
 * Gauss-Legendre grid only (FNL_EUNSUPPORTED here). */
fnl_status fnl_make_shells_healpix(const fnl_shell_desc* desc, int nside, int device, fnl_shells** out);

/* A shell shard of a configuration: the object runs steps (i)-(v) for shells j0 .. j1 - 1 of
 * `desc` (desc->nr shells in all, 0 <= j0 < j1 <= desc->nr) and for no other, so that the work
 * of one realisation can be spread over several devices.  The paper keeps the seeds so that
 * Phi_L can be regenerated at any radius (Sect. 3); here each shard draws, from the same
 * counter-based generator, the noise of the shells its rows of K_l reach (0 .. j1 - 1), and
 * K_l, mu, q^X and v^X are those of the whole configuration restricted to the shard's rows.
 * fnl_generate's outputs are then partial sums: Eq. 5 and Eq. 3 are sums over shells, so
 * a^X_L, a^X_NL and a^X summed over shards that partition 0 .. nr - 1 equal the whole
 * configuration's up to the rounding order of those sums.  Per-shell inputs and outputs
 * (fnl_filter, fnl_synth, fnl_analyse, fnl_square, fnl_accumulate) are the shard's shells, and
 * an explicit `noise` is [j1][nalm][2] (shells 0 .. j1 - 1 of the configuration).  The
 * Gauss-Legendre grid and every precision form; fnl_shells_info reports the shard's nr.
 * fnl_generate_backward and fnl_ksw_create return FNL_EUNSUPPORTED for a shard, and a batch
 * runs shards in stream mode.  FNL_EINVAL for a range outside 0 <= j0 < j1 <= desc->nr. */
fnl_status fnl_make_shells_shard(const fnl_shell_desc* desc, int j0, int j1, int device, fnl_shells** out);

/* The shard of an object (any pointer may be NULL): its first shell j0, its shell count nr
 * and the configuration's nr_total (j0 = 0 and nr = nr_total for fnl_make_shells). */
fnl_status fnl_shells_shard(const fnl_shells* sh, int* j0, int* nr, int* nr_total);

/* Library version string. */
const char* fnl_version(void);

/* Message of the last failed call on this thread ("" if none). */
const char* fnl_last_error(void);

/* ---- set-up (S0; Sect. 3: auxiliary data computed once per configuration) ---------- */

/* Build the device tables for `desc` on CUDA device `device`: Gauss-Legendre grid,
 * lambda_lm(x_j) tables (FP64 three-term recurrence, converted to the precision's
 * operand format), filters K_l (Eq. 9), quadrature weights q^X_l[i] = w_i r_i^2
 * alpha^X_l(r_i) (Eq. 5), v^X_l = K_l^T q^X_l, mu_i (Eq. 2), FFT twiddles and the
 * scratch of the path.  Synchronous; allocates.  *out receives the object. */
fnl_status fnl_make_shells(const fnl_shell_desc* desc, int device, fnl_shells** out);

/* Free everything fnl_make_shells allocated (NULL is ignored).  Synchronous. */
void fnl_shells_destroy(fnl_shells* sh);

/* Sizes of a shells object: any pointer may be NULL. */
fnl_status fnl_shells_info(const fnl_shells* sh, int* lmax, int* nr, int* ntheta, int* nphi,
                           int* prec, size_t* device_bytes);

/* Copy mu_i (host [nr]) used by the object. */
fnl_status fnl_shells_mu(const fnl_shells* sh, double* mu_out);

/* ---- the hot path (S1-S5) ---------------------------------------------------------- */

/* One realisation, Sect. 2 steps (i)-(v), entirely on the device.
 *  seed, realisation: key of the counter-based noise (Philox4x64-10): the noise of shell j
 *      and entry idx comes from counter (idx, j >> 2, realisation, 0), key (seed, 0), output
 *      word j & 3, whose two 32-bit halves are the Box-Muller uniforms ((hi + 1) 2^-32 and
 *      lo 2^-32); m > 0 entries get unit complex variance, m = 0 entries are real N(0, 1).
 *      FNL_FP64 evaluates the Box-Muller transform in FP64, FNL_FP32 in FP32, and the
 *      tensor-core forms in FP32 with approximate transcendentals (absolute error < 2^-21).
 *  fnl:   f_NL of Eq. 1.
 *  noise: device [nr][nalm][2] explicit n_lm(r_j) (imaginary part of m = 0 ignored; a shell
 *      shard [j0, j1) reads [j1][nalm][2]), or NULL to draw it from (seed, realisation).
 *  aT, aE:     device [nalm][2]: a^X = a^X_L + f_NL a^X_NL (Eq. 3), or NULL.
 *  aLT, aLE:   device [nalm][2]: a^X_L (Eq. 5 applied to Phi_L), or NULL.
 *  aNLT, aNLE: device [nalm][2]: a^X_NL (Eq. 5 applied to Phi_NL), or NULL.
 * Accumulation of the radial quadrature is FP64 in every precision. */
fnl_status fnl_generate(const fnl_shells* sh, uint64_t seed, uint64_t realisation, double fnl,
                        const double* noise, double* aT, double* aE, double* aLT, double* aLE,
                        double* aNLT, double* aNLE, void* stream);

/* Adjoint of fnl_generate (the differentiation form).  For a real loss L of a^T and a^E:
 *  gT, gE: device [nalm][2] dL/da^X as pairs (dL/dRe, dL/dIm), or NULL for zero.
 *  grad_noise: device [nr][nalm][2], or NULL: dL/dn for the noise n of the same call
 *      (explicit `noise`, else the Philox draw of seed and realisation); the imaginary part
 *      of every m = 0 entry is 0, as the forward ignores it.
 *  grad_fnl: device double, or NULL: dL/df_NL = sum_X <gX, a^X_NL>.
 *  aNLT, aNLE: device [nalm][2] a^X_NL of the forward call, or NULL: then they are
 *      recomputed (one more forward pass) when grad_fnl is requested.
 * The chain rule through steps (i)-(v) (Eq. 9, the synthesis, Eq. 2, the analysis, Eq. 5,
 * Eq. 3), with mu a constant: dL/dPhi_NL = f_NL q^X gX; dL/dPhi_L = c_m analysis(2 f s) +
 * q^X gX, s the synthesis of dL/dPhi_NL with m > 0 halved, c_0 = 1 and c_m = 2; dL/dn =
 * K_l^T dL/dPhi_L.  The maps f and s are recomputed on the ring grid, not stored.  Every
 * precision form on the Gauss-Legendre grid: the tensor-core forms run both syntheses and the
 * analysis as their tcgen05 GEMMs (operands split into BF16 terms, FP32 accumulation), the ring
 * product and K_l^T in FP32 (FNL_EUNSUPPORTED on the HEALPix grid and on batch clones). */
fnl_status fnl_generate_backward(const fnl_shells* sh, uint64_t seed, uint64_t realisation, double fnl,
                                 const double* noise, const double* gT, const double* gE,
                                 const double* aNLT, const double* aNLE, double* grad_noise,
                                 double* grad_fnl, void* stream);

/* fnl_generate with host outputs (host [nalm][2] each, any may be NULL): the same path on
 * `stream`.  A page-locked buffer (cudaHostAlloc, cudaHostRegister) is written by the path's
 * last kernel through its device mapping; any other buffer receives a device-to-host copy on
 * `stream` after the path.  The caller synchronises the stream before reading them. */
fnl_status fnl_generate_host(const fnl_shells* sh, uint64_t seed, uint64_t realisation, double fnl,
                             double* aT, double* aE, double* aNLT, double* aNLE, void* stream);

/* Step (i) alone: phiL (device [nalm][nr][2]) = K_l n for the noise of fnl_generate
 * (explicit `noise` or drawn from seed/realisation). */
fnl_status fnl_filter(const fnl_shells* sh, uint64_t seed, uint64_t realisation,
                      const double* noise, double* phiL, void* stream);

/* Step (ii) alone: maps (device [nr][ntheta][nphi]) of the nr real fields whose
 * coefficients are alm (device [nalm][nr][2]; imaginary part of m = 0 ignored). */
fnl_status fnl_synth(const fnl_shells* sh, const double* alm, double* maps, void* stream);

/* Step (iv) alone: alm (device [nalm][nr][2]) = Gauss-Legendre x DFT projection of maps
 * (device [nr][ntheta][nphi]) onto Y_lm, l <= lmax. */
fnl_status fnl_analyse(const fnl_shells* sh, const double* maps, double* alm, void* stream);

/* Steps (ii)-(iv): phiNL (device [nalm][nr][2]) = analysis(synthesis(phiL)^2 - mu). */
fnl_status fnl_square(const fnl_shells* sh, const double* phiL, double* phiNL, void* stream);

/* Step (v) alone (Eq. 5 and Eq. 3): from phiL and/or phiNL (device [nalm][nr][2], either
 * may be NULL and then counts as zero) form aT, aE, aLT, aLE, aNLT, aNLE (device
 * [nalm][2] each, any may be NULL) with f_NL = fnl. */
fnl_status fnl_accumulate(const fnl_shells* sh, const double* phiL, const double* phiNL,
                          double fnl, double* aT, double* aE, double* aLT, double* aLE,
                          double* aNLT, double* aNLE, void* stream);

/* ---- output maps: Stokes I, Q, U of one realisation (Sect. 4) ----------------------- */

/* Tables of the map synthesis: lambda_lm, W_lm and X_lm on the northern rings of the
 * object's grid, in the object's real type (FP64 for FNL_FP64, FP32 otherwise), computed
 * in FP64 on the device; W = (2lam + (-2)lam) / 2 and X = (2lam - (-2)lam) / 2, where
 * +-2Y_lm = +-2lam_lm(theta) e^{i m phi} are the spin-2 harmonics obtained from Y_lm with the
 * spin raising and lowering operators.  Allocates three tables of the size of the SIMT
 * Legendre table plus a [2 (lmax+1)][npairs][6] scratch (owned by the object, freed with
 * it), and synchronises the device.  Idempotent. */
fnl_status fnl_maps_prepare(fnl_shells* sh);

/* Stokes maps of one set of coefficients (needs fnl_maps_prepare; no allocation):
 *   I = sum_lm aT_lm Y_lm,   Q +- iU = sum_lm a_{+-2,lm} +-2Y_lm,   a_{+-2,lm} = -(aE_lm +- i aB_lm)
 * (the sign convention of HEALPix, whose I, Q, U maps the paper produces).
 *  aT, aE: device [nalm][2]; aB: device [nalm][2] or NULL (zero B modes, as the paper's
 *      maps have); the imaginary part of every m = 0 entry is ignored.
 *  maps: device [3][ntheta][nphi] double, (I, Q, U) on the object's ring grid.
 * One pass over the tables per call (one thread per ring pair and m, sums in the real type),
 * then one ring FFT per field.  FNL_EINVAL before fnl_maps_prepare or for a NULL aT, aE or
 * maps. */
fnl_status fnl_maps(const fnl_shells* sh, const double* aT, const double* aE, const double* aB, double* maps,
                    void* stream);

/* ---- the fast cubic f_NL estimator (Sect. 5) ------------------------------------------ */

typedef struct fnl_ksw fnl_ksw; /* opaque: weights, normalisation, a synthesis object of 2 nr fields */

/* Estimator for the configuration of `sh` (its l_max, ring grid, radial nodes r_i, weights
 * w_i, transfer kernels alpha^X_l and filters K_l; same precision form).  Sect. 5 defines
 *   A(r, n) = sum_{i,j in T,E} sum_lm (C^-1)^{ij}_l alpha^i_l(r) a^j_lm Y_lm(n),  B likewise with beta,
 *   S_prim  = int dr r^2 int d^2n A B^2,  and f_NL = S_prim / N with
 *   N = sum_{l1<=l2<=l3} (1/Delta) B^{ijk} (C^-1)^{io}_l1 (C^-1)^{jp}_l2 (C^-1)^{kq}_l3 B^{opq},
 *   B^{ijk} = 2 I_{l1l2l3} int dr r^2 [beta^i_l1 beta^j_l2 alpha^k_l3 + 2 more terms, alpha on each leg],
 *   I_{l1l2l3} = sqrt((2l1+1)(2l2+1)(2l3+1)/(4 pi)) (l1 l2 l3; 0 0 0),  Delta = 6, 2 or 1.
 * On the shells: int dr r^2 = sum_i w_i r_i^2; beta^X_l(r_i) = (K_l K_l^T q^X_l)_i with
 * q^X_l[i] = w_i r_i^2 alpha^X_l(r_i) (the covariance of Phi_L(r_i) and a^X_L, the discrete form of
 * the paper's beta); C^XY_l = (K_l^T q^X_l).(K_l^T q^Y_l), the covariance of a^T_L, a^E_L;
 * C^-1 the Moore-Penrose inverse (full inverse if the smaller eigenvalue exceeds 1e-10 of the
 * larger, else v v^T / lambda of the leading eigenpair); degrees l < 2 left out.
 * N is summed here in FP64 over all l1 <= l2 <= l3 (synchronous; a fraction of a second at
 * l_max 1024).  Needs 3 n_phi complex values of the object's real type in shared memory
 * (FNL_EINVAL above 227 KB).  Allocates device memory (a second set of synthesis scratch for
 * 2 nr fields); `sh` must outlive the estimator.  FNL_EUNSUPPORTED for a shell shard and, in the
 * tensor-core forms, for an odd shell count. */
fnl_status fnl_ksw_create(const fnl_shells* sh, fnl_ksw** out);
void fnl_ksw_destroy(fnl_ksw* k);

/* norm: N (host double, may be NULL); norm_seconds: device time of its sum (may be NULL);
 * rank: host [lmax+1] rank of C_l used, 0 for l < 2 (may be NULL). */
fnl_status fnl_ksw_info(const fnl_ksw* k, double* norm, double* norm_seconds, int* rank);

/* S_prim of one sky (no allocation, asynchronous on `stream`): aT, aE device [nalm][2]
 * (imaginary part of m = 0 ignored); S device double.  The sphere integral is the grid's
 * Gauss-Legendre x rectangle rule, exact for the cubic when ntheta >= (3 lmax + 2) / 2 and
 * nphi >= 3 lmax + 1.  The f_NL estimate is S / N. */
fnl_status fnl_ksw_statistic(const fnl_ksw* k, const double* aT, const double* aE, double* S, void* stream);

/* ---- optimal radial quadrature (Sect. 3) -------------------------------------------------- */

/* The design problem: degrees 0..lmax, a fine grid of ntot shells with nodes r and weights w
 * (the fine line-of-sight rule I = sum_k w_k r_k^2 alpha^X_l(r_k) Phi(r_k)), the transfer kernels
 * on it, and the covariance P_l of Phi on the fine nodes: given (host [lmax+1][ntot][ntot]), or
 * NULL and then built on the device as Eq. 7, C_l(r_i, r_j) = (2/pi) sum_k wk k^2 A k^(ns-4)
 * j_l(k r_i) j_l(k r_j) on the nk-point trapezoid rule over [kmin, kmax].  In both cases
 * eps_l = jitter_rel * mean(diag) is added to the diagonal (the covariance the filters realise). */
typedef struct {
  int lmax;                       /* 0 <= lmax <= 4096 */
  int ntot;                       /* fine shells, 1 <= ntot <= 4096 */
  const double* r;                /* host [ntot] fine nodes */
  const double* w;                /* host [ntot] fine weights */
  const double* alphaT;           /* host [lmax+1][ntot] */
  const double* alphaE;           /* host [lmax+1][ntot] */
  const double* P;                /* host [lmax+1][ntot][ntot] covariance, or NULL (Eq. 7 below) */
  double A, ns, kmin, kmax;       /* P(k) = A k^(ns - 4) and the k range */
  int nk;                         /* k points (>= 2) */
  double jitter_rel;              /* >= 0 */
} fnl_quad_desc;

typedef struct fnl_quad fnl_quad; /* opaque: the fine covariance, c = P q and <I^2> on the device */

/* Builds P_l (FP64, on the device when desc->P is NULL), c^X_l = P_l q^X_l and <I^2>^X_l = q.c,
 * q^X_l[k] = w_k r_k^2 alpha^X_l(r_k).  Synchronous; allocates (lmax+1) ntot^2 doubles. */
fnl_status fnl_quad_create(const fnl_quad_desc* desc, int device, fnl_quad** out);
void fnl_quad_destroy(fnl_quad* q);

/* I2: host [2][lmax+1] <I^2> of T and E (may be NULL); seconds: wall time of fnl_quad_create. */
fnl_status fnl_quad_moments(const fnl_quad* q, double* I2, double* seconds);

/* The paper's greedy: nsel fine nodes, each step adding the node that lowers the summed relative
 * error sum_{l, X: <I^2> > 0} <(I^ - I)^2> / <I^2> most (ties: smallest index), with the optimal
 * weights P_SS w = c_S.  Outputs (host): nodes [nsel] in selection order; weights [2][lmax+1][nsel]
 * (w^X_l on those nodes, to multiply Phi(r_i) directly) or NULL; objective [nsel] after each step
 * or NULL; rel_err [2][lmax+1] at the end or NULL; seconds: wall time, or NULL.
 * Expected error: <I^2> - c_S^T P_SS^-1 c_S, by the pivoted Cholesky factor of P_l. */
fnl_status fnl_quad_greedy(const fnl_quad* q, int nsel, int* nodes, double* weights, double* objective,
                           double* rel_err, double* seconds);

/* Optimal weights on given distinct fine nodes (host [n]): P_SS w = c_S by the same pivoted
 * Cholesky steps; weights host [2][lmax+1][n] (node order as given) or NULL; rel_err host
 * [2][lmax+1] or NULL. */
fnl_status fnl_quad_fit(const fnl_quad* q, int n, const int* nodes, double* weights, double* rel_err);

/* Relative expected error (<I^2> - 2 w.c_S + w^T P_SS w) / <I^2> of any rule: n fine nodes
 * (host [n]) with weights (host [2][lmax+1][n]); rel_err host [2][lmax+1] (0 where <I^2> = 0). */
fnl_status fnl_quad_error(const fnl_quad* q, int n, const int* nodes, const double* weights, double* rel_err);

/* Cap the SMs that the object's persistent kernels occupy: the tensor-core Legendre GEMMs
 * (gemm_sms) and the specialised ring kernel (ring_sms); 0 = all SMs (the default).  For
 * running the DRAM-bound GEMMs of one realisation beside the compute-bound stages of another
 * on disjoint SMs.  FNL_EINVAL outside [0, SM count]. */
fnl_status fnl_shells_set_sm_limits(fnl_shells* sh, int gemm_sms, int ring_sms);

/* Wait for all work on the object's device, then report FNL_ETIMEOUT if a bounded wait
 * inside a tensor-core kernel expired since the last call (the kernels record it in a
 * device word instead of hanging), else FNL_OK.  Clears the word. */
fnl_status fnl_device_status(const fnl_shells* sh);

/* ---- test hooks (no counterpart in the paper) ----------------------------------------- */

/* Make the device allocation after the next n ones fail with FNL_ENOMEM, as if cudaMalloc had
 * failed (once; the hook then turns itself off), so that a test can check that every set-up
 * call unwinds and frees what it had allocated; n = -1 turns the hook off.  Process-wide. */
fnl_status fnl_test_fail_alloc(long n);

/* Launch one bounded mbarrier wait of the tensor-core kernels (the same wait routine) on a
 * barrier that nothing completes, with `limit` tries (1 .. 2^20): the wait runs out, records
 * its code in the object's error word and returns, so fnl_device_status then reports
 * FNL_ETIMEOUT.  Tensor-core objects only (FNL_EINVAL otherwise).  Asynchronous on `stream`. */
fnl_status fnl_test_wait_expiry(const fnl_shells* sh, unsigned limit, void* stream);

/* ---- batching form: many realisations of uneven l_max and N_r in one graph --------- */

typedef struct fnl_batch fnl_batch; /* opaque: streams, events and the captured graph */

/* A batch of n instances; instance i runs the path of shells[i] (objects of any l_max, N_r,
 * grid and precision, all on one device; one object may appear several times).  Every
 * instance gets scratch of its own: a repeated object of the tensor-core forms is given
 * scratch clones that share its tables (device memory the batch allocates and frees).
 *  - Multi-instance mode, when every instance is a whole configuration (no shell shard) in
 *    one tensor-core form, has a ring length with a specialised ring kernel (800, 1600, 3125,
 *    3200; N_r a multiple of its shell group) and n <= 64: each stage of the path is one launch over all instances (the ring
 *    stage one per ring length present).  The tile shape, common to all instances, is picked
 *    here by timing whole batches, and set on the shells objects (synchronous).
 *  - Stream mode otherwise: instances are dealt, largest first (work ~ (l_max + 1)^3 N_r), to
 *    up to `nstreams` streams (0: 4); repeated objects of the FP64/FP32 forms share their
 *    scratch and stay on one stream.
 * The batch keeps the pointers: the objects must outlive it.  Allocates host memory, CUDA
 * streams and events, and device memory for clones and the multi-instance arguments. */
fnl_status fnl_batch_create(fnl_shells* const* shells, int n, int nstreams, fnl_batch** out);

/* Tile widths of the multi-instance launches (synthesis ring pairs, analysis degrees), or 0
 * for a batch in stream mode. */
fnl_status fnl_batch_tiles(const fnl_batch* b, int* nsyn, int* nana);

/* Synchronise the batch's streams and free it (NULL is ignored). */
void fnl_batch_destroy(fnl_batch* b);

/* Number of instances, of streams (0 in multi-instance mode), and (lanes: host [n] or NULL)
 * the stream of each instance. */
fnl_status fnl_batch_info(const fnl_batch* b, int* n, int* nstreams, int* lanes);

/* Steps (i)-(v) of every instance: instance i draws its Philox noise from (seeds[i],
 * realisations[i]) as fnl_generate does, uses f_NL = fnl[i] and writes a^T, a^E (Eq. 3) to
 * aT[i], aE[i] (device [nalm_i][2]).  seeds, realisations, fnl, aT, aE: host arrays of n.
 * The launches of all instances are captured into one CUDA graph (the first call
 * instantiates it, later calls update it in place) and the graph is launched on `stream`:
 * asynchronous, one graph launch per call.  Each instance's result equals that of
 * fnl_generate with the same arguments on its shells object (bit for bit).  The call itself begins a stream capture, so it
 * cannot be made while `stream`'s thread is capturing.  Calls on one batch, and calls on
 * its shells objects, must not overlap on the GPU. */
fnl_status fnl_generate_batch(fnl_batch* b, const uint64_t* seeds, const uint64_t* realisations,
                              const double* fnl, double* const* aT, double* const* aE, void* stream);

/* Autotuner of the tensor-core forms: times whole realisations (one warm-up and two timed,
 * CUDA events on `stream`) for each candidate tile shape of the two Legendre GEMMs --
 * synthesis tiles of up to 256 or 128 ring pairs, analysis tiles of up to 256, 128 or 96
 * degrees -- and keeps the fastest.  The shape changes no result (every output sums its
 * k blocks in the same order).  *nsyn, *nana (nullable) receive the chosen widths (64 for
 * the SIMT forms, whose tiles are fixed and which this call leaves alone).  Synchronous. */
fnl_status fnl_shells_autotune(fnl_shells* sh, void* stream, int* nsyn, int* nana);

/* Set the tile shape of the tensor-core GEMMs by hand: synthesis tiles of at most syn_cap
 * ring pairs, analysis tiles of at most ana_cap degrees, multiples of 16 in [64, 256].
 * Synchronises the device.  FNL_EINVAL for the SIMT forms. */
fnl_status fnl_shells_set_tiles(fnl_shells* sh, int syn_cap, int ana_cap);

/* Share of the dense Legendre work (sum over the problems (m, parity) of K_mp x npairs
 * multiply-adds per column) that the tensor-core GEMMs execute with the current tiles: the
 * GEMMs leave out, per order m, the polar ring pairs where every |lambda_lm| < 2^-30 (whole
 * synthesis tiles, and the analysis's 64-ring-pair k stages below the first live ring pair), a
 * standard SHT economy whose dropped terms stay below 1e-7 of the results.  *syn, *ana
 * (nullable) receive the two shares in (0, 1].  FNL_EINVAL for the SIMT forms (they compute
 * everything). */
fnl_status fnl_shells_gemm_work(const fnl_shells* sh, double* syn, double* ana);

/* ---- step (v) without any allocation ---------------------------------------------- */

/* Largest (lmax + 1) * nr that fnl_accumulate_noalloc accepts. */
#define FNL_NOALLOC_MAX_LNR 524288

/* fnl_accumulate without a shells object and without allocating device memory, for
 * callers that may not allocate: programs whose device memory belongs to another
 * allocator (a cudaMalloc outside it fails or fragments its pool), latency-bound loops
 * (cudaMalloc and cudaFree can synchronise the device), plug-ins held to a fixed memory
 * budget.  The paper has no counterpart to this call.  It computes what fnl_accumulate
 * computes, with the weights q^X_l[i] = w_i r_i^2 alpha^X_l(r_i) formed on each call into a
 * fixed array inside the library instead of a table made by fnl_make_shells.
 *  r, w:            device [nr] radial nodes and weights (8-byte aligned).
 *  alphaT, alphaE:  device [lmax+1][nr] alpha^X_l(r_i) (8-byte aligned).
 *  phiL, phiNL:     device [nalm][nr][2], either may be NULL and then counts as zero.
 *  aT ... aNLE:     device [nalm][2] as in fnl_accumulate, any may be NULL.
 * Every device pointer must belong to the current device; the call runs on `stream`.
 * Sizes: 0 <= lmax <= 4096, 1 <= nr <= 128 and (lmax + 1) * nr <= FNL_NOALLOC_MAX_LNR,
 * else FNL_EINVAL before anything runs.  The array holds 2 * FNL_NOALLOC_MAX_LNR doubles
 * (8 MiB) on every GPU that loads the library, until the process exits.
 * Set-up: the first call in a CUDA context (per device; again after cudaDeviceReset), with
 * that device current, looks up the array's device address (cudaGetSymbolAddress, which may
 * load the library's device code).  Make that first call before any stream capture begins:
 * a first call on a capturing stream returns FNL_EUNSUPPORTED.
 * Every call uses the same array, and keeps in it the weights of the last call: each call
 * rewrites every weight it reads before reading it, so nothing there has to start at zero,
 * but calls that overlap on the GPU (concurrent streams, or threads sharing a device) race
 * on it: a call holds the array from its first kernel (the weights) until its second (the
 * sums) ends on its stream.  Order such calls. */
fnl_status fnl_accumulate_noalloc(int lmax, int nr, const double* r, const double* w,
                                  const double* alphaT, const double* alphaE, const double* phiL,
                                  const double* phiNL, double fnl, double* aT, double* aE,
                                  double* aLT, double* aLE, double* aNLT, double* aNLE, void* stream);

/* ---- per-stage timing -------------------------------------------------------------- */

/* Stages of fnl_generate timed when profiling is on (CUDA events recorded on the
 * caller's stream between the kernels): 0 noise + filter (step (i)), 1 synthesis
 * Legendre GEMM (step (ii)), 2 ring DFTs + square (steps (ii)-(iv)), 3 analysis
 * Legendre GEMM (step (iv)), 4 radial quadrature (step (v)). */
#define FNL_NSTAGES 5

/* Turn event timing of fnl_generate on with a ring of `slots` calls (1..4096), or off
 * (slots = 0).  Each profiled call records FNL_NSTAGES + 1 events on its stream; no call
 * synchronises.  Not thread-safe with a concurrent fnl_generate on the same object. */
fnl_status fnl_profile_enable(fnl_shells* sh, int slots);

/* ms[0..n-1] (host, n <= FNL_NSTAGES) = stage durations summed over the profiled calls
 * since the last read (at most `slots` of them, the most recent); *calls (nullable)
 * receives their number.  Waits for those calls to finish and restarts the count. */
fnl_status fnl_profile_read(fnl_shells* sh, double* ms, int n, int* calls);

/* ---- measured arithmetic peaks (for the rooflines; no counterpart in the paper) ------- */

/* FP64 and FP32 fused multiply-add rates of device `device` in TFLOP/s (2 flops per FMA), each
 * measured with a kernel of independent FMA chains filling every SM (median of five timed
 * launches of ~10 ms, CUDA events).  Either output may be NULL.  Synchronous; allocates a small
 * temporary buffer. */
fnl_status fnl_measure_fma_peaks(int device, double* fp64_tflops, double* fp32_tflops);

/* ---- host-side set-up helpers (no GPU needed) -------------------------------------- */

/* n-point Gauss-Legendre rule: x (host [n], north to south, x_j = cos theta_j), w (host [n]). */
fnl_status fnl_gauss_legendre(int n, double* x, double* w);

/* Radial covariance of Eq. 7 on a uniform trapezoid k rule:
 * C (host [lmax+1][nr][nr]) = (2/pi) sum_k wk k^2 A k^(ns-4) j_l(k r_i) j_l(k r_j). */
fnl_status fnl_covariance(int lmax, int nr, const double* r, double A, double ns, double kmin,
                          double kmax, int nk, double* C);

/* K (host [lmax+1][nr][nr], lower triangular) = chol(C_l + jitter_rel mean(diag C_l) I). */
fnl_status fnl_cholesky_filters(int lmax, int nr, const double* C, double jitter_rel, double* K);

#ifdef __cplusplus
}
#endif

#endif /* FNL_H */
