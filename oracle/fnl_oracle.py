"""Plain FP64 CPU oracle of the local-f_NL a_lm generator (Elsner & Wandelt).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU legs of ``bench.py`` may import this module.  It shares no code, header,
table or helper with the CUDA library and never imports it; the only module
both sides use is ``workloads`` (seeded inputs, no method arithmetic).

What it computes, in the paper's order (Sect. 2, recipe steps (i)-(v)):

  (i)   Phi_L,lm(r_i) = sum_j K_l[i, j] n_lm(r_j)            Eq. 9, K_l = chol(P_Phi,l)
  (ii)  f(theta, phi) = sum_lm Phi_L,lm Y_lm(theta, phi)       per shell, GL ring grid
  (iii) g = f^2 - <Phi_L^2>                                    Eq. 2
  (iv)  Phi_NL,lm = int g Y*_lm dOmega                         GL quadrature x DFT
  (v)   a^X_lm = sum_i w_i r_i^2 alpha^X_l(r_i) Phi_lm(r_i)    Eq. 5, X in {T, E}
        a^X = a^X_L + f_NL a^X_NL                               Eq. 3

with the covariance of Eq. 7 written as C_l(r_i, r_j) = (2/pi) int dk k^2 P(k)
j_l(k r_i) j_l(k r_j) (Eq. 7 with Eq. 8 substituted).

Every function works in float64/complex128.  Library primitives used as steps:
numpy matmul, numpy.fft.rfft/irfft (a DFT of a Hermitian-symmetric spectrum),
numpy.linalg.cholesky.  Nothing is blocked, fused or reordered beyond the
definitions written in each docstring.

The output maps (``maps_iqu``: Stokes I, Q, U from a^T, a^E, a^B) use spin-2 functions
written from the spin raising and lowering operators (``spin2_functions``); their pins are the
operators evaluated by finite differences of scipy's Y_lm, the closed form of 2Y_20,
orthonormality on the grid, the spin-2 analysis round trip, Parseval and the E/B rotation.

A shell shard (``generate_shard``: the recipe's per-shell terms for shells j0 .. j1 - 1) is
pinned by the sum over a partition of the shells equalling ``generate``, and by its a^X_L
against the whole configuration's v^X . n restricted to the shard's rows, written out.

The adjoint (``generate_backward`` and the transposes it chains) is the chain rule
through these steps; its pins are the dot-product test of every transpose against its
pinned forward map and central finite differences of a loss through ``generate``.

Pins (tests/test_oracle_pins.py, CPU): Gauss-Legendre rule vs numpy's leggauss;
lambda_lm vs scipy's spherical harmonics and orthonormality; j_l vs scipy;
Philox vs numpy.random.Philox; Gaunt brute force (Racah 3j) for Phi_L^2 at
l_max <= 8; analysis(synthesis(a)) = a; Parseval monopole; z-rotation and
parity equivariance; linearity in f_NL; f_NL = 0 closed-form covariance.
Every function here is pinned by at least one of them; none is "parity unpinned".
"""
from __future__ import annotations

import math

import numpy as np

from workloads import alm_index, n_alm

FOUR_PI = 4.0 * math.pi
FLUSH = 1e-290  # |lambda_lm| below this is stored as an exact zero


# ---------------------------------------------------------------------------
# Grid: Gauss-Legendre rings (the grid that stands in for HEALPix, Sect. 3)
# ---------------------------------------------------------------------------

def gauss_legendre(n: int) -> tuple[np.ndarray, np.ndarray]:
    """Nodes x_j = cos(theta_j) and weights of the n-point Gauss-Legendre rule.

    Nodes are ordered north to south (x descending).  Roots of P_n found by Newton
    iteration, P_n from the Bonnet recurrence, w_j = 2 / ((1 - x_j^2) P_n'(x_j)^2).
    The rule is made exactly antisymmetric (x_{n-1-j} = -x_j, the middle node of an
    odd rule is 0), as the roots of P_n are.
    """
    i = np.arange(n, dtype=np.float64)
    x = np.cos(math.pi * (i + 0.75) / (n + 0.5))

    def p_and_dp(x):
        p0 = np.ones_like(x)
        p1 = x.copy()
        for k in range(2, n + 1):
            p0, p1 = p1, ((2 * k - 1) * x * p1 - (k - 1) * p0) / k
        if n == 1:
            p0, p1 = np.ones_like(x), x.copy()
        dp = n * (x * p1 - p0) / (x * x - 1.0)
        return p1, dp

    for _ in range(100):
        p, dp = p_and_dp(x)
        dx = p / dp
        x = x - dx
        if np.max(np.abs(dx)) < 1e-15:
            break
    p, dp = p_and_dp(x)
    x = x - p / dp
    x = 0.5 * (x - x[::-1])
    if n % 2 == 1:
        x[n // 2] = 0.0
    _, dp = p_and_dp(x)
    w = 2.0 / ((1.0 - x * x) * dp * dp)
    w = 0.5 * (w + w[::-1])
    return x, w


# ---------------------------------------------------------------------------
# Normalised associated Legendre functions lambda_lm(x)
# Y_lm(theta, phi) = lambda_lm(cos theta) e^{i m phi}, orthonormal, with the
# Condon-Shortley phase (the convention of the HEALPix package the paper used).
# ---------------------------------------------------------------------------

def lambda_mm(lmax: int, x: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """lambda_mm(x) for m = 0..lmax as (mantissa, exponent): lambda_mm = mant * 2**exp.

    lambda_00 = 1/sqrt(4 pi); lambda_mm = -sqrt((2m+1)/(2m)) sin(theta) lambda_{m-1,m-1}.
    The product is renormalised to a mantissa in [0.5, 1) after every factor so that
    no value underflows however small sin(theta)^m becomes.
    """
    x = np.asarray(x, dtype=np.float64)
    s = np.sqrt((1.0 - x) * (1.0 + x))
    mant = np.empty((lmax + 1, x.size))
    expo = np.empty((lmax + 1, x.size), dtype=np.int64)
    v, e = np.frexp(np.full(x.size, 1.0 / math.sqrt(FOUR_PI)))
    e = e.astype(np.int64)
    mant[0], expo[0] = v, e
    for m in range(1, lmax + 1):
        v = v * (-math.sqrt((2.0 * m + 1.0) / (2.0 * m)) * s)
        v, de = np.frexp(v)
        e = e + de
        mant[m], expo[m] = v, e
    return mant, expo


def lambda_column(m: int, lmax: int, x: np.ndarray, mm=None) -> np.ndarray:
    """lambda_lm(x) for l = m..lmax, shape [lmax - m + 1, len(x)].

    Three-term recurrence in l:
      lambda_{m+1,m} = sqrt(2m+3) x lambda_mm,
      lambda_lm = a_lm (x lambda_{l-1,m} - b_lm lambda_{l-2,m}),
      a_lm = sqrt((4l^2 - 1) / (l^2 - m^2)),  b_lm = sqrt(((l-1)^2 - m^2) / (4(l-1)^2 - 1)),
    run on mantissas with a shared binary exponent that is moved by 2^500 whenever
    the mantissa grows past 2^500.  Entries with |lambda| < 1e-290 are set to 0.
    """
    x = np.asarray(x, dtype=np.float64)
    if mm is None:
        mm = lambda_mm(m, x)
    mant, expo = mm
    y1 = mant[m].copy()  # lambda_{l-1,m} mantissa
    y2 = np.zeros_like(y1)  # lambda_{l-2,m} mantissa
    e = expo[m].copy()
    out = np.empty((lmax - m + 1, x.size))
    out[0] = np.ldexp(y1, e)
    big = 2.0 ** 500
    for l in range(m + 1, lmax + 1):
        a = math.sqrt((4.0 * l * l - 1.0) / (l * l - m * m))
        b = math.sqrt(((l - 1.0) ** 2 - m * m) / (4.0 * (l - 1.0) ** 2 - 1.0))
        y = a * (x * y1 - b * y2)
        y2, y1 = y1, y
        hit = np.abs(y1) > big
        if hit.any():
            y1 = np.where(hit, y1 * 2.0 ** -500, y1)
            y2 = np.where(hit, y2 * 2.0 ** -500, y2)
            e = np.where(hit, e + 500, e)
        out[l - m] = np.ldexp(y1, e)
    out[np.abs(out) < FLUSH] = 0.0
    return out


def lambda_table(lmax: int, x: np.ndarray) -> list:
    """All columns: list over m of lambda_column(m, lmax, x)."""
    mm = lambda_mm(lmax, x)
    return [lambda_column(m, lmax, x, mm) for m in range(lmax + 1)]


# ---------------------------------------------------------------------------
# Spherical harmonic transforms of real fields on the GL ring grid
# ---------------------------------------------------------------------------

class Grid:
    """Gauss-Legendre ring grid: n_theta rings at x_j = cos(theta_j) (north to
    south) with weights w_j, n_phi equidistant points phi_k = 2 pi k / n_phi per
    ring (no ring offset).

    ``store=True`` keeps every lambda column (fine up to l_max ~ 512); with
    ``store=False`` columns are recomputed on demand, bounding memory at l_max = 1024."""

    def __init__(self, lmax: int, ntheta: int, nphi: int, store: bool = True):
        self.lmax, self.ntheta, self.nphi = lmax, ntheta, nphi
        self.x, self.w = gauss_legendre(ntheta)
        self._mm = lambda_mm(lmax, self.x)
        self._cols = [lambda_column(m, lmax, self.x, self._mm) for m in range(lmax + 1)] if store else None

    def lam(self, m: int) -> np.ndarray:
        """lambda_lm(x_j) for l = m..lmax, shape [lmax - m + 1, n_theta]."""
        if self._cols is not None:
            return self._cols[m]
        return lambda_column(m, self.lmax, self.x, self._mm)


def synthesis(alm: np.ndarray, grid: Grid) -> np.ndarray:
    """Real fields f(theta_j, phi_k) = sum_{l, |m| <= l} a_lm Y_lm, a_{l,-m} = (-1)^m conj(a_lm).

    alm: [nalm, nsh] complex (m-major triangle).  Returns [nsh, n_theta, n_phi].
    Step 1: F_m(theta_j) = sum_l lambda_lm(x_j) a_lm            (matmul per m)
    Step 2: f_jk = F_0 + 2 Re sum_{m>=1} F_m e^{i m phi_k}        (inverse real DFT)
    """
    L = grid.lmax
    alm = np.asarray(alm, dtype=np.complex128)
    if alm.ndim == 1:
        alm = alm[:, None]
    nsh = alm.shape[1]
    F = np.zeros((nsh, grid.ntheta, grid.nphi // 2 + 1), dtype=np.complex128)
    for m in range(L + 1):
        rows = alm_index(np.arange(m, L + 1), m, L)
        F[:, :, m] = (grid.lam(m).T @ alm[rows, :]).T
    # irfft(F) * n = F_0 + 2 Re sum_{m=1}^{n/2-1} F_m e^{2 pi i m k / n} (+ Nyquist, zero here
    # because l_max < n_phi / 2); the imaginary part of F_0 is dropped, as for a real field.
    return np.fft.irfft(F, n=grid.nphi, axis=-1) * grid.nphi


def analysis(maps: np.ndarray, grid: Grid) -> np.ndarray:
    """a_lm = int f Y*_lm dOmega by GL quadrature in theta and the rectangle rule in phi.

    maps: [nsh, n_theta, n_phi] real.  Returns [nalm, nsh] complex.
    Step 1: G_m(theta_j) = (2 pi / n_phi) sum_k f_jk e^{-i m phi_k}   (forward real DFT)
    Step 2: a_lm = sum_j w_j lambda_lm(x_j) G_m(theta_j)             (matmul per m)
    """
    L = grid.lmax
    maps = np.asarray(maps, dtype=np.float64)
    if maps.ndim == 2:
        maps = maps[None]
    nsh = maps.shape[0]
    G = np.fft.rfft(maps, axis=-1) * (2.0 * math.pi / grid.nphi)  # [nsh, ntheta, nphi/2+1]
    out = np.zeros((n_alm(L), nsh), dtype=np.complex128)
    for m in range(L + 1):
        rows = alm_index(np.arange(m, L + 1), m, L)
        out[rows, :] = grid.lam(m) @ (grid.w[:, None] * G[:, :, m].T)
    return out


# ---------------------------------------------------------------------------
# Radial statistics: covariance (Eq. 7), filter (Eq. 9), <Phi_L^2> (Eq. 2)
# ---------------------------------------------------------------------------

def spherical_jn_table(lmax: int, x: np.ndarray) -> np.ndarray:
    """Spherical Bessel j_l(x) for l = 0..lmax, shape [lmax+1, len(x)], x > 0.

    For x > lmax + 60 the upward recurrence j_{l+1} = (2l+1)/x j_l - j_{l-1} from
    j_0 = sin x / x, j_1 = sin x / x^2 - cos x / x is stable (l < x throughout).
    Otherwise Miller's downward recurrence from l = lmax + 200 + x (j_{N+1} = 0,
    j_N = 1), renormalised by powers of two to avoid overflow and scaled so
    that sum_l (2l+1) j_l^2 = 1, with the sign of j_0 (or of j_1 where j_0 is
    small).
    """
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros((lmax + 1, x.size))
    up = x > lmax + 60.0
    if up.any():
        xu = x[up]
        j0 = np.sin(xu) / xu
        out[0, up] = j0
        if lmax >= 1:
            j1 = np.sin(xu) / (xu * xu) - np.cos(xu) / xu
            out[1, up] = j1
            a, b = j0, j1
            for l in range(1, lmax):
                a, b = b, (2.0 * l + 1.0) / xu * b - a
                out[l + 1, up] = b
    dn = ~up
    if dn.any():
        xd = x[dn]
        nstart = int(lmax + 200 + np.max(xd))
        ynext = np.zeros_like(xd)
        y = np.ones_like(xd)
        e = np.zeros(xd.size, dtype=np.int64)  # exponent carried by y at the current l
        mant = np.zeros((lmax + 1, xd.size))
        expo = np.zeros((lmax + 1, xd.size), dtype=np.int64)
        # sum rule accumulated relative to the running exponent
        ssum = np.zeros_like(xd)
        for l in range(nstart, 0, -1):
            if l <= lmax:
                mant[l], expo[l] = y, e
            ssum = ssum + (2.0 * l + 1.0) * y * y
            yprev = (2.0 * l + 1.0) / xd * y - ynext
            ynext, y = y, yprev
            hit = np.abs(y) > 2.0 ** 400
            if hit.any():
                s = 2.0 ** -400
                y = np.where(hit, y * s, y)
                ynext = np.where(hit, ynext * s, ynext)
                ssum = np.where(hit, ssum * s * s, ssum)
                e = np.where(hit, e + 400, e)
        mant[0], expo[0] = y, e
        ssum = ssum + y * y
        # true value j_l = c * mant_l * 2^(expo_l - e0), c = 1/sqrt(ssum) up to sign
        norm = 1.0 / np.sqrt(ssum)
        j0_true = np.sin(xd) / xd
        j1_true = np.sin(xd) / (xd * xd) - np.cos(xd) / xd
        use_j0 = np.abs(j0_true) > 0.1 * np.abs(j1_true)
        ref_true = np.where(use_j0, j0_true, j1_true)
        ref_num = np.where(use_j0, mant[0] * norm,
                           np.ldexp(mant[1], expo[1] - e) * norm if lmax >= 1 else mant[0] * norm)
        sign = np.sign(ref_true) * np.sign(ref_num)
        sign[sign == 0] = 1.0
        for l in range(lmax + 1):
            out[l, dn] = sign * np.ldexp(mant[l] * norm, expo[l] - e)
    out[np.abs(out) < FLUSH] = 0.0
    return out


def k_rule(kmin: float, kmax: float, nk: int) -> tuple[np.ndarray, np.ndarray]:
    """Uniform trapezoid rule on [kmin, kmax] with nk points (end points included)."""
    k = np.linspace(kmin, kmax, nk)
    h = (kmax - kmin) / (nk - 1)
    wk = np.full(nk, h)
    wk[0] = wk[-1] = 0.5 * h
    return k, wk


def covariance(lmax: int, r: np.ndarray, A: float, ns: float, kmin: float, kmax: float,
               nk: int, chunk: int = 128) -> np.ndarray:
    """C_l(r_i, r_j) = (2/pi) sum_k wk k^2 A k^(ns-4) j_l(k r_i) j_l(k r_j), shape [lmax+1, nr, nr].

    Eq. 7 with Delta^2_R(k) = k^3 P(k) / (2 pi^2) (Eq. 8) and P(k) = A k^(ns-4):
    4 pi Delta^2_R(k) / k = (2/pi) k^2 P(k).
    """
    r = np.asarray(r, dtype=np.float64)
    nr = r.size
    k, wk = k_rule(kmin, kmax, nk)
    pk = (2.0 / math.pi) * wk * k * k * A * k ** (ns - 4.0)
    C = np.zeros((lmax + 1, nr, nr))
    for s in range(0, nk, chunk):
        ks, ps = k[s:s + chunk], pk[s:s + chunk]
        xs = (ks[:, None] * r[None, :]).ravel()
        J = spherical_jn_table(lmax, xs).reshape(lmax + 1, ks.size, nr)
        C += np.einsum("lki,k,lkj->lij", J, ps, J, optimize=True)
    return C


def filters(C: np.ndarray, jitter_rel: float) -> np.ndarray:
    """K_l = cholesky(C_l + eps_l I), eps_l = jitter_rel * mean(diag C_l); lower triangular."""
    L1, nr, _ = C.shape
    K = np.empty_like(C)
    eye = np.eye(nr)
    for l in range(L1):
        eps = jitter_rel * np.mean(np.diag(C[l]))
        K[l] = np.linalg.cholesky(C[l] + eps * eye)
    return K


def mu_ensemble(K: np.ndarray) -> np.ndarray:
    """<Phi_L^2(r_i)> over the ensemble for a field band-limited at l_max:
    mu_i = sum_l (2l+1)/(4 pi) (K_l K_l^T)[i, i]  (addition theorem)."""
    L1 = K.shape[0]
    l = np.arange(L1, dtype=np.float64)
    diag = np.einsum("lij,lij->li", K, K)
    return ((2.0 * l + 1.0)[:, None] / FOUR_PI * diag).sum(axis=0)


# ---------------------------------------------------------------------------
# Noise: Philox4x64-10 counter-based generator (Salmon et al., SC'11) + Box-Muller
# ---------------------------------------------------------------------------

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
_M32 = np.uint64(0xFFFFFFFF)
PHILOX_M0 = np.uint64(0xD2E7470EE14C6C93)
PHILOX_M1 = np.uint64(0xCA5A826395121157)
PHILOX_W0 = np.uint64(0x9E3779B97F4A7C15)
PHILOX_W1 = np.uint64(0xBB67AE8584CAA73B)


def _mulhilo64(a, b):
    """(high, low) 64-bit halves of the 128-bit product a * b (uint64 arrays)."""
    a = np.asarray(a, dtype=np.uint64)
    b = np.asarray(b, dtype=np.uint64)
    s32 = np.uint64(32)
    lo = a * b
    al, ah = a & _M32, a >> s32
    bl, bh = b & _M32, b >> s32
    t = al * bl
    c1 = ah * bl + (t >> s32)
    c2 = al * bh + (c1 & _M32)
    hi = ah * bh + (c1 >> s32) + (c2 >> s32)
    return hi, lo


def philox4x64(c0, c1, c2, c3, k0, k1, rounds: int = 10):
    """Philox4x64-R block function: 4 counter words and 2 key words (uint64) to 4
    output words.  Each round: (h0, l0) = M0 * c0, (h1, l1) = M1 * c2, new
    counter (h1 ^ c1 ^ k0, l1, h0 ^ c3 ^ k1, l0); the key is bumped by the Weyl
    constants (W0, W1) between rounds."""
    with np.errstate(over="ignore"):
        c = [np.asarray(v, dtype=np.uint64) for v in (c0, c1, c2, c3)]
        k0 = np.asarray(k0, dtype=np.uint64)
        k1 = np.asarray(k1, dtype=np.uint64)
        for r in range(rounds):
            if r:
                k0 = k0 + PHILOX_W0
                k1 = k1 + PHILOX_W1
            h0, l0 = _mulhilo64(PHILOX_M0, c[0])
            h1, l1 = _mulhilo64(PHILOX_M1, c[2])
            c = [h1 ^ c[1] ^ k0, l1, h0 ^ c[3] ^ k1, l0]
    return c


def philox_noise(lmax: int, nr: int, seed: int, realisation: int) -> np.ndarray:
    """White noise n_lm(r_j) drawn from (seed, realisation), shape [nr, nalm] complex.

    Counter (idx(l, m), j >> 2, realisation, 0), key (seed, 0).  Shell j uses output word
    w = w_{j mod 4}, split into two 32-bit halves:
      u1 = ((w >> 32) + 1) 2^-32 in (0, 1],  u2 = (w mod 2^32) 2^-32 in [0, 1),
      rho = sqrt(-2 ln u1), g1 = rho cos(2 pi u2), g2 = rho sin(2 pi u2)  (Box-Muller).
    n = (g1 + i g2) / sqrt(2) for m > 0 (unit complex variance); n = g1 for m = 0.
    """
    na = n_alm(lmax)
    idx = np.arange(na, dtype=np.uint64)
    out = np.empty((nr, na), dtype=np.complex128)
    s32 = np.uint64(32)
    low = np.uint64(0xFFFFFFFF)
    for jq in range((nr + 3) // 4):
        w = philox4x64(idx, np.uint64(jq), np.uint64(realisation), np.uint64(0),
                       np.uint64(seed), np.uint64(0))
        for q in range(4):
            j = 4 * jq + q
            if j >= nr:
                break
            u1 = ((w[q] >> s32) + np.uint64(1)).astype(np.float64) * 2.0 ** -32
            u2 = (w[q] & low).astype(np.float64) * 2.0 ** -32
            rho = np.sqrt(-2.0 * np.log(u1))
            g1 = rho * np.cos(2.0 * math.pi * u2)
            g2 = rho * np.sin(2.0 * math.pi * u2)
            n = (g1 + 1j * g2) / math.sqrt(2.0)
            n[: lmax + 1] = g1[: lmax + 1]
            out[j] = n
    return out


# ---------------------------------------------------------------------------
# The generator, Sect. 2 recipe steps (i)-(v)
# ---------------------------------------------------------------------------

def phi_linear(K: np.ndarray, noise: np.ndarray) -> np.ndarray:
    """Step (i), Eq. 9: Phi_L,lm(r_i) = sum_j K_l[i, j] n_lm(r_j).

    noise [nr, nalm] complex (the imaginary part of m = 0 entries is ignored);
    returns [nalm, nr] complex."""
    L = K.shape[0] - 1
    nt = np.array(np.asarray(noise, dtype=np.complex128).T)  # [nalm, nr]
    nt[: L + 1, :] = nt[: L + 1, :].real
    out = np.empty((nt.shape[0], K.shape[1]), dtype=np.complex128)
    for l in range(L + 1):
        rows = alm_index(l, np.arange(l + 1), L)  # (l, m) for m = 0..l
        out[rows, :] = nt[rows, :] @ K[l].T
    return out


def phi_nonlinear(phi_L: np.ndarray, mu: np.ndarray, grid: Grid) -> np.ndarray:
    """Steps (ii)-(iv), Eq. 2: Phi_NL,lm = analysis(synthesis(Phi_L)^2 - mu), per shell.

    phi_L [nalm, nsh], mu [nsh]; returns [nalm, nsh]."""
    f = synthesis(phi_L, grid)
    g = f * f - np.asarray(mu, dtype=np.float64)[:, None, None]
    return analysis(g, grid)


def quadrature_weights(r, w, alpha) -> np.ndarray:
    """q_l[i] = w_i r_i^2 alpha_l(r_i), the discretised line-of-sight integral of Eq. 5."""
    r = np.asarray(r, dtype=np.float64)
    return np.asarray(alpha, dtype=np.float64) * (np.asarray(w, dtype=np.float64) * r * r)[None, :]


def radial_quadrature(phi: np.ndarray, q: np.ndarray) -> np.ndarray:
    """Step (v), Eq. 5: a_lm = sum_i q_l[i] Phi_lm(r_i); phi [nalm, nr], q [lmax+1, nr]."""
    L = q.shape[0] - 1
    out = np.empty(phi.shape[0], dtype=np.complex128)
    for m in range(L + 1):
        ls = np.arange(m, L + 1)
        rows = alm_index(ls, m, L)
        out[rows] = np.einsum("ri,ri->r", phi[rows, :], q[ls, :])
    return out


def generate(K, noise, grid: Grid, r, w, alphaT, alphaE, fnl: float, mu=None, shells=None):
    """Full recipe for one realisation; returns a dict of complex [nalm] arrays
    aT, aE (Eq. 3), aLT, aLE, aNLT, aNLE (Eq. 5), and the intermediates phiL, phiNL.

    ``shells`` (optional index array) restricts steps (ii)-(iv) to a subset of
    shells; then aNL* are not formed (they need every shell) and phiNL holds only
    the subset's columns."""
    phiL = phi_linear(K, noise)
    if mu is None:
        mu = mu_ensemble(K)
    qT = quadrature_weights(r, w, alphaT)
    qE = quadrature_weights(r, w, alphaE)
    out = {"phiL": phiL, "aLT": radial_quadrature(phiL, qT), "aLE": radial_quadrature(phiL, qE)}
    if shells is not None:
        sel = np.asarray(shells)
        out["phiNL"] = phi_nonlinear(phiL[:, sel], np.asarray(mu)[sel], grid)
        return out
    phiNL = phi_nonlinear(phiL, mu, grid)
    out["phiNL"] = phiNL
    out["aNLT"] = radial_quadrature(phiNL, qT)
    out["aNLE"] = radial_quadrature(phiNL, qE)
    out["aT"] = out["aLT"] + fnl * out["aNLT"]
    out["aE"] = out["aLE"] + fnl * out["aNLE"]
    return out


def generate_shard(K, noise, grid: Grid, r, w, alphaT, alphaE, fnl: float, j0: int, j1: int, mu=None):
    """Shells j0 .. j1 - 1 of the recipe: their Phi_L (rows j0 .. j1 - 1 of Eq. 9, which read
    the noise of shells 0 .. j1 - 1 only), their Phi_NL (steps (ii)-(iv), shell by shell) and
    their terms of the radial quadrature (Eq. 5) and of Eq. 3.  noise [nr, nalm] holds every
    shell of the configuration; mu (default: ``mu_ensemble(K)``) is the configuration's.

    Eq. 5 and Eq. 3 are sums over shells of per-shell terms, so the outputs of shards that
    partition 0 .. nr - 1 sum to ``generate``'s aLT, aLE, aNLT, aNLE, aT, aE."""
    sel = np.arange(j0, j1)
    phiL = phi_linear(K, noise)[:, sel]
    if mu is None:
        mu = mu_ensemble(K)
    qT = quadrature_weights(r, w, alphaT)[:, sel]
    qE = quadrature_weights(r, w, alphaE)[:, sel]
    phiNL = phi_nonlinear(phiL, np.asarray(mu)[sel], grid)
    out = {"phiL": phiL, "phiNL": phiNL,
           "aLT": radial_quadrature(phiL, qT), "aLE": radial_quadrature(phiL, qE),
           "aNLT": radial_quadrature(phiNL, qT), "aNLE": radial_quadrature(phiNL, qE)}
    out["aT"] = out["aLT"] + fnl * out["aNLT"]
    out["aE"] = out["aLE"] + fnl * out["aNLE"]
    return out


# ---------------------------------------------------------------------------
# Adjoint of the generator (differentiation form): gradients of a real loss L of
# a^T and a^E with respect to the white noise n and to f_NL.  Complex numbers are
# treated as pairs of reals, and a gradient array holds dL/dRe + i dL/dIm.  Each
# function below is the transpose, under the real inner product <u, v> =
# sum Re(conj(u) v), of the corresponding forward map above.
# ---------------------------------------------------------------------------

def synthesis_adjoint(fbar: np.ndarray, grid: Grid) -> np.ndarray:
    """Transpose of ``synthesis``: fbar [nsh, n_theta, n_phi] real -> [nalm, nsh].

    The forward map is f_jk = sum_l [Re a_l0 lambda_l0 + 2 sum_{m>0} lambda_lm (Re a_lm cos m phi_k
    - Im a_lm sin m phi_k)], so dL/dRe a_lm = c_m sum_jk lambda_lm(x_j) cos(m phi_k) fbar_jk and
    dL/dIm a_lm = -c_m sum_jk lambda_lm(x_j) sin(m phi_k) fbar_jk, with c_0 = 1, c_m = 2 (m > 0),
    and 0 for Im a_l0 (the forward ignores it).  sum_k fbar_jk e^{-i m phi_k} is rfft(fbar)_m."""
    L = grid.lmax
    fbar = np.asarray(fbar, dtype=np.float64)
    if fbar.ndim == 2:
        fbar = fbar[None]
    nsh = fbar.shape[0]
    Fb = np.fft.rfft(fbar, axis=-1)  # [nsh, ntheta, nphi/2+1]
    out = np.zeros((n_alm(L), nsh), dtype=np.complex128)
    for m in range(L + 1):
        rows = alm_index(np.arange(m, L + 1), m, L)
        c = 1.0 if m == 0 else 2.0
        out[rows, :] = c * (grid.lam(m) @ Fb[:, :, m].T)
    out[: L + 1, :] = out[: L + 1, :].real
    return out


def analysis_adjoint(abar: np.ndarray, grid: Grid) -> np.ndarray:
    """Transpose of ``analysis``: abar [nalm, nsh] -> [nsh, n_theta, n_phi] real.

    The forward map is Re a_lm = W_j sum lambda_lm cos(m phi_k) f_jk and Im a_lm =
    -W_j sum lambda_lm sin(m phi_k) f_jk with W_j = w_j 2 pi / n_phi, so
    dL/df_jk = W_j sum_lm lambda_lm(x_j) Re(abar_lm e^{i m phi_k}) over m >= 0, every m once:
    an inverse real DFT of B_m(x_j) = sum_l lambda_lm abar_lm with the m > 0 terms halved
    (irfft doubles them)."""
    L = grid.lmax
    abar = np.asarray(abar, dtype=np.complex128)
    if abar.ndim == 1:
        abar = abar[:, None]
    nsh = abar.shape[1]
    B = np.zeros((nsh, grid.ntheta, grid.nphi // 2 + 1), dtype=np.complex128)
    for m in range(L + 1):
        rows = alm_index(np.arange(m, L + 1), m, L)
        B[:, :, m] = (grid.lam(m).T @ abar[rows, :]).T * (1.0 if m == 0 else 0.5)
    f = np.fft.irfft(B, n=grid.nphi, axis=-1) * grid.nphi
    return f * (grid.w * (2.0 * math.pi / grid.nphi))[None, :, None]


def phi_linear_adjoint(K: np.ndarray, phibar: np.ndarray) -> np.ndarray:
    """Transpose of ``phi_linear``: phibar [nalm, nr] -> noise gradient [nr, nalm],
    nbar_lm(r_j) = sum_i K_l[i, j] phibar_lm(r_i); 0 for Im n_l0 (the forward ignores it)."""
    L = K.shape[0] - 1
    phibar = np.asarray(phibar, dtype=np.complex128)
    out = np.empty((phibar.shape[0], K.shape[2]), dtype=np.complex128)
    for l in range(L + 1):
        rows = alm_index(l, np.arange(l + 1), L)
        out[rows, :] = phibar[rows, :] @ K[l]
    out[: L + 1, :] = out[: L + 1, :].real
    return out.T.copy()


def radial_quadrature_adjoint(abar: np.ndarray, q: np.ndarray) -> np.ndarray:
    """Transpose of ``radial_quadrature``: abar [nalm] -> [nalm, nr], phibar_lm(r_i) = q_l[i] abar_lm."""
    L = q.shape[0] - 1
    ls, _ = _lm_arrays(L)
    return np.asarray(abar, dtype=np.complex128)[:, None] * q[ls, :]


def _lm_arrays(L: int):
    ls = np.concatenate([np.arange(m, L + 1) for m in range(L + 1)])
    ms = np.concatenate([np.full(L + 1 - m, m) for m in range(L + 1)])
    return ls, ms


def generate_backward(K, noise, grid: Grid, r, w, alphaT, alphaE, fnl: float, gT, gE, mu=None):
    """Gradients of a real loss L(a^T, a^E) given gX = dL/da^X (pairs, [nalm] complex):
    returns (dL/dn [nr, nalm] complex, dL/df_NL float).

    By the chain rule through the forward recipe, with q^X the quadrature weights:
      dL/df_NL      = sum_X <gX, a^X_NL>
      dL/dPhi_NL    = f_NL sum_X q^X gX                        (quadrature, Eq. 5)
      dL/dg         = analysis^T(dL/dPhi_NL)                    (step (iv))
      dL/df         = 2 f dL/dg, f = synthesis(Phi_L)           (square, Eq. 2; mu is a constant)
      dL/dPhi_L     = synthesis^T(dL/df) + sum_X q^X gX         (step (ii) and the linear part)
      dL/dn         = phi_linear^T(dL/dPhi_L)                   (step (i), Eq. 9)"""
    fw = generate(K, noise, grid, r, w, alphaT, alphaE, fnl, mu=mu)
    gT = np.asarray(gT, dtype=np.complex128)
    gE = np.asarray(gE, dtype=np.complex128)
    dfnl = float(np.sum((np.conj(gT) * fw["aNLT"]).real) + np.sum((np.conj(gE) * fw["aNLE"]).real))
    qT = quadrature_weights(r, w, alphaT)
    qE = quadrature_weights(r, w, alphaE)
    lin = radial_quadrature_adjoint(gT, qT) + radial_quadrature_adjoint(gE, qE)
    gbar = analysis_adjoint(fnl * lin, grid)
    f = synthesis(fw["phiL"], grid)
    phibar = synthesis_adjoint(2.0 * f * gbar, grid) + lin
    return phi_linear_adjoint(K, phibar), dfnl


# ---------------------------------------------------------------------------
# Output maps: Stokes I, Q, U on the ring grid from a^T, a^E, a^B.  The paper's deliverable is
# temperature and polarization maps, the three Stokes maps I, Q, U (Sect. 4; its Fig. 2 shows
# I and the polarization intensity sqrt(Q^2 + U^2)).
# ---------------------------------------------------------------------------

def spin2_functions(m: int, grid: Grid) -> tuple[np.ndarray, np.ndarray]:
    """W_lm(x_j) and X_lm(x_j) for l = m..lmax, shape [lmax - m + 1, n_theta] each, with
    W = (2lam + (-2)lam) / 2 and X = (2lam - (-2)lam) / 2, where sY_lm = slam_lm(theta) e^{i m phi}.

    Definition: the spin-weighted harmonics come from Y_lm by the spin raising and lowering
    operators, 2Y_lm = N_l edth^2 Y_lm and -2Y_lm = N_l edthbar^2 Y_lm, N_l = ((l-1) l (l+1) (l+2))^(-1/2),
    with edth eta = -(sin th)^s (d_th + i / sin th d_phi)[(sin th)^(-s) eta] on spin weight s and
    edthbar eta = -(sin th)^(-s) (d_th - i / sin th d_phi)[(sin th)^s eta].  Applied twice to
    lam_lm e^{i m phi}, with the Legendre equation for lam'' and
    sin th lam'_lm = l x lam_lm - c_lm lam_{l-1,m}, c_lm = sqrt((2l+1)(l^2 - m^2) / (2l-1)):
       W = N_l [((2 m^2 - 2 l x^2) lam_lm + 2 x c_lm lam_{l-1,m}) / sin^2 th - l (l+1) lam_lm]
       X = N_l 2 m [(1 - l) x lam_lm + c_lm lam_{l-1,m}] / sin^2 th,
    both 0 for l < 2."""
    L = grid.lmax
    x = grid.x
    lam = grid.lam(m)                                       # [L - m + 1, ntheta], l = m..L
    prev = np.vstack([np.zeros((1, x.size)), lam[:-1]])     # lam_{l-1,m} (zero at l = m)
    ls = np.arange(m, L + 1, dtype=np.float64)[:, None]
    c = np.sqrt((2 * ls + 1) * (ls * ls - m * m) / np.maximum(2 * ls - 1, 1.0))
    s2 = (1.0 - x) * (1.0 + x)
    with np.errstate(divide="ignore", invalid="ignore"):
        nl = np.where(ls >= 2, 1.0 / np.sqrt(np.maximum((ls - 1) * ls * (ls + 1) * (ls + 2), 1.0)), 0.0)
    W = nl * (((2.0 * m * m - 2.0 * ls * x * x) * lam + 2.0 * x * c * prev) / s2 - ls * (ls + 1) * lam)
    X = nl * 2.0 * m * ((1.0 - ls) * x * lam + c * prev) / s2
    return W, X


def maps_iqu(aT, aE, aB, grid: Grid) -> np.ndarray:
    """Stokes maps [3, n_theta, n_phi] = (I, Q, U) of one realisation.

    I = sum_lm a^T_lm Y_lm (the spin-0 synthesis); Q + iU = sum_lm a_{2,lm} 2Y_lm and
    Q - iU = sum_lm a_{-2,lm} -2Y_lm with a_{+-2,lm} = -(a^E_lm +- i a^B_lm) (the convention of
    HEALPix, whose maps the paper makes).  With a_{l,-m} = (-1)^m conj(a_lm) for E and B,
    W_{l,-m} = (-1)^m W_lm and X_{l,-m} = -(-1)^m X_lm, every ring reduces to m >= 0:
       Q_m = -sum_l (E_lm W_lm + i B_lm X_lm),   U_m = sum_l (i E_lm X_lm - B_lm W_lm),
       Q = Q_0 + 2 Re sum_{m>0} Q_m e^{i m phi},  likewise U (X_l0 = 0).
    aB may be None (zero)."""
    L = grid.lmax
    aT = np.asarray(aT, dtype=np.complex128)
    aE = np.asarray(aE, dtype=np.complex128)
    aB = np.zeros_like(aE) if aB is None else np.asarray(aB, dtype=np.complex128)
    half = grid.nphi // 2 + 1
    Qm = np.zeros((grid.ntheta, half), dtype=np.complex128)
    Um = np.zeros_like(Qm)
    for m in range(L + 1):
        rows = alm_index(np.arange(m, L + 1), m, L)
        W, X = spin2_functions(m, grid)
        E, B = aE[rows], aB[rows]
        Qm[:, m] = -(W.T @ E + 1j * (X.T @ B))
        Um[:, m] = 1j * (X.T @ E) - W.T @ B
    I = synthesis(aT[:, None], grid)[0]
    Q = np.fft.irfft(Qm, n=grid.nphi, axis=-1) * grid.nphi
    U = np.fft.irfft(Um, n=grid.nphi, axis=-1) * grid.nphi
    return np.stack([I, Q, U])


def analysis_spin2(Q: np.ndarray, U: np.ndarray, grid: Grid) -> tuple[np.ndarray, np.ndarray]:
    """(a^E, a^B) from Q, U maps [n_theta, n_phi]: a_{+-2,lm} = int (Q +- iU) +-2Y*_lm dOmega by GL
    quadrature and the rectangle rule, then a^E = -(a_2 + a_-2) / 2, a^B = i (a_2 - a_-2) / 2, i.e.
       a^E_lm = -sum_j w_j (W_lm Q^_m + i X_lm U^_m),  a^B_lm = sum_j w_j (i X_lm Q^_m - W_lm U^_m),
    Q^_m = (2 pi / n_phi) sum_k Q_jk e^{-i m phi_k}.  Exact for band-limited maps on this grid."""
    L = grid.lmax
    Qh = np.fft.rfft(np.asarray(Q, dtype=np.float64), axis=-1) * (2.0 * math.pi / grid.nphi)
    Uh = np.fft.rfft(np.asarray(U, dtype=np.float64), axis=-1) * (2.0 * math.pi / grid.nphi)
    aE = np.zeros(n_alm(L), dtype=np.complex128)
    aB = np.zeros_like(aE)
    for m in range(L + 1):
        rows = alm_index(np.arange(m, L + 1), m, L)
        W, X = spin2_functions(m, grid)
        q, u = grid.w * Qh[:, m], grid.w * Uh[:, m]
        aE[rows] = -(W @ q + 1j * (X @ u))
        aB[rows] = 1j * (X @ q) - W @ u
    return aE, aB


__all__ = [
    "FOUR_PI", "FLUSH", "gauss_legendre", "lambda_mm", "lambda_column", "lambda_table", "Grid",
    "synthesis", "analysis", "spherical_jn_table", "k_rule", "covariance", "filters",
    "mu_ensemble", "philox4x64", "philox_noise", "phi_linear", "phi_nonlinear",
    "quadrature_weights", "radial_quadrature", "generate", "generate_shard", "synthesis_adjoint", "analysis_adjoint",
    "phi_linear_adjoint", "radial_quadrature_adjoint", "generate_backward", "spin2_functions", "maps_iqu",
    "analysis_spin2",
]
