"""Plain FP64 CPU oracle of the fast cubic f_NL estimator (Sect. 5 of Elsner & Wandelt).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: only ``tests/``,
``__graft_entry__.smoke()`` and the CPU legs of ``bench.py`` may import it.  It shares no
code with the CUDA library.

What it computes (Sect. 5, the estimator the paper runs on its maps):

  A(r, n) = sum_{i,j in T,E} sum_lm (C^-1)^{ij}_l alpha^i_l(r) a^j_lm Y_lm(n)
  B(r, n) = sum_{i,j in T,E} sum_lm (C^-1)^{ij}_l beta^i_l(r)  a^j_lm Y_lm(n)
  S_prim  = int dr r^2 int d^2n A B^2
  f_NL    = S_prim / N,   N = sum_{ijk,opq} sum_{l1<=l2<=l3} B^{ijk}_{l1l2l3} (C^-1)^{io}_{l1}
            (C^-1)^{jp}_{l2} (C^-1)^{kq}_{l3} B^{opq}_{l1l2l3} / Delta_{l1l2l3}
  B^{ijk}_{l1l2l3} = 2 I_{l1l2l3} int dr r^2 [beta^i_l1 beta^j_l2 alpha^k_l3
                     + beta^k_l3 beta^i_l1 alpha^j_l2 + beta^j_l2 beta^k_l3 alpha^i_l1]
  I_{l1l2l3} = sqrt((2l1+1)(2l2+1)(2l3+1) / (4 pi)) (l1 l2 l3; 0 0 0)

Readings, for the synthetic shells of the generator (each also in the function that takes it):
  - beta^X_l(r_i) = sum_j (K_l K_l^T)[i, j] w_j r_j^2 alpha^X_l(r_j).  The paper's beta is
    4 pi int dk Delta^2(k)/k g_l(k) j_l(kr) with alpha = (2/pi) int dk k^2 g_l j_l; as
    4 pi Delta^2/k = (2/pi) k^2 P(k), beta_l(r) = int dr' r'^2 C_l(r, r') alpha_l(r'), whose
    discrete form on the shells, with the covariance the filters realise, is the line above:
    the covariance of Phi_L(r_i) with a^X_L.
  - C_l = [[C^TT, C^TE], [C^TE, C^EE]] is the covariance of (a^T_L, a^E_L) of the generator,
    C^XY_l = (K_l^T q^X_l) . (K_l^T q^Y_l), q^X_l[i] = w_i r_i^2 alpha^X_l(r_i).
  - C^-1 is the Moore-Penrose inverse: the full inverse when the smaller eigenvalue of C_l
    exceeds 1e-10 of the larger, else v v^T / lambda of the leading eigenpair (T and E
    proportional, as with the workload's kernels alpha^E = 0.1 sin(l/50) alpha^T).  Degrees
    l < 2 are left out (C^-1 = 0), as C^EE_0 = 0.
  - int dr r^2 is the shells' quadrature sum_i w_i r_i^2; int d^2n is the Gauss-Legendre x
    rectangle rule of the map grid, exact for the cubic when n_theta >= (3 l_max + 2) / 2 and
    n_phi >= 3 l_max + 1.

``ksw_normalisation`` evaluates the same N by the identity
int_-1^1 P_l1 P_l2 P_l3 dx = 2 (l1 l2 l3; 0 0 0)^2, exact with a Gauss-Legendre rule of
ceil((3 l_max + 1) / 2) nodes; it is pinned against the direct sum of the paper's form and
serves where that sum is too slow in Python (large l_max, rank-one or well-conditioned C_l).

Pins (tests/test_ksw_pins.py, CPU): (l1 l2 l3; 0 0 0) against Racah's exact 3j; S_prim against
the Gaunt brute-force sum at small l_max; the direct normalisation against the quadrature
form; N against the exact Gaussian variance of S_prim (Wick's theorem on its cubic form);
the pseudo-inverse against the T-only estimator when E is proportional to T; sampled
Gaussian skies (mean and variance of f_NL).
"""
from __future__ import annotations

import math

import numpy as np

from workloads import alm_index

from .fnl_oracle import Grid, gauss_legendre, synthesis

RANK_RCOND = 1e-10
LMIN = 2


def ksw_weights(K: np.ndarray, r, w, alphaT, alphaE, lmin: int = LMIN, rcond: float = RANK_RCOND) -> dict:
    """Per-degree ingredients of the estimator from the generator's shells.

    K: [l_max+1, nr, nr] filters (K_l K_l^T = the realised covariance of Phi_L).
    Returns alpha, beta [2, l_max+1, nr] (T, E), C, Cinv [l_max+1, 2, 2], rank [l_max+1],
    u [nr] = w_i r_i^2."""
    r = np.asarray(r, dtype=np.float64)
    u = np.asarray(w, dtype=np.float64) * r * r
    alpha = np.stack([np.asarray(alphaT, dtype=np.float64), np.asarray(alphaE, dtype=np.float64)])
    L1 = alpha.shape[1]
    q = alpha * u[None, None, :]
    cov = np.einsum("lij,lkj->lik", K, K)                       # K_l K_l^T
    beta = np.einsum("lik,xlk->xli", cov, q)                     # (K K^T) q^X
    v = np.einsum("lji,xlj->xli", K, q)                          # K^T q^X
    C = np.einsum("xli,yli->lxy", v, v)
    Cinv = np.zeros_like(C)
    rank = np.zeros(L1, dtype=int)
    for l in range(lmin, L1):
        lam, vec = np.linalg.eigh(C[l])                          # ascending
        if lam[1] <= 0.0:
            continue
        if lam[0] > rcond * lam[1]:
            Cinv[l] = np.linalg.inv(C[l])
            rank[l] = 2
        else:
            Cinv[l] = np.outer(vec[:, 1], vec[:, 1]) / lam[1]
            rank[l] = 1
    return {"alpha": alpha, "beta": beta, "C": C, "Cinv": Cinv, "rank": rank, "u": u}


def ksw_filtered(aT, aE, wts: dict) -> tuple[np.ndarray, np.ndarray]:
    """Coefficients of A and B on every shell, [nalm, nr] each:
    A_lm(r) = sum_{i,j} (C^-1)^{ij}_l alpha^i_l(r) a^j_lm, B likewise with beta."""
    a = np.stack([np.asarray(aT, dtype=np.complex128), np.asarray(aE, dtype=np.complex128)])
    L = wts["Cinv"].shape[0] - 1
    fA = np.einsum("xlr,lxy->ylr", wts["alpha"], wts["Cinv"])    # [j, l, r]
    fB = np.einsum("xlr,lxy->ylr", wts["beta"], wts["Cinv"])
    nr = fA.shape[2]
    At = np.zeros((a.shape[1], nr), dtype=np.complex128)
    Bt = np.zeros_like(At)
    for m in range(L + 1):
        ls = np.arange(m, L + 1)
        rows = alm_index(ls, m, L)
        for j in range(2):
            At[rows] += fA[j][ls] * a[j][rows][:, None]
            Bt[rows] += fB[j][ls] * a[j][rows][:, None]
    return At, Bt


def ksw_statistic(aT, aE, grid: Grid, wts: dict) -> float:
    """S_prim = sum_i w_i r_i^2 int A(r_i) B(r_i)^2 d^2n, the sphere by the grid's rule:
    sum_j w^GL_j (2 pi / n_phi) sum_k."""
    At, Bt = ksw_filtered(aT, aE, wts)
    A = synthesis(At, grid)
    B = synthesis(Bt, grid)
    ring = np.einsum("sjk->sj", A * B * B)
    sphere = ring @ grid.w * (2.0 * math.pi / grid.nphi)
    return float(np.dot(wts["u"], sphere))


def three_j_000(l1: int, l2: int, l3: int) -> float:
    """(l1 l2 l3; 0 0 0): zero unless the triangle holds and J = l1 + l2 + l3 is even; then
    (-1)^(J/2) sqrt((J-2l1)! (J-2l2)! (J-2l3)! / (J+1)!) (J/2)! / ((J/2-l1)! (J/2-l2)! (J/2-l3)!),
    evaluated through log-gamma."""
    J = l1 + l2 + l3
    if J % 2 or l3 < abs(l1 - l2) or l3 > l1 + l2:
        return 0.0
    g = J // 2
    lg = math.lgamma
    v = 0.5 * (lg(J - 2 * l1 + 1) + lg(J - 2 * l2 + 1) + lg(J - 2 * l3 + 1) - lg(J + 2))
    v += lg(g + 1) - lg(g - l1 + 1) - lg(g - l2 + 1) - lg(g - l3 + 1)
    return (-1.0) ** g * math.exp(v)


def ksw_bispectrum(l1: int, l2: int, l3: int, wts: dict) -> np.ndarray:
    """b^{ijk}_{l1l2l3} = 2 sum_s u_s [beta^i_l1 beta^j_l2 alpha^k_l3 + beta^k_l3 beta^i_l1 alpha^j_l2
    + beta^j_l2 beta^k_l3 alpha^i_l1](r_s), [2, 2, 2]; B^prim = I_{l1l2l3} b."""
    al, be, u = wts["alpha"], wts["beta"], wts["u"]
    t = (np.einsum("s,is,js,ks->ijk", u, be[:, l1], be[:, l2], al[:, l3])
         + np.einsum("s,ks,is,js->ijk", u, be[:, l3], be[:, l1], al[:, l2])
         + np.einsum("s,js,ks,is->ijk", u, be[:, l2], be[:, l3], al[:, l1]))
    return 2.0 * t


def ksw_normalisation_direct(wts: dict) -> float:
    """The paper's normalisation, summed as written: over l1 <= l2 <= l3 <= l_max, with
    Delta = 6 (all equal), 2 (two equal), 1, B^prim = I b and the three C^-1 contractions."""
    Cinv = wts["Cinv"]
    L = Cinv.shape[0] - 1
    total = 0.0
    for l1 in range(L + 1):
        for l2 in range(l1, L + 1):
            for l3 in range(l2, min(L, l1 + l2) + 1):
                w3 = three_j_000(l1, l2, l3)
                if w3 == 0.0:
                    continue
                I = math.sqrt((2 * l1 + 1) * (2 * l2 + 1) * (2 * l3 + 1) / (4.0 * math.pi)) * w3
                B = I * ksw_bispectrum(l1, l2, l3, wts)
                if Cinv[l1].any() and Cinv[l2].any() and Cinv[l3].any():
                    CB = np.einsum("io,jp,kq,opq->ijk", Cinv[l1], Cinv[l2], Cinv[l3], B)
                    delta = 6.0 if l1 == l2 == l3 else 2.0 if (l1 == l2 or l2 == l3) else 1.0
                    total += float(np.sum(B * CB)) / delta
    return total


def ksw_normalisation(wts: dict, nx: int | None = None) -> float:
    """The same N through int P_l1 P_l2 P_l3 dx = 2 (l1 l2 l3; 0 0 0)^2 and the symmetry of the
    summand (sum over l1 <= l2 <= l3 with 1/Delta = 1/6 of the sum over all ordered triples):
       N = 1/(12 pi) sum_{r,r'} u_r u_r' int dx [3 F^aa F^bb F^bb + 6 F^ab F^ba F^bb](x; r, r'),
       F^XY(x; r, r') = sum_l (2l+1) P_l(x) X_l(r)^T C^-1_l Y_l(r'),   X, Y in {alpha, beta},
    the x integral by Gauss-Legendre with nx >= (3 l_max + 1) / 2 nodes (exact).

    Exact in exact arithmetic, but the signed sums over (r, r') and x cancel when C_l is
    ill-conditioned (the weak eigen-direction of C^-1 enters every F): it agrees with the
    direct sum to ~1e-14 for a rank-one or well-conditioned C_l, and is used only there."""
    al, be, Cinv, u = wts["alpha"], wts["beta"], wts["Cinv"], wts["u"]
    L = Cinv.shape[0] - 1
    if nx is None:
        nx = (3 * L + 2) // 2
    x, wx = gauss_legendre(nx)
    P = np.polynomial.legendre.legvander(x, L) * (2.0 * np.arange(L + 1) + 1.0)[None, :]   # [nx, L+1]

    def pair(X, Y):
        return np.einsum("xlr,lxy,yls->lrs", X, Cinv, Y)          # [l, r, r']

    F = {k: np.einsum("gl,lrs->grs", P, pair(X, Y)) for k, (X, Y) in
         {"aa": (al, al), "bb": (be, be), "ab": (al, be), "ba": (be, al)}.items()}
    Q = 3.0 * F["aa"] * F["bb"] ** 2 + 6.0 * F["ab"] * F["ba"] * F["bb"]
    return float(np.einsum("g,r,s,grs->", wx, u, u, Q)) / (12.0 * math.pi)


__all__ = ["RANK_RCOND", "LMIN", "ksw_weights", "ksw_filtered", "ksw_statistic", "three_j_000", "ksw_bispectrum",
           "ksw_normalisation_direct", "ksw_normalisation"]
