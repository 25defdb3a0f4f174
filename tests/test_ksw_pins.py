"""Pins of the cubic-estimator oracle (oracle/ksw_oracle.py) to facts other than itself (CPU).

- (l1 l2 l3; 0 0 0) against Racah's exact 3j symbols.
- S_prim (grid synthesis and the grid's quadrature) against the Gaunt brute-force sum
  sum_s w_s r_s^2 sum_{l_k, m_k} A_{l1m1} B_{l2m2} B_{l3m3} int Y Y Y, all m of both signs.
- The normalisation summed as the paper writes it against the Legendre-quadrature form.
- The normalisation against the exact variance of S_prim over Gaussian skies of covariance
  C_l, from Wick's theorem applied to the cubic form of S_prim (its coefficients extracted by
  polarisation of the oracle's own S_prim); the mean of S_prim is zero.
- With E proportional to T (the workload's kernels) the pseudo-inverse estimator is the
  temperature-only one.
- Sampled Gaussian skies: mean and variance of f_NL = S_prim / N.
- Planted mistakes in the normalisation (no Delta, no factor 2, C in place of C^-1) fail the
  Wick pin.
"""
import itertools
import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.wigner import gaunt, wigner3j


def _independent_kernels(L, nr, seed):
    """Transfer kernels whose T and E parts are not proportional (C_l of full rank)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(0.5, 1.5, (L + 1, nr)), rng.uniform(-1.0, 1.0, (L + 1, nr))


def _weights(L, nr, independent, seed=3):
    r, w = W.radial_grid(nr)
    if independent:
        aT, aE = _independent_kernels(L, nr, seed)
    else:
        aT, aE = W.transfer_kernels(L, r)
    K = W.random_lower_filters(L, nr, seed=seed, scale=1e-4)
    return O.ksw_weights(K, r, w, aT, aE)


def _gaussian_sky(wts, L, rng):
    """a^T, a^E with <a^X_lm conj(a^Y_lm)> = C^XY_l (m = 0 real)."""
    aT = np.zeros(W.n_alm(L), complex)
    aE = np.zeros_like(aT)
    for l in range(L + 1):
        lam, vec = np.linalg.eigh(wts["C"][l])
        S = vec * np.sqrt(np.maximum(lam, 0.0))[None, :]
        for m in range(l + 1):
            i = W.alm_index(l, m, L)
            if m == 0:
                z = S @ rng.standard_normal(2)
            else:
                z = S @ (rng.standard_normal(2) + 1j * rng.standard_normal(2)) / math.sqrt(2.0)
            aT[i], aE[i] = z
    return aT, aE


def test_three_j_000_against_racah():
    for l1, l2, l3 in itertools.product(range(9), repeat=3):
        assert abs(O.three_j_000(l1, l2, l3) - wigner3j(l1, l2, l3, 0, 0, 0)) < 1e-14


@pytest.mark.parametrize("independent", [True, False])
def test_statistic_matches_gaunt_brute_force(independent):
    L, nr = 4, 2
    wts = _weights(L, nr, independent)
    a = W.random_alm(L, 2, seed=8)
    aT, aE = a[:, 0], a[:, 1]
    grid = O.Grid(L, 8, 13)   # exact for the cubic: 2 * 8 - 1 >= 3 L, 13 >= 3 L + 1
    S = O.ksw_statistic(aT, aE, grid, wts)
    At, Bt = O.ksw_filtered(aT, aE, wts)

    def full(col, l, m):
        v = col[W.alm_index(l, abs(m), L)]
        return v if m >= 0 else (-1) ** m * np.conj(v)

    ref = 0.0
    lms = [(l, m) for l in range(L + 1) for m in range(-l, l + 1)]
    for s in range(nr):
        tot = 0.0
        for (l1, m1), (l2, m2) in itertools.product(lms, lms):
            m3 = -m1 - m2
            for l3 in range(abs(m3), L + 1):
                g = gaunt(l1, l2, l3, m1, m2, m3)
                if g != 0.0:
                    tot += g * full(At[:, s], l1, m1) * full(Bt[:, s], l2, m2) * full(Bt[:, s], l3, m3)
        assert abs(tot.imag) < 1e-10 * abs(tot.real)
        ref += wts["u"][s] * tot.real
    assert abs(S - ref) < 1e-12 * abs(ref)


@pytest.mark.parametrize("independent,L,nr", [(True, 10, 3), (False, 10, 3), (True, 16, 2), (False, 24, 2)])
def test_normalisation_direct_equals_quadrature_form(independent, L, nr):
    wts = _weights(L, nr, independent)
    assert (wts["rank"][2:] == (2 if independent else 1)).all() and (wts["rank"][:2] == 0).all()
    nd = O.ksw_normalisation_direct(wts)
    nq = O.ksw_normalisation(wts)
    assert nd > 0 and abs(nd - nq) < 1e-12 * nd


def _cubic_form(wts, L, grid):
    """Symmetric T with S_prim(p) = sum T_abc p_a p_b p_c over the real parameters p of
    (a^T, a^E) at l >= 2, by polarisation of the oracle's S_prim; and the covariance of p."""
    params = []   # (field, l, m, part)
    for f in range(2):
        for l in range(2, L + 1):
            params.append((f, l, 0, 0))
            for m in range(1, l + 1):
                params += [(f, l, m, 0), (f, l, m, 1)]
    n = len(params)

    def alm_of(p):
        a = [np.zeros(W.n_alm(L), complex), np.zeros(W.n_alm(L), complex)]
        for v, (f, l, m, part) in zip(p, params):
            if v:
                a[f][W.alm_index(l, m, L)] += v * (1j if part else 1.0)
        return a

    cache = {}

    def S(idx):
        key = tuple(sorted(idx))
        if key not in cache:
            p = np.zeros(n)
            for i in idx:
                p[i] += 1.0
            aT, aE = alm_of(p)
            cache[key] = O.ksw_statistic(aT, aE, grid, wts)
        return cache[key]

    T = np.zeros((n, n, n))
    for a, b, c in itertools.combinations_with_replacement(range(n), 3):
        v = (S((a, b, c)) - S((a, b)) - S((a, c)) - S((b, c)) + S((a,)) + S((b,)) + S((c,))) / 6.0
        for perm in set(itertools.permutations((a, b, c))):
            T[perm] = v
    cov = np.zeros((n, n))
    for i, (f, l, m, part) in enumerate(params):
        for j, (g, l2, m2, part2) in enumerate(params):
            if (l, m, part) == (l2, m2, part2):
                cov[i, j] = wts["C"][l][f, g] * (1.0 if m == 0 else 0.5)
    return T, cov


@pytest.mark.parametrize("independent", [True, False])
def test_normalisation_is_gaussian_variance_of_statistic(independent):
    L, nr = 3, 2
    wts = _weights(L, nr, independent)
    grid = O.Grid(L, 6, 10)   # exact for the cubic
    T, cov = _cubic_form(wts, L, grid)
    lin = np.einsum("abc,bc->a", T, cov)                  # E[S] = 0 needs the linear part to vanish
    full = 6.0 * np.einsum("abc,ad,be,cf,def->", T, cov, cov, cov, T)
    part = 9.0 * lin @ cov @ lin
    N = O.ksw_normalisation_direct(wts)
    assert abs(part) < 1e-12 * full
    assert abs(full - N) < 1e-10 * N
    # planted mistakes, each far outside that bar
    Cinv, C = wts["Cinv"], wts["C"]

    def planted(delta_one=False, half_b=False, use_C=False):
        tot = 0.0
        for l1 in range(L + 1):
            for l2 in range(l1, L + 1):
                for l3 in range(l2, min(L, l1 + l2) + 1):
                    w3 = O.three_j_000(l1, l2, l3)
                    if w3 == 0.0 or min(l1, l2, l3) < 2:
                        continue
                    I = math.sqrt((2 * l1 + 1) * (2 * l2 + 1) * (2 * l3 + 1) / (4 * math.pi)) * w3
                    B = I * O.ksw_bispectrum(l1, l2, l3, wts) * (0.5 if half_b else 1.0)
                    M = C if use_C else Cinv
                    d = 1.0 if delta_one else (6.0 if l1 == l2 == l3 else 2.0 if (l1 == l2 or l2 == l3) else 1.0)
                    tot += float(np.einsum("ijk,io,jp,kq,opq->", B, M[l1], M[l2], M[l3], B)) / d
        return tot

    assert abs(planted() - full) < 1e-10 * full
    for kw in ({"delta_one": True}, {"half_b": True}, {"use_C": True}):
        assert abs(planted(**kw) - full) > 0.05 * full, kw


def test_pseudo_inverse_is_temperature_only_when_e_follows_t():
    L, nr = 12, 3
    r, w = W.radial_grid(nr)
    aT_k, aE_k = W.transfer_kernels(L, r)
    K = W.random_lower_filters(L, nr, seed=5, scale=1e-4)
    both = O.ksw_weights(K, r, w, aT_k, aE_k)
    tonly = O.ksw_weights(K, r, w, aT_k, np.zeros_like(aE_k))
    assert (both["rank"][2:] == 1).all() and (tonly["rank"][2:] == 1).all()
    c = 0.1 * np.sin(np.arange(L + 1) / 50.0)          # alpha^E_l = c_l alpha^T_l
    aT = W.random_alm(L, 1, seed=2)[:, 0]
    ls, _ = W.alm_lm(L)
    aE = c[ls] * aT
    grid = O.Grid(L, 19, 40)
    s_both = O.ksw_statistic(aT, aE, grid, both)
    s_t = O.ksw_statistic(aT, np.zeros_like(aT), grid, tonly)
    assert abs(s_both - s_t) < 1e-11 * abs(s_t)
    n_both, n_t = O.ksw_normalisation_direct(both), O.ksw_normalisation_direct(tonly)
    assert abs(n_both - n_t) < 1e-11 * n_t


@pytest.mark.slow
def test_sampled_gaussian_skies_give_unbiased_unit_variance():
    """f_NL = S_prim / N over 400 Gaussian skies: mean 0 within 4 standard errors, variance
    1/N within 4 standard errors of a sample variance (sqrt(2 / M))."""
    L, nr, M = 12, 3, 400
    wts = _weights(L, nr, True)
    N = O.ksw_normalisation_direct(wts)
    grid = O.Grid(L, 19, 40)
    rng = np.random.default_rng(11)
    f = np.array([O.ksw_statistic(*_gaussian_sky(wts, L, rng), grid, wts) / N for _ in range(M)])
    sigma = 1.0 / math.sqrt(N)
    assert abs(f.mean()) < 4 * sigma / math.sqrt(M)
    assert abs(f.var() / sigma ** 2 - 1.0) < 4 * math.sqrt(2.0 / M)
