"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test names what fixes the expected value: a library routine (numpy, scipy,
mpmath), a closed form (Gaunt integrals from Racah's 3j formula, Parseval,
the addition theorem), an exact symmetry of the method, or a seeded ensemble
statistic.  The mutation tests at the end plant mistakes in the oracle (on the
CPU) and check that at least one pin catches each of them.
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.wigner import gaunt, wigner3j

# ---------------------------------------------------------------------------
# Grid and Legendre functions
# ---------------------------------------------------------------------------


@pytest.mark.parametrize("n", [1, 2, 3, 5, 25, 49, 100, 385, 769])
def test_gauss_legendre_matches_numpy_and_integrates_polynomials(n):
    x, w = O.gauss_legendre(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    assert np.all(np.diff(x) < 0)  # north to south
    assert np.max(np.abs(x - xr[::-1])) < 1e-14
    # numpy's own weights are only good to ~1e-9 at n ~ 1000; the moment test below is the sharp pin
    assert np.max(np.abs(w - wr[::-1]) / wr[::-1]) < 5e-9
    for k in range(0, 2 * n, max(1, (2 * n) // 12)):
        exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
        assert abs(np.dot(w, x ** k) - exact) < 1e-13


def test_lambda_matches_scipy_spherical_harmonics_low_l():
    sp = pytest.importorskip("scipy.special")
    L = 40
    x, _ = O.gauss_legendre(31)
    theta = np.arccos(x)
    tab = O.lambda_table(L, x)
    for m in range(L + 1):
        for l in range(m, L + 1):
            ref = sp.sph_harm_y(l, m, theta, 0.0).real  # includes the Condon-Shortley phase
            assert np.max(np.abs(tab[m][l - m] - ref)) < 1e-13, (l, m)


def test_lambda_high_l_matches_mpmath():
    # arbitrary-precision associated Legendre function (hypergeometric series) at l up to 1024
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    L = 1024
    cases = [(1024, 0, 0.7), (1024, 0, 0.9999), (1024, 7, 0.1), (1024, 300, 0.7), (1024, 900, 0.1),
             (662, 300, 0.7), (1000, 1000, 0.1), (1024, 1000, 0.1), (700, 650, 0.5)]
    for l, m, x in cases:
        col = O.lambda_column(m, L, np.array([x]))
        ref = mp.sqrt((2 * l + 1) / (4 * mp.pi) * mp.factorial(l - m) / mp.factorial(l + m)) \
            * mp.legenp(l, m, x, maxprec=200000)  # legenp includes the Condon-Shortley phase
        ref = float(ref)
        assert abs(col[l - m, 0] - ref) <= 1e-12 * max(abs(ref), 1e-3), (l, m, x)


@pytest.mark.parametrize("m", [0, 1, 64, 511, 900, 1024])
def test_lambda_orthonormal_on_gl_grid_lmax1024(m):
    # 2 pi sum_j w_j lambda_lm lambda_l'm = delta_ll' for n_theta >= l_max + 1
    L = 1024
    x, w = O.gauss_legendre(1537)
    lam = O.lambda_column(m, L, x)
    M = 2.0 * math.pi * (lam * w) @ lam.T
    assert np.max(np.abs(M - np.eye(M.shape[0]))) < 2e-13


def test_addition_theorem_on_grid():
    # lambda_l0^2 + 2 sum_{m>0} lambda_lm^2 = (2l+1)/(4 pi) at every ring
    L = 96
    g = O.Grid(L, 145, 290)
    for l in (0, 1, 17, 96):
        s = g.lam(0)[l] ** 2 + 2.0 * sum(g.lam(m)[l - m] ** 2 for m in range(1, l + 1))
        assert np.max(np.abs(s - (2 * l + 1) / (4 * math.pi))) < 1e-12


# ---------------------------------------------------------------------------
# Spherical harmonic transforms
# ---------------------------------------------------------------------------


@pytest.mark.parametrize("lmax,nt,nph", [(8, 9, 17), (32, 49, 100), (64, 65, 130)])
def test_analysis_of_synthesis_is_identity(lmax, nt, nph):
    g = O.Grid(lmax, nt, nph)
    a = W.random_alm(lmax, 3, seed=lmax)
    b = O.analysis(O.synthesis(a, g), g)
    assert np.max(np.abs(a - b)) < 1e-13 * np.max(np.abs(a)) * 10


def test_synthesis_matches_direct_sum_of_spherical_harmonics():
    sp = pytest.importorskip("scipy.special")
    L, nt, nph = 6, 7, 13
    g = O.Grid(L, nt, nph)
    a = W.random_alm(L, 1, seed=3)[:, 0]
    f = O.synthesis(a, g)[0]
    theta = np.arccos(g.x)[:, None]
    phi = 2 * math.pi * np.arange(nph)[None, :] / nph
    ref = np.zeros((nt, nph))
    for l in range(L + 1):
        for m in range(-l, l + 1):
            alm = a[W.alm_index(l, abs(m), L)]
            if m < 0:
                alm = (-1) ** m * np.conj(alm)
            ref += (alm * sp.sph_harm_y(l, m, theta, phi)).real
    assert np.max(np.abs(f - ref)) < 1e-13


def _gaunt_square(a, L, mu):
    """int (f^2 - mu) Y*_lm dOmega for f = sum a_lm Y_lm, by Gaunt sums (Eq. 22 prefactor)."""
    def A(l, m):
        v = a[W.alm_index(l, abs(m), L)]
        return v if m >= 0 else (-1) ** m * np.conj(v)
    out = np.zeros(W.n_alm(L), dtype=complex)
    for l in range(L + 1):
        for m in range(l + 1):
            s = 0j
            for l1 in range(L + 1):
                for l2 in range(abs(l - l1), min(L, l + l1) + 1):
                    if (l1 + l2 + l) % 2:
                        continue
                    for m1 in range(-l1, l1 + 1):
                        m2 = m - m1
                        if abs(m2) > l2:
                            continue
                        s += A(l1, m1) * A(l2, m2) * (-1) ** m * gaunt(l1, l2, l, m1, m2, -m)
            if l == 0:
                s -= math.sqrt(4 * math.pi) * mu
            out[W.alm_index(l, m, L)] = s
    return out


def _oracle_square(a, L, mu):
    nt, nph = W.grid_for_lmax(L)
    g = O.Grid(L, nt, nph)
    return O.phi_nonlinear(a[:, None], np.array([mu]), g)[:, 0]


@pytest.mark.parametrize("L,seed", [(2, 1), (5, 2), (8, 3)])
def test_square_matches_gaunt_brute_force(L, seed):
    a = W.random_alm(L, 1, seed=seed)[:, 0]
    mu = 0.37
    got = _oracle_square(a, L, mu)
    ref = _gaunt_square(a, L, mu)
    assert np.max(np.abs(got - ref)) < 1e-13 * max(1.0, np.max(np.abs(ref)))


def test_wigner3j_against_sympy_and_orthogonality():
    # sum_{l3, m3} (2 l3 + 1) (l1 l2 l3; m1 m2 m3)^2 = 1
    for l1, l2, m1, m2 in [(3, 4, 1, -2), (5, 5, 0, 0), (7, 2, -3, 1)]:
        s = sum((2 * l3 + 1) * wigner3j(l1, l2, l3, m1, m2, -m1 - m2) ** 2
                for l3 in range(abs(l1 - l2), l1 + l2 + 1))
        assert abs(s - 1.0) < 1e-14
    wig = pytest.importorskip("sympy.physics.wigner")
    for args in [(2, 3, 4, 1, -1, 0), (6, 4, 4, -3, 2, 1), (8, 8, 6, 0, 0, 0), (5, 6, 7, 2, 3, -5)]:
        assert abs(wigner3j(*args) - float(wig.wigner_3j(*args))) < 1e-15


def test_parseval_monopole_identity():
    # Phi_NL,00 = (sum_l [|a_l0|^2 + 2 sum_{m>0} |a_lm|^2] - 4 pi mu) / sqrt(4 pi)
    L = 48
    nt, nph = W.grid_for_lmax(L)
    g = O.Grid(L, nt, nph)
    a = W.random_alm(L, 4, seed=9)
    mu = np.array([0.0, 0.5, 1.3, 2.0])
    out = O.phi_nonlinear(a, mu, g)
    l, m = W.alm_lm(L)
    wgt = np.where(m == 0, 1.0, 2.0)[:, None]
    power = (wgt * np.abs(a) ** 2).sum(axis=0)
    ref = (power - 4 * math.pi * mu) / math.sqrt(4 * math.pi)
    assert np.max(np.abs(out[0] - ref)) < 1e-12 * np.max(np.abs(ref))


def test_parseval_monopole_on_minimal_grids():
    """The monopole of the square equals Parseval's closed form on every grid with
    n_theta >= l_max + 1 and n_phi >= 2 l_max + 2, not only on the exact-square grids: f^2 has
    frequencies up to 2 l_max (none aliased onto m = 0 once n_phi > 2 l_max) and its ring
    means are polynomials of degree <= 2 l_max in cos theta (exact for n_theta >= l_max + 1
    Gauss-Legendre nodes).  On such a grid the other coefficients of the square are aliased
    (they differ from the exact-grid values), and one ring fewer breaks the monopole too."""
    L = 24
    a = W.random_alm(L, 3, seed=19)
    mu = np.array([0.3, 1.1, 0.0])
    l, m = W.alm_lm(L)
    wgt = np.where(m == 0, 1.0, 2.0)[:, None]
    ref = ((wgt * np.abs(a) ** 2).sum(axis=0) - 4 * math.pi * mu) / math.sqrt(4 * math.pi)
    exact = O.phi_nonlinear(a, mu, O.Grid(L, *W.grid_for_lmax(L)))
    for nt, nph in ((L + 1, 2 * L + 2), (L + 5, 54), (30, 60)):
        out = O.phi_nonlinear(a, mu, O.Grid(L, nt, nph))
        assert np.max(np.abs(out[0] - ref)) < 1e-12 * np.max(np.abs(ref)), (nt, nph)
        assert np.max(np.abs(out[1:] - exact[1:])) > 1e-6 * np.max(np.abs(exact[1:])), (nt, nph)
    short = O.phi_nonlinear(a, mu, O.Grid(L, L, 2 * L + 2))
    assert np.max(np.abs(short[0] - ref)) > 1e-8 * np.max(np.abs(ref))


def test_single_monopole_mode():
    L = 16
    nt, nph = W.grid_for_lmax(L)
    g = O.Grid(L, nt, nph)
    a = np.zeros((W.n_alm(L), 1), dtype=complex)
    c, mu = 1.7, 0.05
    a[0, 0] = c
    out = O.phi_nonlinear(a, np.array([mu]), g)[:, 0]
    assert abs(out[0] - (c * c / math.sqrt(4 * math.pi) - math.sqrt(4 * math.pi) * mu)) < 1e-14
    assert np.max(np.abs(out[1:])) < 1e-14


def test_z_rotation_equivariance():
    L = 24
    nt, nph = W.grid_for_lmax(L)
    g = O.Grid(L, nt, nph)
    a = W.random_alm(L, 2, seed=11)
    _, m = W.alm_lm(L)
    psi = 0.7371  # not a grid angle: equivariance holds because the projection is exact
    rot = np.exp(-1j * m * psi)[:, None]
    mu = np.array([0.2, 0.1])
    out = O.phi_nonlinear(a, mu, g)
    out_r = O.phi_nonlinear(a * rot, mu, g)
    assert np.max(np.abs(out_r - out * rot)) < 1e-12 * np.max(np.abs(out))


def test_parity_equivariance():
    L = 24
    nt, nph = W.grid_for_lmax(L)
    g = O.Grid(L, nt, nph)
    a = W.random_alm(L, 2, seed=12)
    l, m = W.alm_lm(L)
    par = ((-1.0) ** (l + m))[:, None]
    mu = np.array([0.2, 0.1])
    out = O.phi_nonlinear(a, mu, g)
    out_p = O.phi_nonlinear(a * par, mu, g)
    assert np.max(np.abs(out_p - out * par)) < 1e-12 * np.max(np.abs(out))


# ---------------------------------------------------------------------------
# Radial statistics
# ---------------------------------------------------------------------------


def test_spherical_jn_matches_scipy():
    sp = pytest.importorskip("scipy.special")
    xs = np.concatenate([np.linspace(1.3, 40, 60), np.linspace(40, 1200, 80), np.linspace(1200, 4500, 40)])
    J = O.spherical_jn_table(1024, xs)
    for l in (0, 1, 2, 7, 50, 333, 800, 1024):
        ref = sp.spherical_jn(l, xs)
        scale = np.maximum(np.abs(ref), 1e-6 * np.max(np.abs(ref)))
        ok = np.abs(ref) > 1e-250
        assert np.max(np.abs(J[l][ok] - ref[ok]) / scale[ok]) < 5e-12, l
        assert np.all(np.abs(J[l][~ok]) < 1e-240)


def test_covariance_matches_scipy_brute_force():
    sp = pytest.importorskip("scipy.special")
    L, nr = 6, 4
    r, _ = W.radial_grid(nr)
    cp = W.COV
    C = O.covariance(L, r, cp.A, cp.ns, cp.kmin, cp.kmax, cp.nk)
    k = np.linspace(cp.kmin, cp.kmax, cp.nk)
    h = k[1] - k[0]
    wk = np.full(cp.nk, h)
    wk[[0, -1]] = h / 2
    for l in range(L + 1):
        J = sp.spherical_jn(l, k[:, None] * r[None, :])
        ref = (2 / math.pi) * np.einsum("k,ki,kj->ij", wk * k ** 2 * cp.A * k ** (cp.ns - 4), J, J)
        assert np.max(np.abs(C[l] - ref)) < 1e-12 * np.max(np.abs(ref))


def test_filters_are_cholesky_factors():
    L, nr = 12, 16
    r, _ = W.radial_grid(nr)
    cp = W.COV
    C = O.covariance(L, r, cp.A, cp.ns, cp.kmin, cp.kmax, cp.nk)
    K = O.filters(C, cp.jitter_rel)
    for l in range(L + 1):
        assert np.allclose(np.triu(K[l], 1), 0.0)
        assert np.all(np.diag(K[l]) > 0)
        eps = cp.jitter_rel * np.mean(np.diag(C[l]))
        assert np.max(np.abs(K[l] @ K[l].T - C[l] - eps * np.eye(nr))) < 1e-12 * np.max(np.abs(C[l]))


def test_mu_is_pixel_variance_of_the_ensemble():
    # mu_i = <Phi_L^2(r_i, n)>: compare with the sample mean of f^2 over pixels and draws
    L, nr, nreal = 12, 3, 96
    K = W.random_lower_filters(L, nr, seed=5, scale=1.0)
    mu = O.mu_ensemble(K)
    nt, nph = W.grid_for_lmax(L)
    g = O.Grid(L, nt, nph)
    acc = np.zeros(nr)
    samples = []
    for s in range(nreal):
        phi = O.phi_linear(K, W.gaussian_noise(L, nr, seed=1000 + s))
        f = O.synthesis(phi, g)
        # area-weighted sky mean of f^2 for each shell
        v = np.einsum("sjk,j->s", f * f, g.w) * (2 * math.pi / nph) / (4 * math.pi)
        samples.append(v)
    samples = np.array(samples)
    mean = samples.mean(axis=0)
    err = samples.std(axis=0, ddof=1) / math.sqrt(nreal)
    assert np.all(np.abs(mean - mu) < 5 * err)


# ---------------------------------------------------------------------------
# Noise generator
# ---------------------------------------------------------------------------


def test_philox_matches_numpy_bit_generator():
    rng = np.random.default_rng(77)
    for _ in range(8):
        ctr = [int(v) for v in rng.integers(0, 2 ** 63, size=4, dtype=np.int64)]
        key = [int(v) for v in rng.integers(0, 2 ** 63, size=2, dtype=np.int64)]
        # numpy's Philox increments its counter before producing each 4-word block
        bg = np.random.Philox(counter=[ctr[0] - 1, ctr[1], ctr[2], ctr[3]], key=key)
        ref = bg.random_raw(4)
        got = O.philox4x64(*[np.uint64(c) for c in ctr], np.uint64(key[0]), np.uint64(key[1]))
        assert [int(v) for v in got] == [int(v) for v in ref]


def test_philox_noise_statistics():
    st = pytest.importorskip("scipy.stats")
    L, nr = 64, 16
    n = O.philox_noise(L, nr, seed=1, realisation=0)
    _, m = W.alm_lm(L)
    m0 = n[:, m == 0]
    mp = n[:, m > 0]
    assert np.all(m0.imag == 0)
    assert st.kstest(m0.real.ravel(), "norm").pvalue > 1e-3
    assert st.kstest(math.sqrt(2) * mp.real.ravel(), "norm").pvalue > 1e-3
    assert st.kstest(math.sqrt(2) * mp.imag.ravel(), "norm").pvalue > 1e-3
    assert abs(np.mean(np.abs(mp) ** 2) - 1.0) < 0.02
    # distinct shells, seeds and realisations draw distinct numbers
    n2 = O.philox_noise(L, nr, seed=1, realisation=1)
    n3 = O.philox_noise(L, nr, seed=2, realisation=0)
    assert abs(np.corrcoef(n.real.ravel(), n2.real.ravel())[0, 1]) < 0.02
    assert abs(np.corrcoef(n.real.ravel(), n3.real.ravel())[0, 1]) < 0.02
    assert abs(np.corrcoef(n[0].real, n[1].real)[0, 1]) < 0.05


# ---------------------------------------------------------------------------
# Whole generator
# ---------------------------------------------------------------------------


def _small_setup(L=12, nr=6, seed=3):
    r, w = W.radial_grid(nr)
    aT, aE = W.transfer_kernels(L, r)
    cp = W.COV
    K = O.filters(O.covariance(L, r, cp.A, cp.ns, cp.kmin, cp.kmax, cp.nk), cp.jitter_rel)
    nt, nph = W.grid_for_lmax(L)
    return r, w, aT, aE, K, O.Grid(L, nt, nph)


def _radial_integral_errors(nr: int = 128, L: int = 7) -> tuple[float, float]:
    """Step (v) against the radial integral a_lm = int dr r^2 Phi_lm(r) alpha_l(r) (Eq. 5 of
    Sect. 2) in closed form, on the workload's midpoint rule over [R_MIN, R_MAX]:
    - Phi_lm(r) = 1 + i and alpha_l(r) = c_l (a different constant per degree): the integral is
      c_l (1 + i) (R_MAX^3 - R_MIN^3) / 3, which the midpoint rule misses by the known amount
      -(R_MAX - R_MIN) h^2 / 12 per unit c_l (the error term of a quadratic);
    - alpha_l(r) = c_l / r^2: the integral c_l (1 + i) (R_MAX - R_MIN), exact for the rule.
    Returns the two largest relative errors over all (l, m)."""
    r, w = W.radial_grid(nr)
    h = (W.R_MAX - W.R_MIN) / nr
    c = 1.0 + 0.37 * np.arange(L + 1)
    l, _ = W.alm_lm(L)
    phi = np.full((W.n_alm(L), nr), 1.0 + 1.0j)
    a1 = O.radial_quadrature(phi, O.quadrature_weights(r, w, c[:, None] * np.ones((1, nr))))
    i1 = c[l] * (1.0 + 1.0j) * ((W.R_MAX ** 3 - W.R_MIN ** 3) / 3.0 - (W.R_MAX - W.R_MIN) * h * h / 12.0)
    a2 = O.radial_quadrature(phi, O.quadrature_weights(r, w, c[:, None] / (r * r)[None, :]))
    i2 = c[l] * (1.0 + 1.0j) * (W.R_MAX - W.R_MIN)
    return float(np.max(np.abs(a1 - i1) / np.abs(i1))), float(np.max(np.abs(a2 - i2) / np.abs(i2)))


def test_radial_quadrature_integrates_the_r2_measure():
    e1, e2 = _radial_integral_errors()
    assert e1 < 1e-13 and e2 < 1e-13


def test_planted_radial_quadrature_mistakes_are_caught(monkeypatch):
    mod = O.fnl_oracle
    orig_q, orig_rq = mod.quadrature_weights, mod.radial_quadrature
    # the r^2 of the measure dropped
    monkeypatch.setattr(mod, "quadrature_weights", lambda r, w, alpha: orig_q(r, w, alpha) / np.asarray(r) ** 2)
    monkeypatch.setattr(O, "quadrature_weights", mod.quadrature_weights)
    assert min(_radial_integral_errors()) > 1e-3
    monkeypatch.undo()
    # the weights of degree l applied to the coefficients of degree l + 1
    monkeypatch.setattr(mod, "radial_quadrature", lambda phi, q: orig_rq(phi, np.roll(q, 1, axis=0)))
    monkeypatch.setattr(O, "radial_quadrature", mod.radial_quadrature)
    assert min(_radial_integral_errors()) > 1e-3
    monkeypatch.undo()


def test_linearity_in_fnl():
    r, w, aT, aE, K, g = _small_setup()
    n = O.philox_noise(12, 6, seed=1, realisation=0)
    a0 = O.generate(K, n, g, r, w, aT, aE, 0.0)
    a1 = O.generate(K, n, g, r, w, aT, aE, 37.5)
    for X in ("T", "E"):
        d = a1["a" + X] - a0["a" + X]
        assert np.max(np.abs(d - 37.5 * a0["aNL" + X])) < 1e-12 * np.max(np.abs(d))


def test_fnl0_power_spectrum_matches_closed_form():
    # Cov(a^X_L,lm, a^Y_L,lm) = q^X_l^T K_l K_l^T q^Y_l (Eq. 5 with Eq. 9); chi^2 over l
    L, nr, nreal = 12, 6, 64
    r, w, aT, aE, K, g = _small_setup(L, nr)
    qT = O.quadrature_weights(r, w, aT)
    qE = O.quadrature_weights(r, w, aE)
    l, m = W.alm_lm(L)
    est = {"TT": np.zeros(L + 1), "EE": np.zeros(L + 1)}
    for s in range(nreal):
        n = O.philox_noise(L, nr, seed=100 + s, realisation=0)
        phiL = O.phi_linear(K, n)
        for X, q in (("T", qT), ("E", qE)):
            a = O.radial_quadrature(phiL, q)
            p = np.abs(a) ** 2 * np.where(m == 0, 1.0, 2.0)
            est[X + X] += np.bincount(l, weights=p, minlength=L + 1) / (2 * l_range(L) + 1)
    chi2, dof = 0.0, 0
    for X, q in (("T", qT), ("E", qE)):
        th = np.einsum("li,lij,lkj,lk->l", q, K, K, q)
        for ll in range(1 if X == "E" else 0, L + 1):
            mean = est[X + X][ll] / nreal
            var = 2 * th[ll] ** 2 / ((2 * ll + 1) * nreal)  # chi^2 with (2l+1) dof per draw
            chi2 += (mean - th[ll]) ** 2 / var
            dof += 1
    assert chi2 < dof + 5 * math.sqrt(2 * dof)


def l_range(L):
    return np.arange(L + 1, dtype=float)


def test_fnl0_linear_part_is_the_filtered_noise_projection():
    # a^X_L = v^X . n with v^X_l = K_l^T q^X_l: the quadrature of Eq. 5 applied to Eq. 9
    r, w, aT, aE, K, g = _small_setup()
    n = O.philox_noise(12, 6, seed=5, realisation=2)
    out = O.generate(K, n, g, r, w, aT, aE, 0.0)
    q = O.quadrature_weights(r, w, aT)
    l, m = W.alm_lm(12)
    nn = n.copy()
    nn[:, m == 0] = nn[:, m == 0].real
    v = np.einsum("lij,li->lj", K, q)
    ref = np.einsum("ij,ji->i", v[l], nn)
    assert np.max(np.abs(out["aLT"] - ref)) < 1e-13 * np.max(np.abs(ref))


def test_planted_filter_mistakes_are_caught(monkeypatch):
    """Step (i) with K_l transposed (Phi_L(r_i) = sum_j K_l[j, i] n(r_j)), or with the noise
    of degree l filtered by K of degree l + 1, fails the f_NL = 0 projection pin above."""
    def projection_pin_fails():
        try:
            test_fnl0_linear_part_is_the_filtered_noise_projection()
        except AssertionError:
            return True
        return False

    assert not projection_pin_fails()
    mod = O.fnl_oracle
    orig = mod.phi_linear
    monkeypatch.setattr(mod, "phi_linear", lambda K, n: orig(np.transpose(K, (0, 2, 1)), n))
    assert projection_pin_fails()
    monkeypatch.undo()
    monkeypatch.setattr(mod, "phi_linear", lambda K, n: orig(np.roll(K, 1, axis=0), n))
    assert projection_pin_fails()
    monkeypatch.undo()


@pytest.mark.parametrize("parts", [[(0, 6)], [(0, 3), (3, 6)], [(0, 1), (1, 4), (4, 5), (5, 6)]])
def test_shell_shards_sum_to_the_whole_recipe(parts):
    # Eq. 5 and Eq. 3 sum per-shell terms: shards partitioning the shells add up to the recipe
    r, w, aT, aE, K, g = _small_setup()
    n = O.philox_noise(12, 6, seed=7, realisation=1)
    whole = O.generate(K, n, g, r, w, aT, aE, 25.0)
    acc = {k: 0.0 for k in ("aT", "aE", "aLT", "aLE", "aNLT", "aNLE")}
    for j0, j1 in parts:
        sh = O.generate_shard(K, n, g, r, w, aT, aE, 25.0, j0, j1)
        assert sh["phiL"].shape[1] == j1 - j0
        for k in acc:
            acc[k] = acc[k] + sh[k]
    for k in acc:
        assert np.max(np.abs(acc[k] - whole[k])) < 1e-12 * np.max(np.abs(whole[k])), k
    # the per-shell fields of a shard are the whole recipe's columns
    sh = O.generate_shard(K, n, g, r, w, aT, aE, 25.0, 2, 5)
    assert np.max(np.abs(sh["phiNL"] - whole["phiNL"][:, 2:5])) < 1e-12 * np.max(np.abs(whole["phiNL"]))


def test_shard_reads_the_noise_of_its_rows_only():
    # rows j0 .. j1 - 1 of the lower-triangular K_l reach the noise of shells < j1: a shard's
    # output does not change when the noise of later shells does, and its a^X_L is v' . n with
    # v'_l = K_l[j0:j1]^T q_l[j0:j1], written out here
    r, w, aT, aE, K, g = _small_setup()
    n = O.philox_noise(12, 6, seed=9, realisation=0)
    j0, j1 = 2, 4
    a = O.generate_shard(K, n, g, r, w, aT, aE, 10.0, j0, j1)
    n2 = n.copy()
    n2[j1:] = 1e3 * (1 + 1j)
    b = O.generate_shard(K, n2, g, r, w, aT, aE, 10.0, j0, j1)
    for k in ("aT", "aE", "aLT", "aNLE"):
        assert np.array_equal(a[k], b[k]), k
    q = O.quadrature_weights(r, w, aE)
    l, m = W.alm_lm(12)
    nn = n.copy()
    nn[:, m == 0] = nn[:, m == 0].real
    v = np.einsum("lij,li->lj", K[:, j0:j1, :], q[:, j0:j1])
    ref = np.einsum("ij,ji->i", v[l], nn)
    assert np.max(np.abs(a["aLE"] - ref)) < 1e-13 * np.max(np.abs(ref))


# ---------------------------------------------------------------------------
# Planted mistakes: each must be caught by a pin above
# ---------------------------------------------------------------------------


def test_planted_mistakes_are_caught(monkeypatch):
    L = 5
    a = W.random_alm(L, 1, seed=21)[:, 0]
    mu = 0.2
    ref = _gaunt_square(a, L, mu)

    def gaunt_pin_fails():
        got = _oracle_square(a, L, mu)
        return np.max(np.abs(got - ref)) > 1e-8

    def identity_pin_fails():
        g = O.Grid(8, 9, 17)
        aa = W.random_alm(8, 1, seed=2)
        return np.max(np.abs(O.analysis(O.synthesis(aa, g), g) - aa)) > 1e-8

    def direct_sum_pin_fails():
        try:
            test_synthesis_matches_direct_sum_of_spherical_harmonics()
        except AssertionError:
            return True
        return False

    assert not gaunt_pin_fails() and not identity_pin_fails() and not direct_sum_pin_fails()
    mod = O.fnl_oracle

    # 1. Condon-Shortley phase dropped from lambda_lm.  The squared-field projection cannot
    # see it (the phase is a rotation by pi about z, and squaring commutes with rotations),
    # so it is the map-level pin that must catch it.
    orig_col = mod.lambda_column
    monkeypatch.setattr(mod, "lambda_column", lambda m, lmax, x, mm=None: orig_col(m, lmax, x, mm) * (-1) ** m)
    assert direct_sum_pin_fails() and not gaunt_pin_fails()
    monkeypatch.undo()

    # 2. <Phi_L^2> added instead of subtracted (Eq. 2)
    orig_nl = O.phi_nonlinear
    monkeypatch.setattr(O, "phi_nonlinear", lambda p, mu_, g: orig_nl(p, -np.asarray(mu_), g))
    assert gaunt_pin_fails()
    monkeypatch.undo()

    # 3. GL weights replaced by equal weights in the analysis
    orig_gl = mod.gauss_legendre
    monkeypatch.setattr(mod, "gauss_legendre", lambda n: (orig_gl(n)[0], np.full(n, 2.0 / n)))
    assert gaunt_pin_fails() and identity_pin_fails()
    monkeypatch.undo()

    # 4. the factor 2 of the m > 0 terms dropped from the synthesis
    def half_syn(alm, grid):
        alm = np.asarray(alm).reshape(np.asarray(alm).shape[0], -1)
        a0 = np.zeros_like(alm)
        a0[: grid.lmax + 1] = alm[: grid.lmax + 1]
        return 0.5 * (orig_syn(alm, grid) + orig_syn(a0, grid))
    orig_syn = O.synthesis
    monkeypatch.setattr(O, "synthesis", half_syn)
    monkeypatch.setattr(mod, "synthesis", half_syn)
    assert gaunt_pin_fails() and identity_pin_fails()
    monkeypatch.undo()

    # 5. wrong sign of the phase in the forward DFT of the analysis
    orig_rfft = np.fft.rfft
    monkeypatch.setattr(mod.np.fft, "rfft", lambda x, axis=-1: np.conj(orig_rfft(x, axis=axis)))
    assert identity_pin_fails()
    monkeypatch.undo()


# ---------------------------------------------------------------------------
# Adjoint (differentiation form): transposes by the dot-product test against the pinned
# forward maps, and the whole gradient by central finite differences
# ---------------------------------------------------------------------------

def _rdot(u, v):
    return float(np.sum((np.conj(np.asarray(u)) * np.asarray(v)).real))


def _random_alm(L, nsh, rng, real_m0=False):
    a = rng.standard_normal((W.n_alm(L), nsh)) + 1j * rng.standard_normal((W.n_alm(L), nsh))
    if real_m0:
        a[: L + 1] = a[: L + 1].real
    return a


@pytest.mark.parametrize("L,nt,nph", [(6, 10, 19), (9, 14, 30)])
def test_transform_adjoints_pass_the_dot_product_test(L, nt, nph):
    rng = np.random.default_rng(11)
    grid = O.Grid(L, nt, nph)
    a = _random_alm(L, 3, rng)            # the imaginary part of m = 0 is ignored by synthesis
    F = rng.standard_normal((3, nt, nph))
    assert _rdot(O.synthesis(a, grid), F) == pytest.approx(_rdot(a, O.synthesis_adjoint(F, grid)), rel=1e-12)
    B = _random_alm(L, 3, rng)
    assert _rdot(O.analysis(F, grid), B) == pytest.approx(_rdot(F, O.analysis_adjoint(B, grid)), rel=1e-12)


def test_filter_and_quadrature_adjoints_pass_the_dot_product_test():
    rng = np.random.default_rng(12)
    L, nr = 7, 5
    K = W.random_lower_filters(L, nr, seed=2, scale=1.0)
    n = _random_alm(L, nr, rng).T
    P = _random_alm(L, nr, rng)
    assert _rdot(O.phi_linear(K, n), P) == pytest.approx(_rdot(n, O.phi_linear_adjoint(K, P)), rel=1e-12)
    q = rng.standard_normal((L + 1, nr))
    A = _random_alm(L, 1, rng)[:, 0]
    assert _rdot(O.radial_quadrature(P, q), A) == pytest.approx(
        _rdot(P, O.radial_quadrature_adjoint(A, q)), rel=1e-12)


def _loss_and_grad(out, dT, dE, wT, wE):
    """L = sum_idx wX |a^X - d^X|^2 and its pair gradients gX = 2 wX (a^X - d^X)."""
    rT, rE = out["aT"] - dT, out["aE"] - dE
    L = float(np.sum(wT * np.abs(rT) ** 2) + np.sum(wE * np.abs(rE) ** 2))
    return L, 2 * wT * rT, 2 * wE * rE


def test_generate_backward_matches_central_differences():
    L, nr = 8, 5
    nt, nph = W.grid_for_lmax(L)
    grid = O.Grid(L, nt, nph)
    r, w = W.radial_grid(nr)
    aT, aE = W.transfer_kernels(L, r)
    K = W.random_lower_filters(L, nr, seed=4, scale=0.3)
    mu = O.mu_ensemble(K)
    rng = np.random.default_rng(13)
    noise = _random_alm(L, nr, rng, real_m0=True).T
    d = O.generate(K, _random_alm(L, nr, rng, real_m0=True).T, grid, r, w, aT, aE, 20.0, mu=mu)
    wT = rng.uniform(0.5, 2.0, W.n_alm(L))
    wE = rng.uniform(0.5, 2.0, W.n_alm(L))
    fnl = 35.0
    loss = lambda n, f: _loss_and_grad(O.generate(K, n, grid, r, w, aT, aE, f, mu=mu), d["aT"], d["aE"], wT, wE)[0]
    _, gT, gE = _loss_and_grad(O.generate(K, noise, grid, r, w, aT, aE, fnl, mu=mu), d["aT"], d["aE"], wT, wE)
    gn, gf = O.generate_backward(K, noise, grid, r, w, aT, aE, fnl, gT, gE, mu=mu)
    eps = 1e-6
    for k in range(6):
        v = _random_alm(L, nr, rng, real_m0=True).T
        fd = (loss(noise + eps * v, fnl) - loss(noise - eps * v, fnl)) / (2 * eps)
        assert _rdot(gn, v) == pytest.approx(fd, rel=1e-7, abs=1e-9 * abs(fd))
    fd = (loss(noise, fnl + eps) - loss(noise, fnl - eps)) / (2 * eps)
    assert gf == pytest.approx(fd, rel=1e-7)
    assert np.all(gn[:, : L + 1].imag == 0.0)


def test_planted_adjoint_mistakes_fail_central_differences():
    """Dropping the m > 0 doubling of the synthesis transpose, or the linear branch, changes
    the gradient by far more than the finite-difference tolerance."""
    L, nr = 6, 4
    nt, nph = W.grid_for_lmax(L)
    grid = O.Grid(L, nt, nph)
    r, w = W.radial_grid(nr)
    aT, aE = W.transfer_kernels(L, r)
    K = W.random_lower_filters(L, nr, seed=5, scale=0.3)
    rng = np.random.default_rng(14)
    noise = _random_alm(L, nr, rng, real_m0=True).T
    gT = _random_alm(L, 1, rng)[:, 0]
    gE = _random_alm(L, 1, rng)[:, 0]
    good, _ = O.generate_backward(K, noise, grid, r, w, aT, aE, 25.0, gT, gE)
    qT = O.quadrature_weights(r, w, aT)
    qE = O.quadrature_weights(r, w, aE)
    fw = O.generate(K, noise, grid, r, w, aT, aE, 25.0)
    lin = O.radial_quadrature_adjoint(gT, qT) + O.radial_quadrature_adjoint(gE, qE)
    gbar = O.analysis_adjoint(25.0 * lin, grid)
    f = O.synthesis(fw["phiL"], grid)
    no_lin = O.phi_linear_adjoint(K, O.synthesis_adjoint(2.0 * f * gbar, grid))
    undoubled = O.phi_linear_adjoint(K, O.synthesis_adjoint(2.0 * f * gbar, grid) * 0.5 + lin)
    for bad in (no_lin, undoubled):
        assert np.linalg.norm(bad - good) > 1e-3 * np.linalg.norm(good)


# ---------------------------------------------------------------------------
# Output maps: spin-2 functions and the Stokes I, Q, U synthesis
# ---------------------------------------------------------------------------

def _edth_numeric(f, s, m, h=1e-4):
    """The spin raising operator on eta(theta) e^{i m phi} of spin weight s, by central
    differences in theta: edth eta = -(sin th)^s (d_th - m / sin th)[(sin th)^(-s) eta]."""
    def g(th):
        u = lambda t: np.sin(t) ** (-s) * f(t)
        d = (u(th + h) - u(th - h)) / (2 * h)
        return -np.sin(th) ** s * (d - m / np.sin(th) * u(th))
    return g


def _edthbar_numeric(f, s, m, h=1e-4):
    """The spin lowering operator: edthbar eta = -(sin th)^(-s) (d_th + m / sin th)[(sin th)^s eta]."""
    def g(th):
        u = lambda t: np.sin(t) ** s * f(t)
        d = (u(th + h) - u(th - h)) / (2 * h)
        return -np.sin(th) ** (-s) * (d + m / np.sin(th) * u(th))
    return g


def test_spin2_functions_follow_the_spin_operators():
    """W +- X = +-2lam against N_l edth^2 Y and N_l edthbar^2 Y evaluated by finite differences
    of scipy's Y_lm: pins the closed forms (signs, c_lm, the 1 / sin^2 terms) to the definition."""
    sp = pytest.importorskip("scipy.special")
    L = 7
    g = O.Grid(L, 9, 16)
    th = np.arccos(g.x)
    for m in range(L + 1):
        W, X = O.spin2_functions(m, g)
        for l in range(max(m, 2), L + 1):
            y = lambda t, l=l, m=m: sp.sph_harm_y(l, m, t, 0.0).real
            nl = 1.0 / math.sqrt((l - 1) * l * (l + 1) * (l + 2))
            p2 = nl * _edth_numeric(_edth_numeric(y, 0, m), 1, m)(th)
            m2 = nl * _edthbar_numeric(_edthbar_numeric(y, 0, m), -1, m)(th)
            scale = max(np.max(np.abs(p2)), np.max(np.abs(m2)), 1e-3)
            assert np.max(np.abs(W[l - m] + X[l - m] - p2)) < 2e-6 * scale, (l, m)
            assert np.max(np.abs(W[l - m] - X[l - m] - m2)) < 2e-6 * scale, (l, m)
        assert np.all(W[: max(0, 2 - m)] == 0) and np.all(X[: max(0, 2 - m)] == 0)


def test_spin2_y20_closed_form():
    """2Y_20 = -2Y_20 = (1/4) sqrt(15 / (2 pi)) sin^2 theta (tabulated closed form)."""
    g = O.Grid(4, 7, 13)
    W, X = O.spin2_functions(0, g)
    ref = 0.25 * math.sqrt(15 / (2 * math.pi)) * (1 - g.x ** 2)
    assert np.max(np.abs(W[2] - ref)) < 1e-15 and np.max(np.abs(X[2])) == 0.0


@pytest.mark.parametrize("m", [0, 1, 2, 5, 31])
def test_spin2_functions_orthonormal_on_gl_grid(m):
    """sum_j w_j 2 pi (+-2lam_l)(+-2lam_l') = delta_ll' for l, l' >= 2 (exact GL quadrature)."""
    L = 40
    g = O.Grid(L, L + 2, 2 * L + 2)
    W, X = O.spin2_functions(m, g)
    lo = max(0, 2 - m)
    for F in (W + X, W - X):
        F = F[lo:]
        gram = 2 * math.pi * (F * g.w) @ F.T
        assert np.max(np.abs(gram - np.eye(F.shape[0]))) < 1e-12


def _random_eb(L, seed):
    rng = np.random.default_rng(seed)
    na = W.n_alm(L)
    out = []
    for _ in range(3):
        a = rng.standard_normal(na) + 1j * rng.standard_normal(na)
        a[: L + 1] = a[: L + 1].real
        out.append(a)
    ls, _ = W.alm_lm(L)
    out[1][ls < 2] = 0.0  # E and B start at l = 2
    out[2][ls < 2] = 0.0
    return out


@pytest.mark.parametrize("L,nt,nph", [(8, 13, 25), (24, 37, 75), (40, 41, 90)])
def test_spin2_analysis_of_synthesis_is_identity(L, nt, nph):
    aT, aE, aB = _random_eb(L, 5 + L)
    g = O.Grid(L, nt, nph)
    I, Q, U = O.maps_iqu(aT, aE, aB, g)
    e, b = O.analysis_spin2(Q, U, g)
    assert np.max(np.abs(e - aE)) < 1e-12 * np.max(np.abs(aE))
    assert np.max(np.abs(b - aB)) < 1e-12 * np.max(np.abs(aB))
    assert np.max(np.abs(I - O.synthesis(aT[:, None], g)[0])) == 0.0


def test_spin2_parseval_and_eb_rotation():
    """int (Q^2 + U^2) dOmega = sum over all m of |E|^2 + |B|^2 (from |a_{+-2}|^2), and the
    exchange E -> -B, B -> E turns (Q, U) into (-U, Q) (a 45-degree rotation of the frame)."""
    L = 24
    aT, aE, aB = _random_eb(L, 2)
    g = O.Grid(L, 40, 80)
    I, Q, U = O.maps_iqu(aT, aE, aB, g)
    integral = 2 * math.pi / g.nphi * np.sum(g.w[:, None] * (Q ** 2 + U ** 2))
    _, ms = W.alm_lm(L)
    wm = np.where(ms == 0, 1.0, 2.0)
    assert abs(integral - np.sum(wm * (np.abs(aE) ** 2 + np.abs(aB) ** 2))) < 1e-11 * integral
    I2, Q2, U2 = O.maps_iqu(aT, -aB, aE, g)
    assert np.max(np.abs(Q2 + U)) < 1e-12 * np.max(np.abs(U)) and np.max(np.abs(U2 - Q)) < 1e-12 * np.max(np.abs(Q))


def test_pure_e_monopole_like_mode_has_no_u():
    """a^E_20 = 1 alone: Q = -(1/4) sqrt(15 / (2 pi)) sin^2 theta on every ring and U = 0."""
    L = 6
    g = O.Grid(L, 10, 19)
    aE = np.zeros(W.n_alm(L), complex)
    aE[W.alm_index(2, 0, L)] = 1.0
    I, Q, U = O.maps_iqu(np.zeros_like(aE), aE, None, g)
    ref = -0.25 * math.sqrt(15 / (2 * math.pi)) * (1 - g.x ** 2)
    assert np.max(np.abs(Q - ref[:, None])) < 1e-15 and np.max(np.abs(U)) < 1e-15 and np.max(np.abs(I)) == 0


def test_planted_spin2_mistakes_are_caught():
    """A flipped X, a dropped lam_{l-1} term or a swapped E/B convention in the maps each fail
    the pins above (checked here on the CPU by recomputing them with the mistake planted)."""
    sp = pytest.importorskip("scipy.special")
    g = O.Grid(6, 8, 15)
    th = np.arccos(g.x)
    good = O.spin2_functions

    def flipped_x(m, grid):
        Wm, Xm = good(m, grid)
        return Wm, -Xm

    def dropped_prev(m, grid):
        Wm, Xm = good(m, grid)
        lam = grid.lam(m)
        ls = np.arange(m, grid.lmax + 1, dtype=float)[:, None]
        nl = np.where(ls >= 2, 1 / np.sqrt(np.maximum((ls - 1) * ls * (ls + 1) * (ls + 2), 1)), 0)
        s2 = 1 - grid.x ** 2
        return nl * ((2.0 * m * m - 2 * ls * grid.x ** 2) * lam / s2 - ls * (ls + 1) * lam), Xm

    def edth_error(fn):
        err = 0.0
        for m in range(1, 4):
            Wm, Xm = fn(m, g)
            for l in range(max(m, 2), 7):
                y = lambda t, l=l, m=m: sp.sph_harm_y(l, m, t, 0.0).real
                nl = 1.0 / math.sqrt((l - 1) * l * (l + 1) * (l + 2))
                p2 = nl * _edth_numeric(_edth_numeric(y, 0, m), 1, m)(th)
                err = max(err, np.max(np.abs(Wm[l - m] + Xm[l - m] - p2)))
        return err

    assert edth_error(good) < 1e-6
    assert edth_error(flipped_x) > 1e-3
    assert edth_error(dropped_prev) > 1e-3
    # swapping the E/B convention (Q + iU = +sum (E + iB) 2Y) breaks the closed form of 2Y_20's Q
    aE = np.zeros(W.n_alm(6), complex)
    aE[W.alm_index(2, 0, 6)] = 1.0
    Q = O.maps_iqu(np.zeros_like(aE), -aE, None, g)[1]
    assert np.max(np.abs(Q + 0.25 * math.sqrt(15 / (2 * math.pi)) * (1 - g.x ** 2)[:, None])) > 1e-2
