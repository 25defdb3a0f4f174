"""Pins of the HEALPix oracle (oracle/healpix_oracle.py) to facts other than itself (CPU).

- Ring geometry against the published pixel centres of n_side = 1 and 2, and the counting
  identities N_pix = 12 n_side^2, sum of ring sizes, z antisymmetry, phi offsets mirrored.
- Synthesis at every pixel against the direct sum of scipy's Y_lm at the pixel centre.
- Analysis against the direct pixel sum (4 pi / N_pix) sum f conj(Y_lm) with scipy's Y_lm.
- The monopole is integrated exactly; the round trip error falls as n_side grows.
- A whole realisation converges, as n_side grows, to the same realisation on a Gauss-Legendre
  grid that evaluates the square exactly (itself pinned by Gaunt brute force); its linear part
  does not depend on the grid.
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W


def test_ring_geometry_small_nsides():
    g = O.HealpixGrid(2, 1)
    assert np.allclose(g.z, [2 / 3, 0, -2 / 3]) and list(g.n) == [4, 4, 4]
    assert np.allclose(g.phi0, [math.pi / 4, 0, math.pi / 4]) and g.npix == 12
    g = O.HealpixGrid(4, 2)
    assert np.allclose(g.z, [11 / 12, 2 / 3, 1 / 3, 0, -1 / 3, -2 / 3, -11 / 12])
    assert list(g.n) == [4, 8, 8, 8, 8, 8, 4] and g.npix == 48
    assert np.allclose(g.phi0, [math.pi / 4, math.pi / 8, 0, math.pi / 8, 0, math.pi / 8, math.pi / 4])
    for ns in (4, 16, 64):
        g = O.HealpixGrid(2, ns)
        assert g.npix == 12 * ns * ns and g.z.size == 4 * ns - 1
        assert np.allclose(g.z, -g.z[::-1]) and np.array_equal(g.n, g.n[::-1])
        assert np.allclose(g.phi0, g.phi0[::-1])


def _ylm_direct(L, theta, phi):
    sp = pytest.importorskip("scipy.special")
    Y = {}
    for l in range(L + 1):
        for m in range(l + 1):
            Y[(l, m)] = sp.sph_harm_y(l, m, theta, phi)
    return Y


def test_synthesis_and_analysis_against_direct_sums():
    L, ns = 6, 4
    g = O.HealpixGrid(L, ns)
    th, ph = g.pixel_angles()
    Y = _ylm_direct(L, th, ph)
    a = W.random_alm(L, 1, seed=3)[:, 0]
    f = O.healpix_synthesis(a, g)[0]
    ref = np.zeros(g.npix)
    for (l, m), y in Y.items():
        c = a[W.alm_index(l, m, L)]
        ref += (c.real * y.real) if m == 0 else 2.0 * np.real(c * y)
    assert np.max(np.abs(f - ref)) < 1e-12 * np.max(np.abs(ref))
    rng = np.random.default_rng(2)
    maps = rng.standard_normal(g.npix)
    got = O.healpix_analysis(maps, g)[:, 0]
    for (l, m), y in Y.items():
        direct = 4 * math.pi / g.npix * np.sum(maps * np.conj(y))
        assert abs(got[W.alm_index(l, m, L)] - direct) < 1e-12 * max(1.0, abs(direct))


def test_monopole_exact_and_round_trip_converges():
    L = 8
    g = O.HealpixGrid(L, 4)
    a00 = O.healpix_analysis(np.ones(g.npix), g)[0, 0]
    assert abs(a00 - math.sqrt(4 * math.pi)) < 1e-13
    a = W.random_alm(L, 1, seed=5)[:, 0]
    errs = []
    for ns in (4, 8, 16, 32):
        g = O.HealpixGrid(L, ns)
        back = O.healpix_analysis(O.healpix_synthesis(a, g), g)[:, 0]
        errs.append(np.linalg.norm(back - a) / np.linalg.norm(a))
    assert all(e2 < e1 for e1, e2 in zip(errs, errs[1:])) and errs[-1] < 1e-2


def _healpix_generate_errors(nsides=(4, 8, 16, 32)):
    L, nr = 6, 4
    r, w = W.radial_grid(nr)
    aT, aE = W.transfer_kernels(L, r)
    cp = W.COV
    K = O.filters(O.covariance(L, r, cp.A, cp.ns, cp.kmin, cp.kmax, cp.nk), cp.jitter_rel)
    n = O.philox_noise(L, nr, seed=7, realisation=1)
    nt, nph = W.grid_for_lmax(L)
    ref = O.generate(K, n, O.Grid(L, nt, nph), r, w, aT, aE, 25.0)
    lin, nl = [], []
    for ns in nsides:
        got = O.healpix_generate(K, n, O.HealpixGrid(L, ns), r, w, aT, aE, 25.0)
        lin.append(max(np.max(np.abs(got[k] - ref[k])) / np.max(np.abs(ref[k])) for k in ("aLT", "aLE")))
        nl.append(max(np.linalg.norm(got[k] - ref[k]) / np.linalg.norm(ref[k]) for k in ("aNLT", "aNLE")))
    return lin, nl


def test_generate_converges_to_the_exact_gauss_legendre_realisation():
    lin, nl = _healpix_generate_errors()
    assert max(lin) < 1e-13
    # the pixel quadrature's error falls as n_side^-2 (measured 0.032, 0.0064, 0.0015, 0.00038)
    assert all(e2 < e1 / 3 for e1, e2 in zip(nl, nl[1:])) and nl[-1] < 1e-3


def test_planted_healpix_mistakes_are_caught(monkeypatch):
    import oracle.healpix_oracle as H
    orig_nl = H.healpix_nonlinear
    # <Phi_L^2> added instead of subtracted (Eq. 2)
    monkeypatch.setattr(H, "healpix_nonlinear", lambda p, mu, g: orig_nl(p, -np.asarray(mu), g))
    _, nl = _healpix_generate_errors((8, 16))
    assert nl[-1] > 1e-2
    monkeypatch.undo()
    # the equal-area pixel weight 4 pi / N_pix dropped from the analysis
    orig_an = H.healpix_analysis
    monkeypatch.setattr(H, "healpix_analysis", lambda maps, g: orig_an(maps, g) * g.npix / (4 * math.pi))
    _, nl = _healpix_generate_errors((8, 16))
    assert nl[-1] > 1e-2
    monkeypatch.undo()
