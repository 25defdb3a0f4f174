"""Plain FP64 CPU oracle of the HEALPix ring grid variant (test infrastructure).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``.  It shares no code with the CUDA library.

The paper's maps live on HEALPix (Sect. 3: n_side = 512 at l_max = 1024).  HEALPix (Gorski et al.
2005) tiles the sphere with N_pix = 12 n_side^2 equal-area pixels whose centres lie on 4 n_side - 1
rings of constant z = cos(theta), ring i = 1 .. 4 n_side - 1 from the north pole:

  north cap,  i < n_side:            z = 1 - i^2 / (3 n_side^2),   n_i = 4 i,        phi_0 = pi / (4 i)
  belt, n_side <= i <= 3 n_side:     z = 4/3 - 2 i / (3 n_side),   n_i = 4 n_side,   phi_0 = s pi / (4 n_side),
                                     s = (i - n_side + 1) mod 2
  south cap,  i > 3 n_side:          the mirror of ring 4 n_side - i (z -> -z, same n_i and phi_0)

with pixel k of ring i at phi = phi_0 + 2 pi k / n_i.  Integrals over the sphere are approximated
by the equal-weight rule int f dOmega ~ (4 pi / N_pix) sum_pixels f, so the transforms are:

  synthesis: f(z_i, phi_ik) = sum_{l, |m| <= l} a_lm lambda_lm(z_i) e^{i m phi_ik}
             (F_m = sum_l lambda_lm a_lm on each ring; m > n_i / 2 aliases on the short rings)
  analysis:  a_lm = (4 pi / N_pix) sum_i lambda_lm(z_i) sum_k f_ik e^{-i m phi_ik}

and steps (ii)-(iv) of the generator on this grid are Phi_NL = analysis((synthesis Phi_L)^2 - mu).
Unlike the Gauss-Legendre grid the rule is not exact; the analysis of a synthesis returns a_lm
up to an error that falls with n_side.

Pins (tests/test_healpix_pins.py, CPU): ring geometry against the published pixel centres of
n_side = 1 and 2 and the counting identities (N_pix = 12 n_side^2, 4 n_side - 1 rings, z
antisymmetric, ring sizes and offsets mirrored); synthesis at every pixel against a direct sum of
scipy's Y_lm at the pixel centre; analysis against a direct pixel sum with scipy's Y_lm; the
monopole integrated exactly; the round trip error falling with n_side.
"""
from __future__ import annotations

import math

import numpy as np

from workloads import alm_index

from .fnl_oracle import lambda_column, lambda_mm


class HealpixGrid:
    """Rings of a HEALPix grid (RING order) with lambda_lm at the ring z values."""

    def __init__(self, lmax: int, nside: int):
        self.lmax, self.nside = lmax, nside
        nr = 4 * nside - 1
        z = np.empty(nr)
        n = np.empty(nr, dtype=int)
        phi0 = np.empty(nr)
        for idx in range(nr):
            i = idx + 1
            ii = i if i <= 2 * nside else 4 * nside - i     # mirror index for the south
            if ii < nside:
                zz, nn, p0 = 1.0 - ii * ii / (3.0 * nside * nside), 4 * ii, math.pi / (4 * ii)
            else:
                s = (ii - nside + 1) % 2
                zz, nn, p0 = 4.0 / 3.0 - 2.0 * ii / (3.0 * nside), 4 * nside, s * math.pi / (4 * nside)
            z[idx] = zz if i <= 2 * nside else -zz
            n[idx], phi0[idx] = nn, p0
        self.z, self.n, self.phi0 = z, n, phi0
        self.offset = np.concatenate([[0], np.cumsum(n)])
        self.npix = int(self.offset[-1])
        self.weight = 4.0 * math.pi / self.npix
        self._mm = lambda_mm(lmax, z)

    def lam(self, m: int) -> np.ndarray:
        """lambda_lm(z_i), l = m..lmax, shape [lmax - m + 1, n_rings]."""
        return lambda_column(m, self.lmax, self.z, self._mm)

    def pixel_angles(self):
        theta = np.repeat(np.arccos(self.z), self.n)
        phi = np.concatenate([p0 + 2.0 * math.pi * np.arange(nn) / nn for p0, nn in zip(self.phi0, self.n)])
        return theta, phi


def healpix_synthesis(alm: np.ndarray, grid: HealpixGrid) -> np.ndarray:
    """Real fields on the pixels (RING order), [nsh, N_pix]; alm [nalm, nsh] (m = 0 real part)."""
    L = grid.lmax
    alm = np.asarray(alm, dtype=np.complex128)
    if alm.ndim == 1:
        alm = alm[:, None]
    nsh, nring = alm.shape[1], grid.z.size
    F = np.zeros((nsh, nring, L + 1), dtype=np.complex128)   # F_m(z_i)
    for m in range(L + 1):
        rows = alm_index(np.arange(m, L + 1), m, L)
        F[:, :, m] = (grid.lam(m).T @ alm[rows, :]).T
    F[:, :, 0] = F[:, :, 0].real
    out = np.zeros((nsh, grid.npix))
    ms = np.arange(1, L + 1)
    for i in range(nring):
        phi = grid.phi0[i] + 2.0 * math.pi * np.arange(grid.n[i]) / grid.n[i]
        e = np.exp(1j * np.outer(phi, ms))                     # [n_i, L]
        ring = F[:, i, 0].real[:, None] + 2.0 * np.real(F[:, i, 1:] @ e.T)
        out[:, grid.offset[i]:grid.offset[i + 1]] = ring
    return out


def healpix_analysis(maps: np.ndarray, grid: HealpixGrid) -> np.ndarray:
    """a_lm = (4 pi / N_pix) sum_pixels f lambda_lm(z) e^{-i m phi}, [nalm, nsh]."""
    L = grid.lmax
    maps = np.atleast_2d(np.asarray(maps, dtype=np.float64))
    nsh, nring = maps.shape[0], grid.z.size
    G = np.zeros((nsh, nring, L + 1), dtype=np.complex128)
    ms = np.arange(L + 1)
    for i in range(nring):
        phi = grid.phi0[i] + 2.0 * math.pi * np.arange(grid.n[i]) / grid.n[i]
        e = np.exp(-1j * np.outer(ms, phi))                    # [L+1, n_i]
        G[:, i, :] = maps[:, grid.offset[i]:grid.offset[i + 1]] @ e.T
    out = np.zeros((alm_index(L, L, L) + 1, nsh), dtype=np.complex128)
    for m in range(L + 1):
        rows = alm_index(np.arange(m, L + 1), m, L)
        out[rows, :] = grid.weight * (grid.lam(m) @ G[:, :, m].T)
    return out


def healpix_nonlinear(phi_L: np.ndarray, mu: np.ndarray, grid: HealpixGrid) -> np.ndarray:
    """Steps (ii)-(iv) on the HEALPix grid: analysis((synthesis Phi_L)^2 - mu), [nalm, nsh]."""
    f = healpix_synthesis(phi_L, grid)
    return healpix_analysis(f * f - np.asarray(mu, dtype=np.float64)[:, None], grid)


def healpix_generate(K, noise, grid: HealpixGrid, r, w, alphaT, alphaE, fnl: float, mu=None) -> dict:
    """The recipe of ``generate`` with steps (ii)-(iv) on the HEALPix grid."""
    from .fnl_oracle import mu_ensemble, phi_linear, quadrature_weights, radial_quadrature
    phiL = phi_linear(K, noise)
    if mu is None:
        mu = mu_ensemble(K)
    qT = quadrature_weights(r, w, alphaT)
    qE = quadrature_weights(r, w, alphaE)
    phiNL = healpix_nonlinear(phiL, mu, grid)
    out = {"aLT": radial_quadrature(phiL, qT), "aLE": radial_quadrature(phiL, qE),
           "aNLT": radial_quadrature(phiNL, qT), "aNLE": radial_quadrature(phiNL, qE)}
    out["aT"] = out["aLT"] + fnl * out["aNLT"]
    out["aE"] = out["aLE"] + fnl * out["aNLE"]
    return out


__all__ = ["HealpixGrid", "healpix_synthesis", "healpix_analysis", "healpix_nonlinear", "healpix_generate"]
