"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds no arithmetic of the f_NL method itself: no Legendre functions,
no covariance, no transforms, no quadrature.  It only fixes the synthetic
workloads (sizes, radial grid, closed-form transfer kernels, covariance
parameters) and draws seeded random arrays (explicit noise, band-limited a_lm)
for tests that bypass the in-path counter-based generator.

The paper's own inputs (CAMB transfer functions, the WMAP5 cosmology, the
400-shell radial grid of Sect. 3) are not available; the closed forms below
stand in for them:

* radial nodes: midpoint rule on [13000, 15000] Mpc, r_i = 13000 + (i + 1/2) dr,
  weights w_i = dr = 2000 / N_r;
* temperature kernel  alpha^T_l(r) = exp(-(r - 14000)^2 / (2 * 200^2)) * cos((r - 14000) l / 14000);
* polarization kernel alpha^E_l(r) = 0.1 * alpha^T_l(r) * sin(l / 50);
* primordial power P(k) = A k^(n_s - 4) with A = 1.6e-8, n_s = 0.96 on a
  4096-point uniform trapezoid rule over k in [1e-4, 0.3] Mpc^-1, with a
  relative diagonal jitter of 1e-10 times the mean diagonal of C_l.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

R_MIN = 13000.0
R_MAX = 15000.0
R_LSS = 14000.0
SIGMA_LSS = 200.0


def n_alm(lmax: int) -> int:
    """Number of (l, m >= 0) coefficients up to lmax."""
    return (lmax + 1) * (lmax + 2) // 2


def alm_index(l, m, lmax: int):
    """Position of (l, m) in the m-major triangle: all l >= m for m = 0, then m = 1, ..."""
    return m * (2 * lmax + 1 - m) // 2 + l


def alm_lm(lmax: int):
    """Arrays (l, m) of every entry of the m-major triangle, in storage order."""
    ls, ms = [], []
    for m in range(lmax + 1):
        ls.append(np.arange(m, lmax + 1))
        ms.append(np.full(lmax + 1 - m, m))
    return np.concatenate(ls), np.concatenate(ms)


def smooth235_at_least(n: int) -> int:
    """Smallest integer >= n whose only prime factors are 2, 3 and 5."""
    k = max(int(n), 1)
    while True:
        v = k
        for p in (2, 3, 5):
            while v % p == 0:
                v //= p
        if v == 1:
            return k
        k += 1


def grid_for_lmax(lmax: int) -> tuple[int, int]:
    """Ring grid that resolves the square of a band-limited field exactly:
    n_theta = ceil((3 lmax + 1) / 2) Gauss-Legendre rings and the smallest
    2/3/5-smooth n_phi >= 3 lmax + 1."""
    return (3 * lmax + 2) // 2, smooth235_at_least(3 * lmax + 1)


def radial_grid(nr: int) -> tuple[np.ndarray, np.ndarray]:
    """Midpoint radial nodes r_i on [13000, 15000] Mpc and weights w_i = dr."""
    dr = (R_MAX - R_MIN) / nr
    r = R_MIN + (np.arange(nr) + 0.5) * dr
    w = np.full(nr, dr)
    return r, w


def transfer_kernels(lmax: int, r: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Closed-form synthetic transfer kernels alpha^T_l(r_i), alpha^E_l(r_i), shape [lmax+1, nr]."""
    l = np.arange(lmax + 1, dtype=np.float64)[:, None]
    d = (np.asarray(r, dtype=np.float64) - R_LSS)[None, :]
    env = np.exp(-d * d / (2.0 * SIGMA_LSS * SIGMA_LSS))
    aT = env * np.cos(d * l / R_LSS)
    aE = 0.1 * aT * np.sin(l / 50.0)
    return np.ascontiguousarray(aT), np.ascontiguousarray(aE)


@dataclass(frozen=True)
class CovParams:
    """Power-law primordial spectrum and the k rule for the radial covariance."""
    A: float = 1.6e-8
    ns: float = 0.96
    kmin: float = 1e-4
    kmax: float = 0.3
    nk: int = 4096
    jitter_rel: float = 1e-10


COV = CovParams()


@dataclass(frozen=True)
class Workload:
    name: str
    lmax: int
    nr: int
    ntheta: int
    nphi: int
    fnl: tuple = (0.0,)
    seeds: tuple = (1,)
    realisations: int = 1

    @property
    def nalm(self) -> int:
        return n_alm(self.lmax)


# The five synthetic workloads.  Sizes follow the paper's production setting
# (l_max = 1024, Sect. 3) scaled over a ladder of smaller cases.
SMALL = Workload("lmax32_nr16", 32, 16, 49, 100, fnl=(100.0,), seeds=(1,))
MEDIUM = Workload("lmax256_nr64", 256, 64, 385, 800, fnl=(0.0, 50.0), seeds=tuple(range(1, 9)), realisations=8)
FULL = Workload("lmax1024_nr128", 1024, 128, 1537, 3200, fnl=(30.0,), seeds=(1,))
GRAD = Workload("lmax512_nr96", 512, 96, 769, 1600, fnl=(20.0,), seeds=(2,))

WORKLOADS = {w.name: w for w in (SMALL, MEDIUM, FULL, GRAD)}


@dataclass(frozen=True)
class BatchInstance:
    lmax: int
    nr: int
    ntheta: int
    nphi: int
    fnl: float
    seed: int
    realisation: int


def batch_instances(n: int = 64, seed: int = 4) -> list[BatchInstance]:
    """Uneven batch: l_max from {128, 256, 512, 1024}, N_r from {32, 64, 96, 128}
    (each uniform), f_NL uniform in [-50, 50], grid by `grid_for_lmax`."""
    rng = np.random.default_rng(seed)
    lm = rng.choice([128, 256, 512, 1024], size=n)
    nr = rng.choice([32, 64, 96, 128], size=n)
    f = rng.uniform(-50.0, 50.0, size=n)
    out = []
    for i in range(n):
        nt, npf = grid_for_lmax(int(lm[i]))
        out.append(BatchInstance(int(lm[i]), int(nr[i]), nt, npf, float(f[i]), 1000 + i, i))
    return out


def gaussian_noise(lmax: int, nr: int, seed: int) -> np.ndarray:
    """Explicit white noise n_lm(r_j), complex, shape [nr, nalm]: m > 0 entries have
    independent real and imaginary parts of variance 1/2; m = 0 entries are real
    with variance 1."""
    rng = np.random.default_rng(seed)
    na = n_alm(lmax)
    z = (rng.standard_normal((nr, na)) + 1j * rng.standard_normal((nr, na))) / math.sqrt(2.0)
    m0 = lmax + 1  # the m = 0 block is the first lmax + 1 entries
    z[:, :m0] = rng.standard_normal((nr, m0))
    return z


def random_alm(lmax: int, nsh: int, seed: int, scale: float = 1.0) -> np.ndarray:
    """Band-limited coefficients of nsh real fields, shape [nalm, nsh] (m = 0 real)."""
    rng = np.random.default_rng(seed)
    na = n_alm(lmax)
    a = (rng.standard_normal((na, nsh)) + 1j * rng.standard_normal((na, nsh))) * (scale / math.sqrt(2.0))
    a[: lmax + 1, :] = a[: lmax + 1, :].real * math.sqrt(2.0)
    return a


def random_lower_filters(lmax: int, nr: int, seed: int, scale: float = 1e-4) -> np.ndarray:
    """Random lower-triangular per-l filters [lmax+1, nr, nr] with a positive diagonal,
    for tests that exercise the path without the covariance set-up."""
    rng = np.random.default_rng(seed)
    K = np.tril(rng.standard_normal((lmax + 1, nr, nr))) * (scale / math.sqrt(nr))
    d = np.arange(nr)
    K[:, d, d] = np.abs(K[:, d, d]) + scale / math.sqrt(nr)
    return K
