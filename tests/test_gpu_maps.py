"""GPU parity of the Stokes maps (fnl_maps_prepare / fnl_maps) against the FP64 oracle.

I = sum a^T Y, Q +- iU = sum a_{+-2} +-2Y with a_{+-2} = -(a^E +- i a^B) (Sect. 4; the HEALPix
sign convention).  Bars: the FP64 object within rel 1e-12 (L2 per map) of oracle.maps_iqu
on the same seeded coefficients; FP32 tables and sums (FP32 and mixed objects) within 1e-5.
At the full l_max = 1024 grid the oracle evaluates sampled rings only (its tables restricted
to those rings' nodes), compared element by element with the same rings of the GPU maps.
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W

from test_gpu_parity import cuda, host, rel_l2

pytestmark = pytest.mark.gpu

FP64_BAR = 1e-12
FP32_BAR = 1e-5


@pytest.fixture(scope="module")
def F():
    import torch
    from paper_0909_0009_gb300 import build
    build.build_library()
    import paper_0909_0009_gb300.fnl as F
    F.load_library()
    assert torch.cuda.is_available()
    return F


def shells(F, lmax, nr, ntheta, nphi, prec):
    r, w = W.radial_grid(nr)
    aT, aE = W.transfer_kernels(lmax, r)
    K = W.random_lower_filters(lmax, nr, seed=lmax + nr, scale=1e-4)
    return F.Shells(lmax, nr, ntheta, nphi, r, w, aT, aE, K=K, prec=prec)


def coefficients(lmax, seed):
    a = W.random_alm(lmax, 3, seed)
    return [np.ascontiguousarray(a[:, k]) for k in range(3)]


def gpu_maps(sh, aT, aE, aB):
    sh.maps_prepare()
    return host(sh.maps(cuda(aT), cuda(aE), None if aB is None else cuda(aB)))


def check_maps(got, ref, bar):
    for k, name in enumerate("IQU"):
        e = rel_l2(got[k], ref[k])
        assert e < bar, (name, e)


@pytest.mark.parametrize("lmax,ntheta,nphi", [
    (32, 49, 100),       # the small workload's grid
    (256, 385, 800),     # the medium workload's grid
    (1, 2, 4),           # no spin-2 content: Q = U = 0
    (2, 3, 6),           # the first spin-2 degree only, odd rings
    (7, 12, 25),         # even ring count (no equator), radix 5
    (40, 61, 125),
    (100, 150, 216),     # a grid wider than the exact-square one
])
def test_fp64_maps_match_oracle(F, lmax, ntheta, nphi):
    sh = shells(F, lmax, 2, ntheta, nphi, "fp64")
    aT, aE, aB = coefficients(lmax, seed=lmax + 7)
    got = gpu_maps(sh, aT, aE, aB)
    ref = O.maps_iqu(aT, aE, aB, O.Grid(lmax, ntheta, nphi))
    if lmax < 2:
        assert np.max(np.abs(got[1:])) == 0.0
        assert rel_l2(got[0], ref[0]) < FP64_BAR
    else:
        check_maps(got, ref, FP64_BAR)


@pytest.mark.parametrize("prec", ["fp32", "bf16x2", "bf16x3"])
def test_fp32_table_maps_match_oracle(F, prec):
    wl = W.MEDIUM
    sh = shells(F, wl.lmax, 16, wl.ntheta, wl.nphi, prec)
    aT, aE, aB = coefficients(wl.lmax, seed=3)
    got = gpu_maps(sh, aT, aE, aB)
    check_maps(got, O.maps_iqu(aT, aE, aB, O.Grid(wl.lmax, wl.ntheta, wl.nphi)), FP32_BAR)


def test_null_b_modes_equal_zero_b_modes(F):
    sh = shells(F, 48, 2, 73, 150, "fp64")
    aT, aE, _ = coefficients(48, seed=5)
    a = gpu_maps(sh, aT, aE, None)
    b = gpu_maps(sh, aT, aE, np.zeros_like(aE))
    assert np.array_equal(a, b)
    check_maps(a, O.maps_iqu(aT, aE, None, O.Grid(48, 73, 150)), FP64_BAR)


def test_single_e_mode_closed_form(F):
    """a^E_20 = 1 alone: Q = -2Y_20 = -(1/4) sqrt(15 / (2 pi)) sin^2 theta on every ring, U = 0."""
    L, nt, nph = 8, 13, 20
    sh = shells(F, L, 2, nt, nph, "fp64")
    z = np.zeros(W.n_alm(L), dtype=np.complex128)
    aE = z.copy()
    aE[W.alm_index(2, 0, L)] = 1.0
    got = gpu_maps(sh, z, aE, None)
    x, _ = O.gauss_legendre(nt)
    ref = -0.25 * math.sqrt(15 / (2 * math.pi)) * (1 - x ** 2)
    assert np.max(np.abs(got[1] - ref[:, None])) < 1e-14
    assert np.max(np.abs(got[2])) < 1e-15 and np.max(np.abs(got[0])) == 0.0


def test_maps_round_trip_through_oracle_analysis(F):
    """The oracle's spin-2 analysis of the GPU's Q, U returns a^E, a^B (exact on this grid)."""
    L, nt, nph = 24, 37, 60
    sh = shells(F, L, 2, nt, nph, "fp64")
    aT, aE, aB = coefficients(L, seed=9)
    got = gpu_maps(sh, aT, aE, aB)
    rE, rB = O.analysis_spin2(got[1], got[2], O.Grid(L, nt, nph))
    # l < 2 carry no spin-2 signal
    keep = np.array([l >= 2 for m in range(L + 1) for l in range(m, L + 1)])
    assert rel_l2(rE[keep], aE[keep]) < 1e-12 and rel_l2(rB[keep], aB[keep]) < 1e-12


def test_maps_errors(F):
    import ctypes
    sh = shells(F, 16, 2, 25, 50, "fp64")
    aT, aE, _ = coefficients(16, seed=1)
    with pytest.raises(F.FnlError):  # before fnl_maps_prepare
        sh.maps(cuda(aT), cuda(aE))
    sh.maps_prepare()
    sh.maps_prepare()  # idempotent
    out = cuda(np.zeros((3, 25, 50)))
    st = F._stream()
    lib = F.load_library()
    for args in ((None, cuda(aE)), (cuda(aT), None)):
        code = lib.fnl_maps(sh.handle, F._ptr(args[0]), F._ptr(args[1]), None, F._ptr(out), st)
        assert code == 1  # FNL_EINVAL
    code = lib.fnl_maps(sh.handle, F._ptr(cuda(aT)), F._ptr(cuda(aE)), None, None, st)
    assert code == 1
    host_maps = np.zeros((3, 25, 50))
    code = lib.fnl_maps(sh.handle, F._ptr(cuda(aT)), F._ptr(cuda(aE)), None,
                        ctypes.c_void_p(host_maps.ctypes.data), st)
    assert code == 1


class RingSubset:
    """The oracle's grid restricted to some rings of an n_theta-ring Gauss-Legendre grid (its
    lambda columns from the oracle's recurrences at those nodes only)."""

    def __init__(self, lmax, ntheta, nphi, rings):
        x, _ = O.gauss_legendre(ntheta)
        self.lmax, self.nphi, self.ntheta = lmax, nphi, len(rings)
        self.x = x[np.asarray(rings)]
        self._mm = O.lambda_mm(lmax, self.x)

    def lam(self, m):
        return O.lambda_column(m, self.lmax, self.x, self._mm)


@pytest.mark.slow
def test_full_grid_sampled_rings(F):
    """l_max = 1024 on the 1537 x 3200 grid, mixed object (FP32 tables): sampled rings of all
    three maps against the oracle element by element, within the FP32 bar per ring."""
    wl = W.FULL
    sh = shells(F, wl.lmax, 8, wl.ntheta, wl.nphi, "bf16x2")
    aT, aE, aB = coefficients(wl.lmax, seed=11)
    got = gpu_maps(sh, aT, aE, aB)
    rings = [0, 1, 17, 400, wl.ntheta // 2, 1100, wl.ntheta - 2, wl.ntheta - 1]
    ref = O.maps_iqu(aT, aE, aB, RingSubset(wl.lmax, wl.ntheta, wl.nphi, rings))
    for k, name in enumerate("IQU"):
        for i, j in enumerate(rings):
            e = rel_l2(got[k, j], ref[k, i])
            assert e < FP32_BAR, (name, j, e)
