"""Host-side tests of libfnl (no GPU): the C ABI loads and exports every symbol of
include/fnl.h, argument validation, and the host set-up helpers against the oracle."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle as O
import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fnl():
    from paper_0909_0009_gb300 import build
    build.build_library()
    import paper_0909_0009_gb300.fnl as F
    F.load_library()
    return F


def _header_symbols():
    src = open(os.path.join(ROOT, "include", "fnl.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fnl_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol(fnl):
    declared = _header_symbols()
    assert declared, "no declarations found"
    lib = ctypes.CDLL(fnl.LIB_PATH)
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(fnl.EXPORTS) == declared
    out = os.popen(f"nm -D --defined-only {fnl.LIB_PATH}").read()
    for name in declared:
        assert re.search(rf"\bT {name}\b", out), name
    assert fnl.load_library().fnl_version().decode().startswith("libfnl")


def test_gauss_legendre_matches_oracle(fnl):
    for n in (1, 2, 7, 49, 385, 1537):
        x, w = fnl.gauss_legendre(n)
        xo, wo = O.gauss_legendre(n)
        assert np.max(np.abs(x - xo)) < 2e-16
        assert np.max(np.abs(w - wo) / wo) < 1e-13


def test_covariance_and_filters_match_oracle(fnl):
    L, nr = 40, 16
    r, _ = W.radial_grid(nr)
    cp = W.COV
    C = fnl.covariance(L, r, cp.A, cp.ns, cp.kmin, cp.kmax, cp.nk)
    Co = O.covariance(L, r, cp.A, cp.ns, cp.kmin, cp.kmax, cp.nk)
    scale = np.abs(Co).max(axis=(1, 2))[:, None, None]
    assert np.max(np.abs(C - Co) / scale) < 1e-12
    K = fnl.cholesky_filters(C, cp.jitter_rel)
    Ko = O.filters(Co, cp.jitter_rel)
    assert np.allclose(np.triu(K, 1), 0)
    assert np.max(np.abs(K - Ko) / np.abs(Ko).max(axis=(1, 2))[:, None, None]) < 1e-9


@pytest.mark.slow
def test_covariance_high_l_matches_oracle(fnl):
    L, nr = 1024, 4
    r, _ = W.radial_grid(nr)
    cp = W.COV
    C = fnl.covariance(L, r, cp.A, cp.ns, cp.kmin, cp.kmax, cp.nk)
    Co = O.covariance(L, r, cp.A, cp.ns, cp.kmin, cp.kmax, cp.nk)
    scale = np.abs(Co).max(axis=(1, 2))[:, None, None]
    assert np.max(np.abs(C - Co) / scale) < 1e-11


def test_host_helpers_reject_bad_arguments(fnl):
    with pytest.raises(fnl.FnlError):
        fnl.gauss_legendre(0)
    with pytest.raises(fnl.FnlError):
        fnl.covariance(4, np.array([-1.0, 2.0]), 1.0, 1.0, 1e-4, 0.3, 16)
    bad = np.zeros((3, 2, 2))
    bad[:, 0, 0] = -1.0
    with pytest.raises(fnl.FnlError, match="positive definite"):
        fnl.cholesky_filters(bad, 0.0)


def test_make_shells_validates_before_touching_the_gpu(fnl):
    r, w = W.radial_grid(4)
    aT, aE = W.transfer_kernels(8, r)
    cases = [dict(lmax=8, nr=4, ntheta=8, nphi=20),    # ntheta < lmax + 1
             dict(lmax=8, nr=4, ntheta=13, nphi=17),   # nphi < 2 lmax + 2
             dict(lmax=8, nr=4, ntheta=13, nphi=49),   # nphi not 2/3/5-smooth
             dict(lmax=0, nr=4, ntheta=13, nphi=27)]   # lmax < 1
    for c in cases:
        with pytest.raises(fnl.FnlError) as e:
            fnl.Shells(c["lmax"], c["nr"], c["ntheta"], c["nphi"], r, w, aT[: c["lmax"] + 1], aE[: c["lmax"] + 1])
        assert e.value.code == 1
