"""GPU parity of the HEALPix grid variant (fnl_make_shells_healpix) against the FP64 oracle.

- fnl_synth and fnl_analyse on RING-ordered maps within 1e-12 of oracle.healpix_synthesis /
  healpix_analysis, including band limits above 2 nside (the short polar rings alias) and
  nside = 1.
- A whole realisation (steps (i)-(v) with (ii)-(iv) on HEALPix) within 1e-12 of the oracle (FP64)
  and the FP32 form within the bound of its ring transforms.
- The Gauss-Legendre-only entry points refuse a HEALPix object.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

from test_gpu_parity import cuda, host, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    import torch
    from paper_0909_0009_gb300 import build
    build.build_library()
    import paper_0909_0009_gb300.fnl as F
    F.load_library()
    assert torch.cuda.is_available()
    return F


def make(F, L, nr, nside, prec="fp64", K=None):
    r, w = W.radial_grid(nr)
    aT, aE = W.transfer_kernels(L, r)
    K = W.random_lower_filters(L, nr, seed=L + nr, scale=1e-4) if K is None else K
    return F.Shells(L, nr, 0, 0, r, w, aT, aE, K=K, prec=prec, nside=nside), (r, w, aT, aE, K)


@pytest.mark.parametrize("L,nside", [(16, 8), (20, 4), (3, 1), (40, 16)])
def test_synth_and_analyse_match_oracle(F, L, nside):
    nr = 3
    sh, _ = make(F, L, nr, nside)
    g = O.HealpixGrid(L, nside)
    a = W.random_alm(L, nr, seed=L)
    maps = host(sh.synth(cuda(np.ascontiguousarray(a))))
    ref = O.healpix_synthesis(a, g)
    assert rel_l2(maps, ref) < 1e-12
    rng = np.random.default_rng(nside)
    m = rng.standard_normal((nr, g.npix))
    got = host(sh.analyse(cuda(m)))
    assert rel_l2(got, O.healpix_analysis(m, g)) < 1e-12


@pytest.mark.parametrize("L,nr,nside", [(16, 4, 8), (24, 3, 8), (48, 5, 32)])
def test_generate_matches_oracle(F, L, nr, nside):
    sh, (r, w, aT, aE, K) = make(F, L, nr, nside)
    n = O.philox_noise(L, nr, 3, 1)
    ref = O.healpix_generate(K, n, O.HealpixGrid(L, nside), r, w, aT, aE, 40.0, mu=sh.mu)
    out = sh.generate(3, 1, 40.0)
    for k in ("aT", "aE", "aLT", "aLE", "aNLT", "aNLE"):
        assert rel_l2(host(out[k]), ref[k]) < 1e-12, k


def test_fp32_generate_against_fp64(F):
    L, nr, nside = 64, 8, 32
    d64, (r, w, aT, aE, K) = make(F, L, nr, nside)
    d32, _ = make(F, L, nr, nside, prec="fp32", K=K)
    a = d64.generate(5, 0, 30.0)
    b = d32.generate(5, 0, 30.0)
    for k in ("aT", "aE", "aNLT", "aNLE"):
        e = rel_l2(host(b[k]), host(a[k]))
        assert e < 2e-5, (k, e)


def test_unsupported_uses_are_refused(F):
    with pytest.raises(F.FnlError):
        make(F, 16, 8, 8, prec="bf16x2")
    sh, _ = make(F, 16, 3, 8)
    with pytest.raises(F.FnlError):
        sh.maps_prepare()
    with pytest.raises(F.FnlError):
        F.Ksw(sh)
