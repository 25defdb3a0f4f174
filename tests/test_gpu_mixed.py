"""GPU parity of the tensor-core forms (BF16-split Legendre GEMMs, FP32 ring FFT).

Stages are compared with the FP64 oracle; whole realisations with the FP64 GPU path on
the same Philox noise.  Bounds: the 2-term split (FNL_BF16X2) carries 16 significant
bits per operand, the 3-term split (FNL_BF16X3) 24; with FP32 FFTs and accumulation the
stage errors stay below the bounds written in each test, and a^X and a^X_NL of a full
l_max = 1024 realisation stay within the 1e-5 precision target.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

STAGE_BOUND = {"bf16x2": 2e-5, "bf16x3": 3e-6}
# the stated precision of the mixed forms: a^X and a^X_NL within rel 1e-5 of the FP64 path
TARGET = 1e-5


def nl_bound(prec: str, nr: int) -> float:
    """The a^X_NL bar of a configuration.  1e-5 for bf16x3 and FP32 everywhere, and for bf16x2
    from N_r = 16 shells on (measured 5.6e-6 .. 7.2e-6 for l_max 7 .. 1024).  With fewer shells
    the quadrature averages the two-term split's per-shell error (about 1.5e-5 rms after the
    synthesis, the square and the analysis) over too few independent shells, and a single draw
    reaches 1.0e-5 (l_max 7, N_r 8): there the bar is 2e-5."""
    return 2e-5 if (prec == "bf16x2" and nr < 16) else TARGET


def rel_l2(got, ref):
    got, ref = np.asarray(got), np.asarray(ref)
    return float(np.linalg.norm((got - ref).ravel()) / max(np.linalg.norm(ref.ravel()), 1e-300))


def cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.fixture(scope="module")
def F():
    from paper_0909_0009_gb300 import build
    build.build_library()
    import paper_0909_0009_gb300.fnl as F
    F.load_library()
    return F


class Pair:
    """A mixed-precision shells object and the FP64 one, on the same filters and mu."""

    def __init__(self, F, lmax, nr, ntheta, nphi, prec, K=None, store=True):
        self.lmax, self.nr, self.ntheta, self.nphi = lmax, nr, ntheta, nphi
        self.r, self.w = W.radial_grid(nr)
        self.aT, self.aE = W.transfer_kernels(lmax, self.r)
        self.K = W.random_lower_filters(lmax, nr, seed=lmax + nr, scale=8e-5) if K is None else K
        self.mu = O.mu_ensemble(self.K)
        self.grid = O.Grid(lmax, ntheta, nphi, store=store)
        args = (lmax, nr, ntheta, nphi, self.r, self.w, self.aT, self.aE)
        self.mx = F.Shells(*args, K=self.K, mu=self.mu, prec=prec)
        self.d64 = F.Shells(*args, K=self.K, mu=self.mu, prec="fp64")


@pytest.mark.parametrize("prec", ["bf16x2", "bf16x3"])
@pytest.mark.parametrize("lmax,nr,ntheta,nphi", [(32, 16, 49, 100), (96, 64, 145, 288), (128, 96, 193, 400)])
def test_stages_match_oracle(F, prec, lmax, nr, ntheta, nphi):
    c = Pair(F, lmax, nr, ntheta, nphi, prec)
    bound = STAGE_BOUND[prec]
    a = W.random_alm(lmax, nr, seed=21)
    assert rel_l2(host(c.mx.synth(cuda(a))), O.synthesis(a, c.grid)) < bound
    maps = np.random.default_rng(22).standard_normal((nr, ntheta, nphi))
    assert rel_l2(host(c.mx.analyse(cuda(maps))), O.analysis(maps, c.grid)) < bound
    phiL = O.phi_linear(c.K, O.philox_noise(lmax, nr, 5, 0))
    assert rel_l2(host(c.mx.square(cuda(phiL))), O.phi_nonlinear(phiL, c.mu, c.grid)) < 3 * bound
    c.mx.device_status()


@pytest.mark.parametrize("prec", ["bf16x2", "bf16x3"])
@pytest.mark.parametrize("lmax,nr,ntheta,nphi", [(256, 8, 385, 800), (300, 16, 452, 800), (512, 8, 769, 1600),
                                                  (1024, 8, 1537, 3200), (700, 24, 1051, 3200),
                                                  (1024, 4, 1537, 3125), (600, 12, 902, 3125),
                                                  (128, 8, 193, 400), (150, 16, 226, 400)])
def test_ring_square_specialised_sizes(F, prec, lmax, nr, ntheta, nphi):
    """n_phi = 400, 800, 1600, 3125 and 3200 have a specialised ring kernel (25 P Q
    factorisation, fused square; 3125 = 25 x 25 x 5 with 125-thread shell groups, 400 with
    16-thread groups in one warp): its square against the FP64 path's on the same Phi_L, odd
    and even n_theta, full and partial band limits."""
    c = Pair(F, lmax, nr, ntheta, nphi, prec, store=False)
    phiL = O.phi_linear(c.K, O.philox_noise(lmax, nr, 5, 0))
    got = host(c.mx.square(cuda(phiL)))
    ref = host(c.d64.square(cuda(phiL)))
    assert rel_l2(got, ref) < 3 * STAGE_BOUND[prec], rel_l2(got, ref)
    c.mx.device_status()


@pytest.mark.parametrize("prec", ["bf16x2", "bf16x3"])
@pytest.mark.parametrize("lmax,nr,ntheta,nphi", [(1, 1, 2, 4), (1, 3, 3, 6), (2, 5, 4, 8), (5, 7, 9, 16),
                                                  (9, 13, 15, 30), (17, 6, 27, 54)])
def test_edge_configurations(F, prec, lmax, nr, ntheta, nphi):
    """The smallest band limits and grids, one shell and shell counts that fill no shell group
    or 128-column tile (odd, below 8): the square per shell within the stage bound, and whole
    realisations against the FP64 path (a^X_L within 1e-6; a^X_NL for the three-term split
    within the 1e-5 bar, and for the two-term split within the per-shell stage bound, since a
    handful of shells averages nothing)."""
    c = Pair(F, lmax, nr, ntheta, nphi, prec)
    phiL = O.phi_linear(c.K, O.philox_noise(lmax, nr, 3, 1))
    got = host(c.mx.square(cuda(phiL)))
    assert rel_l2(got, O.phi_nonlinear(phiL, c.mu, c.grid)) < 3 * STAGE_BOUND[prec]
    nl = TARGET if prec == "bf16x3" else 3 * STAGE_BOUND[prec]
    for seed, fnl in ((1, 30.0), (4, 0.0)):
        a = c.mx.generate(seed, 0, fnl)
        b = c.d64.generate(seed, 0, fnl)
        for k in ("aLT", "aLE"):
            assert rel_l2(host(a[k]), host(b[k])) < 1e-6, k
        for k in ("aNLT", "aNLE"):
            assert rel_l2(host(a[k]), host(b[k])) < nl, (k, rel_l2(host(a[k]), host(b[k])))
    c.mx.device_status()


@pytest.mark.parametrize("prec", ["fp64", "bf16x2"])
def test_host_outputs_equal_device_outputs(F, prec):
    """fnl_generate_host writes page-locked buffers from the path's last kernel and copies into
    pageable ones; both must equal fnl_generate's device outputs bit for bit."""
    import torch
    c = Pair(F, 40, 16, 61, 125, prec)
    ref = {k: host(v) for k, v in c.mx.generate(7, 2, 25.0).items()}
    na = c.mx.nalm
    pinned = [torch.empty(na, dtype=torch.complex128, pin_memory=True).numpy() for _ in range(4)]
    pageable = [np.empty(na, dtype=np.complex128) for _ in range(4)]
    for bufs in (pinned, pageable, [pinned[0], pageable[1], None, pinned[3]]):
        for b in bufs:
            if b is not None:
                b[:] = np.nan
        c.mx.generate_host(7, 2, 25.0, bufs[0], bufs[1], bufs[2], bufs[3])
        torch.cuda.synchronize()
        for b, k in zip(bufs, ("aT", "aE", "aNLT", "aNLE")):
            if b is not None:
                assert np.array_equal(b, ref[k]), k
    c.mx.device_status()


@pytest.mark.parametrize("prec", ["bf16x2", "bf16x3"])
def test_filter_matches_oracle(F, prec):
    c = Pair(F, 64, 32, 97, 200, prec)
    phi = host(c.mx.filter(seed=7, realisation=2))
    # FP32 filter on FP32 noise from the same Philox words
    assert rel_l2(phi, O.phi_linear(c.K, O.philox_noise(64, 32, 7, 2))) < 1e-6


@pytest.mark.parametrize("prec", ["bf16x2", "bf16x3"])
@pytest.mark.parametrize("lmax,nr,ntheta,nphi", [(7, 8, 12, 25), (40, 16, 61, 125), (256, 64, 385, 800)])
def test_generate_matches_fp64_path(F, prec, lmax, nr, ntheta, nphi):
    c = Pair(F, lmax, nr, ntheta, nphi, prec)
    for seed, fnl in ((1, 50.0), (2, 0.0)):
        a = c.mx.generate(seed, 0, fnl)
        b = c.d64.generate(seed, 0, fnl)
        for k in ("aLT", "aLE"):
            assert rel_l2(host(a[k]), host(b[k])) < 1e-6, k
        # a^X carries f_NL times the error of a^X_NL
        for k in ("aT", "aE", "aNLT", "aNLE"):
            assert rel_l2(host(a[k]), host(b[k])) < nl_bound(prec, nr), (k, rel_l2(host(a[k]), host(b[k])))
    c.mx.device_status()


@pytest.mark.parametrize("prec", ["fp32", "bf16x2", "bf16x3"])
@pytest.mark.parametrize("lmax,nr,ntheta,nphi", [(32, 8, 33, 72), (32, 16, 40, 72), (48, 16, 52, 100)])
def test_generate_on_under_resolved_grids(F, prec, lmax, nr, ntheta, nphi):
    """Grids below the exact-square size (n_theta < (3 l_max + 2) / 2, n_phi < 3 l_max + 1,
    down to the smallest accepted n_theta = l_max + 1): the square's coefficients are aliased
    by the grid, and the mixed forms must give the oracle's aliased values.  Their monopole
    comes from Parseval's identity, which equals the grid's own analysis on every accepted
    grid (pinned on the CPU by test_parseval_monopole_on_minimal_grids).  The FP32 form sums the
    monopole on the grid like the oracle, in FP32."""
    c = Pair(F, lmax, nr, ntheta, nphi, prec)
    n = O.philox_noise(lmax, nr, 3, 0)
    ref = O.generate(c.K, n, c.grid, c.r, c.w, c.aT, c.aE, 40.0, mu=c.mu)
    out = c.mx.generate(3, 0, 40.0)
    for k in ("aT", "aE", "aNLT", "aNLE"):
        assert rel_l2(host(out[k]), ref[k]) < nl_bound(prec, nr), (k, rel_l2(host(out[k]), ref[k]))
    if prec != "fp32":  # the FP32 form sums the cancelling f^2 - mu on the grid
        # the monopole is a difference of two nearly equal sums (the sky mean of Phi_L^2 and
        # 4 pi mu) and may be far smaller than either: its error is bounded relative to the terms
        phiL = O.phi_linear(c.K, n)
        _, m = W.alm_lm(lmax)
        wgt = np.where(m == 0, 1.0, 2.0)[:, None]
        qT = O.quadrature_weights(c.r, c.w, c.aT)
        terms = float(np.dot(np.abs(qT[0]), ((wgt * np.abs(phiL) ** 2).sum(axis=0) + 4 * np.pi * c.mu)
                             / np.sqrt(4 * np.pi)))
        mono = abs(host(out["aNLT"])[0] - ref["aNLT"][0])
        assert mono < 1e-6 * terms, (mono, terms)
    c.mx.device_status()


@pytest.mark.parametrize("prec", ["bf16x2", "bf16x3"])
def test_generate_against_oracle_small(F, prec):
    c = Pair(F, 32, 16, 49, 100, prec)
    n = O.philox_noise(32, 16, 1, 0)
    ref = O.generate(c.K, n, c.grid, c.r, c.w, c.aT, c.aE, 100.0, mu=c.mu)
    out = c.mx.generate(1, 0, 100.0)
    for k in ("aT", "aE", "aNLT", "aNLE"):
        assert rel_l2(host(out[k]), ref[k]) < TARGET, k


@pytest.mark.slow
@pytest.mark.parametrize("prec", ["bf16x2", "bf16x3"])
def test_full_size_within_precision_target(F, prec):
    """l_max = 1024, N_r = 128, 1537 x 3200, covariance filters: the mixed form against the
    FP64 GPU path on the same noise, for a^X and for a^X_NL on its own."""
    wl = W.FULL
    r, w = W.radial_grid(wl.nr)
    aT, aE = W.transfer_kernels(wl.lmax, r)
    args = (wl.lmax, wl.nr, wl.ntheta, wl.nphi, r, w, aT, aE)
    mx = F.Shells(*args, prec=prec)
    d64 = F.Shells(*args, prec="fp64")
    a = mx.generate(1, 0, wl.fnl[0])
    b = d64.generate(1, 0, wl.fnl[0])
    errs = {k: rel_l2(host(a[k]), host(b[k])) for k in ("aT", "aE", "aNLT", "aNLE")}
    for k, e in errs.items():
        assert e < TARGET, errs
    mx.device_status()


def test_sm_limits_change_no_result(F):
    """Capping the SMs of the persistent GEMM and ring kernels changes which CTA takes a tile,
    not the order of any sum: the realisation is bit-identical."""
    r, w = W.radial_grid(16)
    aT, aE = W.transfer_kernels(100, r)
    K = W.random_lower_filters(100, 16, seed=3, scale=1e-4)
    sh = F.Shells(100, 16, 151, 800, r, w, aT, aE, K=K, prec="bf16x2")
    ref = sh.generate(2, 1, 25.0, parts=False)
    ref = {k: host(v) for k, v in ref.items()}
    for g, rg in ((30, 0), (0, 40), (7, 9)):
        sh.set_sm_limits(g, rg)
        out = sh.generate(2, 1, 25.0, parts=False)
        for k in ("aT", "aE"):
            assert np.array_equal(host(out[k]), ref[k]), (g, rg, k)
    sh.set_sm_limits(0, 0)
    with pytest.raises(F.FnlError):
        sh.set_sm_limits(-1, 0)


def test_gemm_work_shares(F):
    """fnl_shells_gemm_work: on an exact l_max 512 grid the tensor-core GEMMs leave out part of
    the polar ring pairs (both shares below 1); other synthesis tiles skip other whole tiles and
    leave the analysis's share alone; the SIMT forms compute everything and refuse the call."""
    lmax, nr, nt, nph = 512, 16, 769, 1600
    r, w = W.radial_grid(nr)
    aT, aE = W.transfer_kernels(lmax, r)
    K = W.random_lower_filters(lmax, nr, seed=3, scale=8e-5)
    sh = F.Shells(lmax, nr, nt, nph, r, w, aT, aE, K=K, prec="bf16x2")
    sh.set_tiles(112, 128)
    syn, ana = sh.gemm_work()
    assert 0.6 < syn < 0.99 and 0.6 < ana < 0.99, (syn, ana)
    sh.set_tiles(256, 128)
    syn2, ana2 = sh.gemm_work()
    assert 0.6 < syn2 <= 1.0 and ana2 == ana, (syn2, ana2)
    sh.close()
    d = F.Shells(lmax, nr, nt, nph, r, w, aT, aE, K=K, prec="fp32")
    with pytest.raises(F.FnlError):
        d.gemm_work()
    d.close()
