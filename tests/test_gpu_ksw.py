"""GPU parity of the fast cubic f_NL estimator (fnl_ksw_*) against the FP64 oracle.

- S_prim of the FP64 object within rel 1e-12 of oracle.ksw_statistic, for transfer kernels with
  E proportional to T (the workload's, C_l of rank one) and independent ones (rank two), on
  exact grids, an even ring count and the smallest band limits.
- The normalisation (FP64 on the device for every precision form) within 1e-12 of the sum the
  paper writes (oracle), and at l_max 1024 within 1e-10 of the oracle's quadrature form.
- FP32 and mixed objects: S_prim within the bound of their synthesis (stated below).
- Skies from the generator: the estimate recovers f_NL (mean within 4 standard errors over
  realisations, Gaussian variance 1/N), and at l_max 1024 the mixed estimate agrees with the
  FP64 one to a small fraction of its statistical error.
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W

from test_gpu_parity import cuda, host

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


def kernels(L, nr, independent, seed=3):
    r, w = W.radial_grid(nr)
    if independent:
        rng = np.random.default_rng(seed)
        aT, aE = rng.uniform(0.5, 1.5, (L + 1, nr)), rng.uniform(-1.0, 1.0, (L + 1, nr))
    else:
        aT, aE = W.transfer_kernels(L, r)
    K = W.random_lower_filters(L, nr, seed=seed, scale=1e-4)
    return r, w, aT, aE, K


def setup(F, L, nr, nt, nph, prec, independent):
    r, w, aT, aE, K = kernels(L, nr, independent)
    sh = F.Shells(L, nr, nt, nph, r, w, aT, aE, K=K, prec=prec)
    return sh, F.Ksw(sh), O.ksw_weights(K, r, w, aT, aE)


def sky(L, seed):
    a = W.random_alm(L, 2, seed=seed, scale=1e-5)
    return np.ascontiguousarray(a[:, 0]), np.ascontiguousarray(a[:, 1])


@pytest.mark.parametrize("independent", [False, True])
@pytest.mark.parametrize("L,nr,nt,nph", [
    (32, 4, 49, 100),     # the small workload's grid (exact for the cubic)
    (20, 3, 32, 64),      # even ring count
    (2, 2, 4, 8),         # only l = 2 contributes
    (48, 5, 75, 150),
])
def test_fp64_statistic_and_norm_match_oracle(F, L, nr, nt, nph, independent):
    sh, k, wts = setup(F, L, nr, nt, nph, "fp64", independent)
    assert np.array_equal(k.rank, wts["rank"])
    aT, aE = sky(L, seed=L + nr)
    S = float(host(k.statistic(cuda(aT), cuda(aE))))
    ref = O.ksw_statistic(aT, aE, O.Grid(L, nt, nph), wts)
    assert abs(S - ref) < 1e-12 * abs(ref), (S, ref)
    if L <= 32:
        nref = O.ksw_normalisation_direct(wts)
        assert abs(k.norm - nref) < 1e-12 * nref, (k.norm, nref)


def test_odd_shell_count_of_the_tensor_core_forms_is_refused(F):
    # the tensor-core coefficient kernel takes a field's shells two at a time; the SIMT forms
    # take any count (the FP64 cases above include 3 and 5 shells)
    r, w, aT, aE, K = kernels(24, 5, False)
    sh = F.Shells(24, 5, 37, 75, r, w, aT, aE, K=K, prec="bf16x2")
    with pytest.raises(F.FnlError) as e:
        F.Ksw(sh)
    assert e.value.code == 4 and "even" in str(e.value)
    sh.close()


def test_band_limit_one_has_no_estimator(F):
    sh, k, wts = setup(F, 1, 2, 3, 6, "fp64", False)
    aT, aE = sky(1, seed=1)
    assert k.norm == 0.0 and float(host(k.statistic(cuda(aT), cuda(aE)))) == 0.0


@pytest.mark.parametrize("prec,bar,L,nt,nph", [
    ("fp32", 2e-5, 48, 75, 150), ("bf16x2", 2e-4, 48, 75, 150), ("bf16x3", 2e-5, 48, 75, 150),
    # ring lengths with the specialised ring kernel of the tensor-core forms
    ("bf16x2", 2e-4, 100, 151, 800), ("bf16x3", 2e-5, 120, 181, 400)])
def test_reduced_precision_statistic(F, prec, bar, L, nt, nph):
    """FP32 / mixed synthesis of A and B (relative map errors ~1e-7 / ~1e-5 per stage) make
    S_prim, a sum with cancellations, accurate to the bar stated here relative to the scale
    sqrt(sum over the rings of (A B^2)^2) of its terms (measured: 6e-9 FP32, 4e-7 / 9e-7 bf16x3,
    1.5e-6 bf16x2)."""
    nr = 8
    sh, k, wts = setup(F, L, nr, nt, nph, prec, True)
    aT, aE = sky(L, seed=4)
    S = float(host(k.statistic(cuda(aT), cuda(aE))))
    grid = O.Grid(L, nt, nph)
    ref = O.ksw_statistic(aT, aE, grid, wts)
    At, Bt = O.ksw_filtered(aT, aE, wts)
    A, B = O.synthesis(At, grid), O.synthesis(Bt, grid)
    w = wts["u"][:, None, None] * grid.w[None, :, None] * (2 * math.pi / nph)
    scale = math.sqrt(float(np.sum((w * A * B * B) ** 2)))
    print(f"{prec} l_max {L} {nt}x{nph}: |S - S_oracle| / scale = {abs(S - ref) / scale:.3g}")
    assert abs(S - ref) < bar * scale, (S, ref, scale)
    nref = O.ksw_normalisation_direct(wts) if L <= 32 else O.ksw_normalisation(wts)
    assert abs(k.norm - nref) < 1e-12 * nref


def test_norm_at_lmax_1024_matches_quadrature_form(F):
    L, nr = 1024, 4
    nt, nph = W.FULL.ntheta, W.FULL.nphi
    sh, k, wts = setup(F, L, nr, nt, nph, "bf16x2" if nr % 8 == 0 else "fp32", False)
    nref = O.ksw_normalisation(wts)
    assert abs(k.norm - nref) < 1e-10 * nref, (k.norm, nref)
    assert k.norm_seconds < 5.0


@pytest.mark.slow
def test_estimate_recovers_fnl_from_generated_skies(F):
    """l_max 256, N_r 16, exact grid, filters of the Eq. 7 covariance: 48 skies at f_NL = 0 and
    48 at f_NL = f0 (20 sigma); means within 4 standard errors, Gaussian variance 1/N within
    4 sqrt(2 / M)."""
    import torch
    L, nr, nt, nph = 256, 16, 385, 800
    r, w = W.radial_grid(nr)
    aT, aE = W.transfer_kernels(L, r)
    sh = F.Shells(L, nr, nt, nph, r, w, aT, aE, prec="bf16x2")
    k = F.Ksw(sh)
    sigma = 1.0 / math.sqrt(k.norm)
    f0 = 20.0 * sigma
    M = 48
    est = {}
    for f in (0.0, f0):
        vals = []
        for i in range(M):
            o = sh.generate(7, i, f, parts=False)
            vals.append(k.statistic(o["aT"], o["aE"]))
        torch.cuda.synchronize()
        est[f] = np.array([float(v.item()) for v in vals]) / k.norm
    print(f"sigma(f_NL) = {sigma:.4g}; f_NL = 0: mean {est[0.0].mean():.4g}, sd {est[0.0].std():.4g}; "
          f"f_NL = {f0:.4g}: mean {est[f0].mean():.4g}, sd {est[f0].std():.4g}")
    se = sigma / math.sqrt(M)
    assert abs(est[0.0].mean()) < 4 * se
    assert abs(est[f0].mean() - f0) < 4 * se * max(1.0, est[f0].std() / sigma)
    assert abs(est[0.0].var() / sigma ** 2 - 1.0) < 4 * math.sqrt(2.0 / M)


@pytest.mark.slow
def test_full_size_mixed_estimate_matches_fp64(F):
    """l_max 1024, N_r 128, 1537 x 3200: one generated sky (f_NL = 30); the bf16x2 estimator's
    f_NL within 1e-2 standard deviations of the FP64 estimator's, same normalisation."""
    wl = W.FULL
    r, w = W.radial_grid(wl.nr)
    aT, aE = W.transfer_kernels(wl.lmax, r)
    K = W.random_lower_filters(wl.lmax, wl.nr, seed=1, scale=8e-5)
    mixed = F.Shells(wl.lmax, wl.nr, wl.ntheta, wl.nphi, r, w, aT, aE, K=K, prec="bf16x2")
    o = mixed.generate(1, 0, 30.0, parts=False)
    km = F.Ksw(mixed)
    f_mixed = km.fnl(o["aT"], o["aE"])
    d64 = F.Shells(wl.lmax, wl.nr, wl.ntheta, wl.nphi, r, w, aT, aE, K=K, prec="fp64")
    kd = F.Ksw(d64)
    f_64 = kd.fnl(o["aT"], o["aE"])
    sigma = 1.0 / math.sqrt(kd.norm)
    print(f"l_max 1024: f_NL mixed {f_mixed:.6g}, FP64 {f_64:.6g}, sigma {sigma:.4g}; "
          f"norm {km.norm:.6g} / {kd.norm:.6g} in {km.norm_seconds:.3f} s")
    assert abs(km.norm - kd.norm) < 1e-12 * kd.norm
    assert abs(f_mixed - f_64) < 1e-2 * sigma
