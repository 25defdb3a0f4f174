"""GPU parity of the adjoint (differentiation form) through the C ABI.

* fnl_generate_backward against the oracle's chain rule (``generate_backward``, itself
  pinned by dot-product tests and finite differences on the CPU): FP64 within rel 1e-12.
* The torch.autograd binding against the same, and against finite differences of the GPU
  forward at the l_max = 512, N_r = 96 workload (769 x 1600 grid): the loss
  L = sum_lm |a^T - d^T|^2 / C^TT_l + |a^E - d^E|^2 / C^EE_l, d drawn from a second seed at
  f_NL = 20, C_l from 16 f_NL = 0 draws, central differences with step 1e-6 in FP64 along
  32 random directions whose entries are drawn like the noise (unit variance per entry).
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

from test_gpu_parity import FP64_BAR, Case, cuda, host, rel_l2

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


def _random_g(lmax, seed):
    rng = np.random.default_rng(seed)
    na = W.n_alm(lmax)
    return rng.standard_normal(na) + 1j * rng.standard_normal(na)


def _check_backward(c, seed, real, fnl, noise=None, bar=FP64_BAR, gT=True, gE=True):
    gt = _random_g(c.lmax, 100 + seed) if gT else np.zeros(W.n_alm(c.lmax), complex)
    ge = _random_g(c.lmax, 200 + seed) if gE else np.zeros(W.n_alm(c.lmax), complex)
    n = O.philox_noise(c.lmax, c.nr, seed, real) if noise is None else noise
    ref_n, ref_f = O.generate_backward(c.K, n, c.grid, c.r, c.w, c.aT, c.aE, fnl, gt, ge, mu=c.mu)
    gn, gf = c.sh.generate_backward(seed, real, fnl, gT=cuda(gt) if gT else None, gE=cuda(ge) if gE else None,
                                    noise=None if noise is None else cuda(noise))
    e_n = rel_l2(host(gn), ref_n)
    e_f = abs(float(host(gf)) - ref_f) / max(abs(ref_f), 1e-300)
    assert e_n < bar and e_f < bar, (e_n, e_f)
    return e_n, e_f


@pytest.fixture(scope="module")
def small(F):
    wl = W.SMALL
    return Case(F, wl.lmax, wl.nr, wl.ntheta, wl.nphi)


def test_backward_philox_matches_oracle(small):
    _check_backward(small, 1, 0, 100.0)


def test_backward_explicit_noise_matches_oracle(small):
    _check_backward(small, 0, 0, -35.0, noise=W.gaussian_noise(small.lmax, small.nr, seed=4))


@pytest.mark.parametrize("gT,gE", [(True, False), (False, True)])
def test_backward_one_sided_loss(small, gT, gE):
    _check_backward(small, 2, 1, 60.0, gT=gT, gE=gE)


def test_backward_medium_matches_oracle(F):
    wl = W.MEDIUM
    c = Case(F, wl.lmax, wl.nr, wl.ntheta, wl.nphi, K=W.random_lower_filters(wl.lmax, wl.nr, seed=6, scale=8e-5))
    _check_backward(c, 3, 0, 50.0)


@pytest.mark.parametrize("lmax,nr,ntheta,nphi", [
    (1, 1, 2, 4), (2, 3, 4, 6), (5, 8, 9, 27), (7, 2, 12, 25), (13, 16, 20, 45),
])
def test_backward_edge_grids_match_oracle(F, lmax, nr, ntheta, nphi):
    c = Case(F, lmax, nr, ntheta, nphi, K=W.random_lower_filters(lmax, nr, seed=lmax, scale=1e-4))
    _check_backward(c, 3, 1, 17.0)


def test_backward_fp32_form(F, small):
    c32 = F.Shells(small.lmax, small.nr, small.ntheta, small.nphi, small.r, small.w, small.aT, small.aE,
                   K=small.K, mu=small.mu, prec="fp32")
    c = Case.__new__(Case)
    c.__dict__.update(small.__dict__)
    c.sh = c32
    # FP32 filter, Legendre sums and ring DFTs; FP64 quadrature: the forward's ~1e-6 bound
    _check_backward(c, 1, 0, 100.0, bar=2e-5)


def test_grad_fnl_with_and_without_forward_parts(small):
    """dL/df_NL from the a^X_NL the caller passes equals the one recomputed inside."""
    gt, ge = cuda(_random_g(small.lmax, 1)), cuda(_random_g(small.lmax, 2))
    out = small.sh.generate(5, 0, 10.0)
    _, f1 = small.sh.generate_backward(5, 0, 10.0, gT=gt, gE=ge, aNLT=out["aNLT"], aNLE=out["aNLE"],
                                       want_noise=False)
    _, f2 = small.sh.generate_backward(5, 0, 10.0, gT=gt, gE=ge, want_noise=False)
    assert abs(float(host(f1)) - float(host(f2))) <= 1e-14 * abs(float(host(f2)))


@pytest.mark.parametrize("prec,bar", [("bf16x2", 1e-5), ("bf16x3", 1e-6)])
@pytest.mark.parametrize("lmax,nr,ntheta,nphi", [(32, 16, 49, 100), (256, 64, 385, 800), (9, 5, 15, 30),
                                                  (17, 7, 27, 54)])
def test_backward_tensor_core_forms(F, prec, bar, lmax, nr, ntheta, nphi):
    """The adjoint of the tensor-core forms (both syntheses and the analysis as tcgen05 GEMMs on
    BF16-split operands, FP32 ring product and K_l^T) against the oracle's FP64 chain rule.
    dL/dn within `bar` (measured 3.7e-7 .. 2.2e-6 for bf16x2, 8e-8 .. 1.9e-7 for bf16x3);
    dL/df_NL = sum_X <gX, a^X_NL> is a dot product whose value may cancel far below its terms,
    so its error is bounded relative to sum_X |gX| |a^X_NL| (Cauchy-Schwarz), by the forward's
    own 1e-5 bar on a^X_NL."""
    K = W.random_lower_filters(lmax, nr, seed=6, scale=8e-5)
    c = Case(F, lmax, nr, ntheta, nphi, prec=prec, K=K, store=lmax <= 64)
    gt, ge = _random_g(lmax, 101), _random_g(lmax, 201)
    n = O.philox_noise(lmax, nr, 3, 0)
    ref_n, ref_f = O.generate_backward(c.K, n, c.grid, c.r, c.w, c.aT, c.aE, 50.0, gt, ge, mu=c.mu)
    ref = O.generate(c.K, n, c.grid, c.r, c.w, c.aT, c.aE, 50.0, mu=c.mu)
    gn, gf = c.sh.generate_backward(3, 0, 50.0, gT=cuda(gt), gE=cuda(ge))
    assert rel_l2(host(gn), ref_n) < bar, rel_l2(host(gn), ref_n)
    scale = np.linalg.norm(gt) * np.linalg.norm(ref["aNLT"]) + np.linalg.norm(ge) * np.linalg.norm(ref["aNLE"])
    assert abs(float(host(gf)) - ref_f) < 1e-5 * scale, (float(host(gf)), ref_f, scale)
    # the imaginary part of every m = 0 entry is zero, as the forward ignores it
    _, m = W.alm_lm(lmax)
    assert np.all(host(gn)[:, m == 0].imag == 0.0)
    c.sh.device_status()


def test_backward_rejects_batch_clones_and_healpix(F, small):
    hp = F.Shells(small.lmax, small.nr, small.ntheta, small.nphi, small.r, small.w, small.aT, small.aE,
                  K=small.K, mu=small.mu, prec="fp64", nside=8)
    with pytest.raises(F.FnlError) as e:
        hp.generate_backward(1, 0, 1.0, gT=cuda(_random_g(small.lmax, 1)))
    assert e.value.code == 4
    hp.close()


def test_autograd_matches_oracle(small):
    import torch
    from paper_0909_0009_gb300.autograd import generate
    n = W.gaussian_noise(small.lmax, small.nr, seed=8)
    wt, we = _random_g(small.lmax, 3), _random_g(small.lmax, 4)
    noise = cuda(n).requires_grad_(True)
    f = torch.tensor(42.0, dtype=torch.float64, requires_grad=True)
    aT, aE = generate(small.sh, noise, f)
    # L = Re <wt, aT> + Re <we, aE>: dL/daT = wt, dL/daE = we
    loss = (torch.conj(cuda(wt)) * aT).real.sum() + (torch.conj(cuda(we)) * aE).real.sum()
    loss.backward()
    ref_n, ref_f = O.generate_backward(small.K, n, small.grid, small.r, small.w, small.aT, small.aE, 42.0, wt, we,
                                       mu=small.mu)
    assert rel_l2(host(noise.grad), ref_n) < FP64_BAR
    assert abs(float(f.grad) - ref_f) < FP64_BAR * abs(ref_f)


def test_autograd_gradcheck_tiny(F):
    """torch.autograd.gradcheck (numerical Jacobian in FP64) on an l_max = 4 case."""
    import torch
    from paper_0909_0009_gb300.autograd import generate
    lmax, nr = 4, 3
    nt, npf = W.grid_for_lmax(lmax)
    c = Case(F, lmax, nr, nt, npf, K=W.random_lower_filters(lmax, nr, seed=2, scale=0.3))
    n = torch.from_numpy(W.gaussian_noise(lmax, nr, seed=3)).cuda()
    m0 = torch.zeros_like(n, dtype=torch.bool)
    m0[:, : lmax + 1] = True
    n = torch.where(m0, n.real.to(n.dtype), n).requires_grad_(True)  # the forward ignores Im n_l0
    f = torch.tensor(3.0, dtype=torch.float64, requires_grad=True)

    with torch.no_grad():
        scale = float(generate(c.sh, n, f)[0].abs().max())

    def fn(noise, fnl):
        # Im n_l0 is not an input of the method: project it out so the numerical Jacobian agrees
        noise = torch.where(m0, noise.real.to(noise.dtype), noise)
        aT, aE = generate(c.sh, noise, fnl)
        return aT / scale, aE / scale  # O(1) outputs, so that atol means something

    assert torch.autograd.gradcheck(fn, (n, f), eps=1e-6, atol=1e-8, rtol=1e-6)


# ---------------------------------------------------------------------------------------
# finite differences at l_max = 512, N_r = 96 on the 769 x 1600 grid
# ---------------------------------------------------------------------------------------

@pytest.mark.slow
def test_finite_differences_grad_workload(F):
    import torch
    from paper_0909_0009_gb300.autograd import generate
    wl = W.GRAD
    r, w = W.radial_grid(wl.nr)
    aT, aE = W.transfer_kernels(wl.lmax, r)
    sh = F.Shells(wl.lmax, wl.nr, wl.ntheta, wl.nphi, r, w, aT, aE, prec="fp64")  # K from Eq. 7
    L = wl.lmax
    ls, ms = W.alm_lm(L)
    wm = torch.from_numpy(np.where(ms == 0, 1.0, 2.0)).cuda()
    # C_l from the f_NL = 0 ensemble of 16 draws (seeds 100..115)
    acc = {"T": torch.zeros(L + 1, dtype=torch.float64, device="cuda"),
           "E": torch.zeros(L + 1, dtype=torch.float64, device="cuda")}
    lt = torch.from_numpy(ls).cuda()
    for s in range(100, 116):
        o = sh.generate(s, 0, 0.0, parts=False)
        for X in ("T", "E"):
            acc[X].index_add_(0, lt, wm * o["a" + X].abs() ** 2)
    ell = torch.arange(L + 1, dtype=torch.float64, device="cuda")
    Cl = {X: acc[X] / 16.0 / (2 * ell + 1) for X in acc}
    keep = (lt >= 2).to(torch.float64)  # C^EE_0 = 0: l < 2 left out of the loss
    inv = {X: keep * wm / torch.where(lt >= 2, Cl[X][lt], torch.ones_like(Cl[X][lt])) for X in Cl}
    d = sh.generate(wl.seeds[0], 0, wl.fnl[0], parts=False)  # data: second seed, f_NL = 20
    n0 = cuda(W.gaussian_noise(L, wl.nr, seed=1))
    f0 = float(wl.fnl[0])

    def loss_terms(aT_, aE_):
        return (inv["T"] * (aT_ - d["aT"]).abs() ** 2).sum() + (inv["E"] * (aE_ - d["aE"]).abs() ** 2).sum()

    noise = n0.clone().requires_grad_(True)
    fnl = torch.tensor(f0, dtype=torch.float64, device="cuda", requires_grad=True)
    aT_, aE_ = generate(sh, noise, fnl)
    loss_terms(aT_, aE_).backward()
    gn, gf = noise.grad.detach(), float(fnl.grad)

    def dloss(pairs):
        # L(+) - L(-) in factored form, sum inv |.|^2 differences without cancelling the sums:
        # |p - d|^2 - |q - d|^2 = Re((p - q) conj(p + q - 2 d))
        s = 0.0
        for X, (p, q) in zip(("T", "E"), pairs):
            s += float((inv[X] * ((p - q) * torch.conj(p + q - 2 * d["a" + X])).real).sum())
        return s

    h = 1e-6
    gen = torch.Generator(device="cuda").manual_seed(7)
    errs = []
    m0 = torch.zeros(wl.nr, W.n_alm(L), dtype=torch.bool, device="cuda")
    m0[:, : L + 1] = True
    for _ in range(32):
        u = torch.randn((wl.nr, W.n_alm(L)), dtype=torch.complex128, device="cuda", generator=gen)
        u = torch.where(m0, u.real.to(u.dtype), u)
        # entries distributed like the noise itself (unit variance each), so a step of 1e-6 is
        # a relative change of 1e-6 in every n_lm(r_j); normalising u over all 2.5e7 entries
        # would leave each entry a step of ~2e-10, below what FP64 differences resolve
        npl, nmi = n0 + h * u, n0 - h * u
        op = sh.generate(0, 0, f0, noise=npl, parts=False)
        om = sh.generate(0, 0, f0, noise=nmi, parts=False)
        fd = dloss([(op["aT"], om["aT"]), (op["aE"], om["aE"])]) / (2 * h)
        # the step actually taken: n0 +- h u rounds h u (~1e-10 per entry against n0 ~ 1) to a
        # relative ~1e-6, which would otherwise swamp the comparison
        du = (npl - nmi) / (2 * h)
        an = float((torch.conj(gn) * du).real.sum())
        errs.append(abs(fd - an) / abs(an))
    # f_NL direction
    op = sh.generate(0, 0, f0 + h, noise=n0, parts=False)
    om = sh.generate(0, 0, f0 - h, noise=n0, parts=False)
    fd_f = dloss([(op["aT"], om["aT"]), (op["aE"], om["aE"])]) / (2 * h)
    err_f = abs(fd_f - gf) / abs(gf)
    print(f"FD vs adjoint at l_max=512: noise directions max rel {max(errs):.2e} median "
          f"{float(np.median(errs)):.2e}; f_NL rel {err_f:.2e}")
    assert max(errs) < 1e-6 and err_f < 1e-6, (errs, err_f)
