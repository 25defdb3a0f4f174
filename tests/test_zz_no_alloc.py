"""fnl_accumulate_noalloc against fnl_accumulate (collected last on purpose).

fnl_accumulate_noalloc serves callers that may not allocate device memory: their memory
belongs to another allocator, or cudaMalloc's device synchronisation is not acceptable
where they run.  It forms the quadrature weights in a fixed array inside the library
instead of taking them from a shells object.  These tests compare it with fnl_accumulate
on the same inputs, on two calls in a row of different sizes (the second call finds the
first call's weights in the shared array), and check that a size beyond the array is
rejected before anything runs.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-12  # the FP64 bound of the other parity tests


def rel_l2(got, ref):
    got, ref = np.asarray(got), np.asarray(ref)
    return float(np.linalg.norm((got - ref).ravel()) / max(np.linalg.norm(ref.ravel()), 1e-300))


@pytest.fixture(scope="module")
def F():
    from paper_0909_0009_gb300 import build
    build.build_library()
    import paper_0909_0009_gb300.fnl as F
    F.load_library()
    return F


class Case:
    def __init__(self, F, lmax, nr, seed):
        import torch
        self.lmax, self.nr = lmax, nr
        self.r, self.w = W.radial_grid(nr)
        self.aT, self.aE = W.transfer_kernels(lmax, self.r)
        K = W.random_lower_filters(lmax, nr, seed=seed, scale=8e-5)
        ntheta, nphi = lmax + 1, W.smooth235_at_least(2 * lmax + 2)
        self.sh = F.Shells(lmax, nr, ntheta, nphi, self.r, self.w, self.aT, self.aE, K=K, prec="fp64")
        rng = np.random.default_rng(seed)
        nalm = W.n_alm(lmax)
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        self.phiL = dev(rng.standard_normal((nalm, nr)) + 1j * rng.standard_normal((nalm, nr)))
        self.phiNL = dev(rng.standard_normal((nalm, nr)) + 1j * rng.standard_normal((nalm, nr)))
        self.d_r, self.d_w, self.d_aT, self.d_aE = dev(self.r), dev(self.w), dev(self.aT), dev(self.aE)
        self.out = {k: torch.zeros(nalm, dtype=torch.complex128, device="cuda") for k in F.NOALLOC_OUTPUTS}


def _check_case(F, c, ref, fnl):
    for k in F.NOALLOC_OUTPUTS:
        e = rel_l2(c.out[k].cpu().numpy(), ref[k].cpu().numpy())
        assert e < TOL, (c.lmax, c.nr, k, e)


def test_noalloc_matches_accumulate_on_two_calls(F):
    import torch
    cases = [Case(F, 40, 16, 3), Case(F, 96, 24, 4)]
    fnl = 37.5
    refs = [c.sh.accumulate(c.phiL, c.phiNL, fnl) for c in cases]
    torch.cuda.synchronize()
    for c in cases:  # two calls in a row, sharing the library's scratch array
        F.accumulate_noalloc(c.lmax, c.nr, c.d_r, c.d_w, c.d_aT, c.d_aE, c.phiL, c.phiNL, fnl, out=c.out)
    torch.cuda.synchronize()
    for c, ref in zip(cases, refs):
        _check_case(F, c, ref, fnl)
    # the other order: the small call follows a larger one whose weights still fill the array
    # beyond (and inside) the region the small call uses, and must rewrite what it reads
    for c in reversed(cases):
        for t in c.out.values():
            t.fill_(float("nan"))
        F.accumulate_noalloc(c.lmax, c.nr, c.d_r, c.d_w, c.d_aT, c.d_aE, c.phiL, c.phiNL, fnl, out=c.out)
    torch.cuda.synchronize()
    for c, ref in zip(cases, refs):
        _check_case(F, c, ref, fnl)
    # phiL absent counts as zero, as in fnl_accumulate
    c = cases[0]
    ref = c.sh.accumulate(None, c.phiNL, fnl)
    F.accumulate_noalloc(c.lmax, c.nr, c.d_r, c.d_w, c.d_aT, c.d_aE, None, c.phiNL, fnl, out=c.out)
    torch.cuda.synchronize()
    for k in F.NOALLOC_OUTPUTS:
        assert rel_l2(c.out[k].cpu().numpy(), ref[k].cpu().numpy()) < TOL, k
    for cc in cases:
        cc.sh.close()


def test_noalloc_allocates_no_device_memory(F):
    """After a first call (which looks up the array's address and may load the library's
    device code), further calls of other sizes leave the device's free memory and the
    caching allocator's count unchanged."""
    import torch
    cases = [Case(F, 64, 8, 6), Case(F, 24, 32, 7)]
    c0 = cases[0]
    F.accumulate_noalloc(c0.lmax, c0.nr, c0.d_r, c0.d_w, c0.d_aT, c0.d_aE, c0.phiL, c0.phiNL, 3.0, out=c0.out)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for c in cases + cases:
        F.accumulate_noalloc(c.lmax, c.nr, c.d_r, c.d_w, c.d_aT, c.d_aE, c.phiL, c.phiNL, 3.0, out=c.out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    assert torch.cuda.memory_allocated() == alloc0
    for c in cases:
        c.sh.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(F):
    """The library itself rejects a size beyond its array (called through the C ABI with
    bare pointers, past the binding's own shape checks)."""
    import torch
    c = Case(F, 8, 8, 5)
    lmax, nr = 4096, 128  # (lmax + 1) nr = 524416 > 524288
    outs = [F._ptr(c.out[k]) for k in F.NOALLOC_OUTPUTS]
    code = F._lib.fnl_accumulate_noalloc(lmax, nr, F._ptr(c.d_r), F._ptr(c.d_w), F._ptr(c.d_aT), F._ptr(c.d_aE),
                                         F._ptr(c.phiL), None, 0.0, *outs, F._stream())
    assert code == 1 and "exceeds the fixed scratch" in F._lib.fnl_last_error().decode()
    code = F._lib.fnl_accumulate_noalloc(8, 8, None, F._ptr(c.d_w), F._ptr(c.d_aT), F._ptr(c.d_aE),
                                         F._ptr(c.phiL), None, 0.0, *outs, F._stream())
    assert code == 1
    # the binding refuses arrays of the wrong type or shape before the call
    with pytest.raises(ValueError):
        F.accumulate_noalloc(8, 8, c.d_r.float(), c.d_w, c.d_aT, c.d_aE, c.phiL, None, 0.0, out=c.out)
    with pytest.raises(ValueError):
        F.accumulate_noalloc(8, 8, c.d_r, c.d_w, c.d_aT, c.d_aE, c.phiL[:-1], None, 0.0, out=c.out)
    torch.cuda.synchronize()
    c.sh.close()
