"""Failure paths of the library on the GPU, made without faulting or hanging the GPU.

- A bounded device wait that runs out: the test hook fnl_test_wait_expiry runs the wait
  routine of the tensor-core kernels on an mbarrier that nothing completes, with a short
  try limit.  The wait records its code in the object's error word and returns; the host
  then reads FNL_ETIMEOUT from fnl_device_status, the word is cleared, and the context stays
  usable (a realisation right after it is bit-identical to one before).
- A device allocation that fails: the hook fnl_test_fail_alloc makes the n-th allocation of
  the set-up fail as cudaMalloc would (without calling it); fnl_make_shells must return
  FNL_ENOMEM and free everything it had allocated (the device's free memory is back where it
  was).
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    from paper_0909_0009_gb300 import build
    build.build_library()
    import paper_0909_0009_gb300.fnl as F
    F.load_library()
    return F


def _make(F, prec, lmax=64, nr=16, ntheta=97, nphi=200):
    r, w = W.radial_grid(nr)
    aT, aE = W.transfer_kernels(lmax, r)
    K = W.random_lower_filters(lmax, nr, seed=11, scale=8e-5)
    return F.Shells(lmax, nr, ntheta, nphi, r, w, aT, aE, K=K, prec=prec)


def test_bounded_wait_expires_and_reports_timeout(F):
    import torch
    sh = _make(F, "bf16x2")
    ref = {k: v.cpu().numpy() for k, v in sh.generate(5, 1, 20.0, parts=False).items()}
    sh.device_status()  # nothing recorded so far
    assert F._lib.fnl_test_wait_expiry(sh.handle, 2000, F._stream()) == 0
    with pytest.raises(F.FnlError) as err:
        sh.device_status()
    assert err.value.code == 5 and "code 6" in str(err.value)
    sh.device_status()  # the word was cleared
    out = sh.generate(5, 1, 20.0, parts=False)
    torch.cuda.synchronize()
    for k in ("aT", "aE"):
        assert np.array_equal(out[k].cpu().numpy(), ref[k]), k
    sh.device_status()
    # the hook refuses objects without the error word and out-of-range limits
    s64 = _make(F, "fp64")
    assert F._lib.fnl_test_wait_expiry(s64.handle, 10, F._stream()) == 1
    assert F._lib.fnl_test_wait_expiry(sh.handle, 0, F._stream()) == 1
    s64.close()
    sh.close()


@pytest.mark.parametrize("prec", ["bf16x2", "fp64"])
def test_failed_allocation_unwinds_make_shells(F, prec):
    import torch
    _make(F, prec).close()  # loads every set-up kernel once
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    failed = 0
    try:
        for n in (0, 1, 3, 8, 15, 25, 40):
            assert F._lib.fnl_test_fail_alloc(n) == 0
            try:
                sh = _make(F, prec)
            except F.FnlError as e:
                assert e.code == 2 and "simulated" in str(e), str(e)
                failed += 1
            else:  # fewer allocations than n + 1: the object is whole
                sh.close()
            F._lib.fnl_test_fail_alloc(-1)
            torch.cuda.synchronize()
            free, _ = torch.cuda.mem_get_info()
            assert free == free0, (n, free0 - free)
    finally:
        F._lib.fnl_test_fail_alloc(-1)
    assert failed >= 5
    sh = _make(F, prec)  # the hook is off again
    sh.generate(1, 0, 10.0, parts=False)
    torch.cuda.synchronize()
    sh.close()
    assert F._lib.fnl_test_fail_alloc(-2) == 1
