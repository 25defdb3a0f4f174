"""GPU parity of shell shards (fnl_make_shells_shard).

A shard runs steps (i)-(v) for a contiguous range of shells of a configuration; the radial
quadrature (Eq. 5) and Eq. 3 are sums over shells, so the outputs of shards that partition the
shells add up to the whole configuration's.  Every shell's Phi_L, Phi_NL and the BF16 stages
are computed exactly as in the whole object (the same noise words, the same order of the
filter sums); only the quadrature's partial sums are split, so the sums agree to the rounding
of those sums (1e-12 of the output scale).  Each shard is also checked against the oracle's
shard terms, and the entry points that need a whole configuration refuse a shard.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

OUTS = ("aT", "aE", "aLT", "aLE", "aNLT", "aNLE")
LMAX, NR, NT, NP = 64, 32, 97, 200


@pytest.fixture(scope="module")
def F():
    from paper_0909_0009_gb300 import build
    build.build_library()
    import paper_0909_0009_gb300.fnl as F
    F.load_library()
    return F


def _inputs(lmax=LMAX, nr=NR):
    r, w = W.radial_grid(nr)
    aT, aE = W.transfer_kernels(lmax, r)
    K = W.random_lower_filters(lmax, nr, seed=21, scale=8e-5)
    return r, w, aT, aE, K


def _host(out):
    import torch
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16x2", "bf16x3"])
@pytest.mark.parametrize("parts", [[(0, 16), (16, 32)], [(0, 8), (8, 24), (24, 32)], [(0, 5), (5, 18), (18, 32)]])
def test_shards_sum_to_the_whole_configuration(F, prec, parts):
    r, w, aT, aE, K = _inputs()
    whole = F.Shells(LMAX, NR, NT, NP, r, w, aT, aE, K=K, prec=prec)
    ref = _host(whole.generate(3, 1, 25.0))
    acc = {k: 0.0 for k in OUTS}
    for j0, j1 in parts:
        sh = F.Shells(LMAX, NR, NT, NP, r, w, aT, aE, K=K, prec=prec, shard=(j0, j1))
        assert sh.nr == j1 - j0 and sh.j0 == j0
        got = _host(sh.generate(3, 1, 25.0))
        for k in OUTS:
            acc[k] = acc[k] + got[k]
        sh.device_status()
        sh.close()
    for k in OUTS:
        scale = np.max(np.abs(ref[k]))
        assert np.max(np.abs(acc[k] - ref[k])) <= 1e-12 * scale, (k, np.max(np.abs(acc[k] - ref[k])) / scale)
    whole.close()


@pytest.mark.parametrize("prec,bound", [("fp64", 1e-12), ("bf16x2", 3e-5)])
def test_shard_matches_oracle_shard_terms(F, prec, bound):
    # the mixed bound is the stage bound of the two-term split on a shard of 8 shells
    lmax, nr, nt, nph = 24, 16, 37, 80
    r, w, aT, aE, K = _inputs(lmax, nr)
    grid = O.Grid(lmax, nt, nph)
    noise = O.philox_noise(lmax, nr, 5, 2)
    whole = F.Shells(lmax, nr, nt, nph, r, w, aT, aE, K=K, prec="fp64")
    mu = whole.mu
    whole.close()
    j0, j1 = 4, 12
    ref = O.generate_shard(K, noise, grid, r, w, aT, aE, 40.0, j0, j1, mu=mu)
    sh = F.Shells(lmax, nr, nt, nph, r, w, aT, aE, K=K, prec=prec, shard=(j0, j1))
    got = _host(sh.generate(5, 2, 40.0))
    for k in OUTS:
        err = np.linalg.norm(got[k] - ref[k]) / np.linalg.norm(ref[k])
        assert err <= bound, (k, err)
    sh.close()


def test_shard_explicit_noise_reads_shells_below_j1(F):
    import torch
    r, w, aT, aE, K = _inputs()
    j0, j1 = 8, 24
    sh = F.Shells(LMAX, NR, NT, NP, r, w, aT, aE, K=K, prec="fp64", shard=(j0, j1))
    noise = torch.from_numpy(np.ascontiguousarray(O.philox_noise(LMAX, NR, 9, 0)[:j1])).cuda()
    a = _host(sh.generate(0, 0, 12.0, noise=noise))
    noise2 = noise.clone()
    noise2[j0:] *= 2.0  # the noise of shells j0 .. j1 - 1 drives the shard linearly in a^X_L
    b = _host(sh.generate(0, 0, 12.0, noise=noise2))
    c = _host(sh.generate(9, 0, 12.0))  # the same shells drawn on the device
    for k in OUTS:
        assert np.max(np.abs(a[k] - c[k])) <= 1e-12 * np.max(np.abs(c[k])), k
    assert np.max(np.abs(b["aLT"] - a["aLT"])) > 1e-3 * np.max(np.abs(a["aLT"]))
    sh.close()


def test_one_rank_sharded_driver_is_the_whole_object(F):
    from paper_0909_0009_gb300 import sharded
    r, w, aT, aE, K = _inputs()
    drv = sharded.ShardedShells(LMAX, NR, NT, NP, r, w, aT, aE, K=K, prec="bf16x2")
    assert drv.range == (0, NR) and drv.world == 1
    got = _host(drv.generate(4, 0, 20.0))
    whole = F.Shells(LMAX, NR, NT, NP, r, w, aT, aE, K=K, prec="bf16x2")
    ref = _host(whole.generate(4, 0, 20.0))
    for k in OUTS:
        assert np.array_equal(got[k], ref[k]), k
    drv.close()
    whole.close()


def test_shard_info_and_refusals(F):
    import ctypes
    r, w, aT, aE, K = _inputs()
    sh = F.Shells(LMAX, NR, NT, NP, r, w, aT, aE, K=K, prec="bf16x2", shard=(8, 16))
    j0, n, nt = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    assert F._lib.fnl_shells_shard(sh.handle, ctypes.byref(j0), ctypes.byref(n), ctypes.byref(nt)) == 0
    assert (j0.value, n.value, nt.value) == (8, 8, NR)
    with pytest.raises(F.FnlError) as e:
        sh.generate_backward(1, 0, 10.0)
    assert e.value.code == 4
    with pytest.raises(F.FnlError) as e:
        F.Ksw(sh)
    assert e.value.code == 4
    sh.close()
    for bad in [(-1, 8), (8, 8), (16, 8), (0, NR + 1)]:
        with pytest.raises(F.FnlError) as e:
            F.Shells(LMAX, NR, NT, NP, r, w, aT, aE, K=K, prec="fp64", shard=bad)
        assert e.value.code == 1, bad


@pytest.mark.parametrize("world", [2, 8])
def test_full_size_shards_sum_to_the_whole_configuration(F, world):
    """The bench's sharded configuration (l_max 1024, N_r 128, 1537 x 3200, bf16x2): the shards
    of `world` ranks (shell_ranges, units of 8 shells) sum to the whole object's outputs."""
    from paper_0909_0009_gb300 import sharded
    wl = W.FULL
    r, w = W.radial_grid(wl.nr)
    aT, aE = W.transfer_kernels(wl.lmax, r)
    K = W.random_lower_filters(wl.lmax, wl.nr, seed=21, scale=8e-5)
    whole = F.Shells(wl.lmax, wl.nr, wl.ntheta, wl.nphi, r, w, aT, aE, K=K, prec="bf16x2")
    ref = _host(whole.generate(2, 3, 30.0))
    whole.close()
    acc = {k: 0.0 for k in OUTS}
    for j0, j1 in sharded.shell_ranges(wl.nr, world):
        sh = F.Shells(wl.lmax, wl.nr, wl.ntheta, wl.nphi, r, w, aT, aE, K=K, prec="bf16x2", shard=(j0, j1))
        got = _host(sh.generate(2, 3, 30.0))
        for k in OUTS:
            acc[k] = acc[k] + got[k]
        sh.device_status()
        sh.close()
    for k in OUTS:
        scale = np.max(np.abs(ref[k]))
        assert np.max(np.abs(acc[k] - ref[k])) <= 1e-12 * scale, (k, np.max(np.abs(acc[k] - ref[k])) / scale)
