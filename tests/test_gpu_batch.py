"""GPU tests of the batching form (fnl_batch_create / fnl_generate_batch) and the tile autotuner.

A batch runs the same kernels on the same inputs as single fnl_generate calls, only
captured into one graph over several streams, so every instance must match the single call
bit for bit; the tile shape changes no accumulation order, so the autotuner's choice must
leave every result bit-identical too.  The uneven l_max = 128 ... 1024 batch of 64
realisations (grids by the exact-square rule) is checked the same way on sampled
instances, and one l_max = 1024 instance against the FP64 GPU path.
"""
import time

import numpy as np
import pytest

import workloads as W

from test_gpu_parity import host, rel_l2

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


def make(F, lmax, nr, prec="bf16x2", seed=0, grid=None):
    nt, npf = grid or W.grid_for_lmax(lmax)
    r, w = W.radial_grid(nr)
    aT, aE = W.transfer_kernels(lmax, r)
    K = W.random_lower_filters(lmax, nr, seed=seed or lmax + nr, scale=8e-5)
    return F.Shells(lmax, nr, nt, npf, r, w, aT, aE, K=K, prec=prec)


def singles(shells, seeds, reals, fnls):
    out = []
    for s, sd, rl, f in zip(shells, seeds, reals, fnls):
        o = s.generate(sd, rl, f, parts=False)
        out.append((host(o["aT"]), host(o["aE"])))
    return out


def assert_same(batch_out, ref):
    for i, ((bt, be), (rt, re)) in enumerate(zip(batch_out, ref)):
        assert np.array_equal(host(bt), rt) and np.array_equal(host(be), re), i


@pytest.mark.parametrize("prec,nstreams", [("bf16x2", 0), ("bf16x2", 1), ("bf16x3", 3), ("fp64", 2), ("fp32", 0)])
def test_batch_matches_single_calls(F, prec, nstreams):
    """Stream mode (ring lengths 50, 100, 150 have no specialised ring kernel)."""
    A, B, C = make(F, 16, 8, prec), make(F, 32, 16, prec), make(F, 48, 24, prec)
    inst = [A, B, A, C, B, C, A]
    b = F.Batch(inst, nstreams=nstreams)
    assert not b.multi
    lanes = b.lanes()
    if prec in ("fp64", "fp32"):
        # repeated objects of the SIMT forms share their scratch: one stream each
        for s in (A, B, C):
            assert len({lanes[i] for i, x in enumerate(inst) if x is s}) == 1
    for call in range(2):  # the second call updates the instantiated graph in place
        seeds = [11 + 7 * i + call for i in range(len(inst))]
        reals = [i % 3 for i in range(len(inst))]
        fnls = [-40.0 + 13.0 * i + call for i in range(len(inst))]
        out = b.generate(seeds, reals, fnls)
        assert_same(out, singles(inst, seeds, reals, fnls))


@pytest.mark.parametrize("prec", ["bf16x2", "bf16x3"])
def test_multi_instance_batch_matches_single_calls(F, prec):
    """Multi-instance mode: ring lengths 800, 1600 and 3125 (specialised kernels), repeated
    objects (scratch clones), two calls (the second updates the graph); every instance bit
    for bit equal to a single call on its object with the tile shape the batch picked."""
    A = make(F, 100, 8, prec, grid=(151, 800))
    B = make(F, 200, 16, prec, grid=(301, 1600))
    C = make(F, 150, 8, prec, grid=(226, 800))
    D = make(F, 300, 12, prec, grid=(451, 3125))
    inst = [A, B, A, C, D, B, A, D]
    b = F.Batch(inst)
    assert b.multi
    syn, ana = b.tiles()
    assert syn in (96, 112, 128) and ana in (128, 256)
    for call in range(2):
        seeds = [5 + 3 * i + call for i in range(len(inst))]
        reals = [i % 2 for i in range(len(inst))]
        fnls = [-25.0 + 9.0 * i - call for i in range(len(inst))]
        out = b.generate(seeds, reals, fnls)
        assert_same(out, singles(inst, seeds, reals, fnls))
    # and against the FP64 GPU path, within the mixed forms' bound
    d64 = make(F, 300, 12, "fp64", grid=(451, 3125))
    ref = d64.generate(seeds[4], reals[4], fnls[4], parts=False)
    assert rel_l2(host(out[4][0]), host(ref["aT"])) < 1e-5


def test_batch_runs_shell_shards_in_stream_mode(F):
    """Shell shards (fnl_make_shells_shard) in a batch: stream mode, every instance bit for bit
    equal to its single call, and the shards of one realisation adding up to the whole object."""
    lmax, nr, grid = 100, 16, (151, 800)
    r, w = W.radial_grid(nr)
    aT, aE = W.transfer_kernels(lmax, r)
    K = W.random_lower_filters(lmax, nr, seed=9, scale=8e-5)
    whole = F.Shells(lmax, nr, *grid, r, w, aT, aE, K=K, prec="bf16x2")
    s0 = F.Shells(lmax, nr, *grid, r, w, aT, aE, K=K, prec="bf16x2", shard=(0, 8))
    s1 = F.Shells(lmax, nr, *grid, r, w, aT, aE, K=K, prec="bf16x2", shard=(8, 16))
    inst = [s0, s1, s0]
    b = F.Batch(inst)
    assert not b.multi
    seeds, reals, fnls = [3, 3, 4], [1, 1, 0], [20.0, 20.0, -5.0]
    out = b.generate(seeds, reals, fnls)
    assert_same(out, singles(inst, seeds, reals, fnls))
    ref = whole.generate(3, 1, 20.0, parts=False)
    for j, k in enumerate(("aT", "aE")):
        got = host(out[0][j]) + host(out[1][j])
        want = host(ref[k])
        assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want)), k
    b.close()
    for sh in (whole, s0, s1):
        sh.close()


def test_batch_rejects_bad_arguments(F):
    A = make(F, 16, 8)
    with pytest.raises(F.FnlError):
        F.Batch([], nstreams=0)
    with pytest.raises(F.FnlError):
        F.Batch([A], nstreams=65)
    b = F.Batch([A])
    import torch
    hostbuf = torch.empty(W.n_alm(16), dtype=torch.complex128)
    with pytest.raises(F.FnlError):
        b.generate([1], [0], [1.0], out=[(hostbuf, hostbuf)])


@pytest.mark.parametrize("lmax,nr", [(48, 24), (256, 64)])
def test_tile_shapes_change_no_result(F, lmax, nr):
    s = make(F, lmax, nr)
    ref = singles([s], [5], [1], [25.0])
    for syn, ana in ((64, 64), (112, 256), (256, 128), (128, 128), (112, 96)):
        s.set_tiles(syn, ana)
        assert_same([tuple(s.generate(5, 1, 25.0, parts=False)[k] for k in ("aT", "aE"))], ref)
    nsyn, nana = s.autotune()
    assert 64 <= nsyn <= 256 and nana in (96, 128, 256)
    assert_same([tuple(s.generate(5, 1, 25.0, parts=False)[k] for k in ("aT", "aE"))], ref)
    with pytest.raises(F.FnlError):
        s.set_tiles(40, 128)


@pytest.mark.slow
def test_uneven_batch_of_64(F):
    """The l_max in {128, 256, 512, 1024}, N_r in {32, 64, 96, 128} batch: 64 realisations,
    f_NL uniform in [-50, 50], one graph launch; sampled instances bit-exact against single
    calls, one l_max = 1024 instance within 1e-5 of the FP64 GPU path."""
    import torch
    insts = W.batch_instances()
    objs = {}
    for x in insts:
        if (x.lmax, x.nr) not in objs:
            objs[(x.lmax, x.nr)] = make(F, x.lmax, x.nr, seed=x.lmax + x.nr)
    tuned = {k: s.autotune() for k, s in objs.items()}
    shells = [objs[(x.lmax, x.nr)] for x in insts]
    b = F.Batch(shells)
    assert b.multi
    seeds = [x.seed for x in insts]
    reals = [x.realisation for x in insts]
    fnls = [x.fnl for x in insts]
    out = b.generate(seeds, reals, fnls)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(3):
        b.generate(seeds, reals, fnls, out=out)
    torch.cuda.synchronize()
    t_batch = (time.perf_counter() - t0) / 3
    t0 = time.perf_counter()
    for s, sd, rl, f in zip(shells, seeds, reals, fnls):
        s.generate(sd, rl, f, parts=False)
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    print(f"uneven batch of 64: {t_batch * 1e3:.1f} ms per graph launch ({64 / t_batch:.1f} realisations/s), "
          f"{t_seq * 1e3:.1f} ms as single calls on one stream; tiles {tuned}")
    pick = [0, 17, 33, 63] + [i for i, x in enumerate(insts) if x.lmax == 1024][:2]
    assert_same([out[i] for i in pick], singles([shells[i] for i in pick], [seeds[i] for i in pick],
                                                [reals[i] for i in pick], [fnls[i] for i in pick]))
    i = next(i for i, x in enumerate(insts) if x.lmax == 1024)
    x = insts[i]
    d64 = make(F, x.lmax, x.nr, prec="fp64", seed=x.lmax + x.nr)
    ref = d64.generate(x.seed, x.realisation, x.fnl, parts=False)
    for k, j in (("aT", 0), ("aE", 1)):
        assert rel_l2(host(out[i][j]), host(ref[k])) < 1e-5, k
