"""Multi-rank host logic of the replicas path, as two gloo ranks on the CPU.

On N GPUs every rank generates its own block of realisations (no data-path collective);
the job's time is the maximum over ranks and its throughput counts every rank's
realisations.  Here two CPU ranks run that logic with the FP64 oracle standing in for the
GPU path at a tiny size, and the test checks that the ranks' realisations are disjoint and
together equal the serial run, and that the timing reduction is a true maximum.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

STEPS = 2
LMAX, NR, NT, NP = 3, 2, 5, 10


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _realisation(real: int):
    import oracle as O
    import workloads as W
    r, w = W.radial_grid(NR)
    aT, aE = W.transfer_kernels(LMAX, r)
    K = W.random_lower_filters(LMAX, NR, seed=3, scale=1e-4)
    grid = O.Grid(LMAX, NT, NP)
    out = O.generate(K, O.philox_noise(LMAX, NR, 1, real), grid, r, w, aT, aE, 30.0)
    return out["aT"]


def _rank(rank: int, world: int, port: int, q):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        reals = [bench.realisation_of(rank, STEPS, i) for i in range(STEPS)]
        maps = [_realisation(k) for k in reals]
        # a rank-dependent "time": the reduction must return the largest
        t = bench.max_over_ranks(1.0 + rank, dist)
        # gather the results for the check only (the path itself exchanges nothing)
        got = [None] * world
        dist.all_gather_object(got, (reals, [m.tolist() for m in maps]))
        q.put((rank, t, bench.job_throughput(world, STEPS, t), got))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_generate_disjoint_realisations():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    world = 2
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    _, t0, v0, gathered = res[0]
    assert t0 == res[1][1] == 2.0                      # max over ranks
    assert v0 == res[1][2] == world * STEPS / 2.0      # every rank's realisations / slowest time
    reals = [k for rr, _ in gathered for k in rr]
    assert sorted(reals) == list(range(world * STEPS))  # disjoint, and together the first N x steps
    for rr, maps in gathered:
        for k, m in zip(rr, maps):
            np.testing.assert_array_equal(np.array(m), _realisation(k))


def test_single_rank_reduction_is_identity():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.realisation_of(0, 5, 3) == 3 and bench.realisation_of(2, 5, 3) == 13
    assert bench.job_throughput(4, 10, 2.0) == 20.0
    with pytest.raises(ZeroDivisionError):
        bench.job_throughput(1, 1, 0.0)
