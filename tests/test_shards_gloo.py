"""Multi-rank host logic of the shell-sharded path, as gloo ranks on the CPU.

On N GPUs every rank runs the shard of its shell range and one all-reduce (sum) of the
partial outputs gives the realisation (`paper_0909_0009_gb300.sharded`).  Here CPU ranks run
that logic with the FP64 oracle's shard terms standing in for the GPU path at a tiny size; the
test checks that the ranges partition the shells and that the all-reduced outputs equal the
serial recipe on every rank, including a rank left without shells.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

LMAX, NR, NT, NP = 4, 6, 7, 14
FNL = 30.0


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _setup():
    import oracle as O
    import workloads as W
    r, w = W.radial_grid(NR)
    aT, aE = W.transfer_kernels(LMAX, r)
    K = W.random_lower_filters(LMAX, NR, seed=3, scale=1e-4)
    return O, r, w, aT, aE, K, O.Grid(LMAX, NT, NP), O.philox_noise(LMAX, NR, 1, 4)


def _rank(rank: int, world: int, align: int, port: int, q):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist

    from paper_0909_0009_gb300 import sharded
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        O, r, w, aT, aE, K, grid, noise = _setup()
        j0, j1 = sharded.shell_ranges(NR, world, align)[rank]

        def partial(out):
            terms = O.generate_shard(K, noise, grid, r, w, aT, aE, FNL, j0, j1)
            for k, t in out.items():
                t.copy_(torch.from_numpy(terms[k]))

        nalm = (LMAX + 1) * (LMAX + 2) // 2
        out = sharded.generate_sharded(partial if j1 > j0 else None, nalm)
        q.put((rank, (j0, j1), {k: v.numpy().copy() for k, v in out.items()}))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,align", [(2, 2), (3, 4)])
def test_gloo_ranks_sum_their_shards_to_the_serial_recipe(world, align):
    # (3, 4): units of 4 shells give ranges (0, 4), (4, 6) and an empty third rank
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, align, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort(key=lambda x: x[0])
    ranges = [rg for _, rg, _ in res]
    covered = [j for j0, j1 in ranges for j in range(j0, j1)]
    assert covered == list(range(NR))  # a partition of the shells, in rank order
    O, r, w, aT, aE, K, grid, noise = _setup()
    whole = O.generate(K, noise, grid, r, w, aT, aE, FNL)
    for _, _, out in res:
        for k, v in out.items():
            assert np.max(np.abs(v - whole[k])) < 1e-12 * np.max(np.abs(whole[k])), k


def test_shell_ranges():
    from paper_0909_0009_gb300.sharded import shell_ranges
    assert shell_ranges(128, 1) == [(0, 128)]
    assert shell_ranges(128, 2) == [(0, 64), (64, 128)]
    assert shell_ranges(128, 3) == [(0, 48), (48, 88), (88, 128)]
    assert shell_ranges(128, 8) == [(16 * i, 16 * i + 16) for i in range(8)]
    assert shell_ranges(20, 4) == [(0, 8), (8, 16), (16, 20), (20, 20)]
    assert shell_ranges(5, 2, align=1) == [(0, 3), (3, 5)]
    for nr in range(1, 40):
        for world in range(1, 6):
            rg = shell_ranges(nr, world, 4)
            assert len(rg) == world and rg[0][0] == 0 and rg[-1][1] == nr
            assert all(a[1] == b[0] for a, b in zip(rg, rg[1:]))
            assert all((j0 % 4 == 0 or j0 == nr) and (j1 % 4 == 0 or j1 == nr) for j0, j1 in rg)
    with pytest.raises(ValueError):
        shell_ranges(0, 2)


def test_single_rank_runs_no_collective():
    import torch

    from paper_0909_0009_gb300 import sharded
    calls = []

    def partial(out):
        calls.append(sorted(out))
        for i, t in enumerate(out.values()):
            t.fill_(complex(i, -i))

    out = sharded.generate_sharded(partial, 5, names=("aT", "aE"))
    assert calls == [["aE", "aT"]]
    assert torch.equal(out["aE"], torch.full((5,), complex(1, -1), dtype=torch.complex128))
    out = sharded.generate_sharded(None, 3, names=("aT",))
    assert torch.count_nonzero(out["aT"]) == 0
