"""Shell-sharded realisations over the ranks of a torch.distributed process group.

The N_r shells of one configuration are split into contiguous ranges, one per rank
(`shell_ranges`).  Each rank makes the shard object of its range (fnl_make_shells_shard) and
runs fnl_generate on it; one all-reduce (sum) of the partial outputs then gives the whole
realisation on every rank.  Nothing else moves between ranks: the radial quadrature (Eq. 5)
and Eq. 3 are sums over shells, and every shard draws the noise its rows of K_l reach from the
same counter-based generator (the paper keeps the seeds so that Phi_L can be regenerated
anywhere, Sect. 3).

This module only places buffers and calls the collective; every step of the path runs in the
library's kernels.
"""
from __future__ import annotations

OUTPUTS = ("aT", "aE", "aLT", "aLE", "aNLT", "aNLE")


def shell_ranges(nr: int, world: int, align: int = 8) -> list[tuple[int, int]]:
    """Contiguous shell ranges [j0, j1), one per rank, covering 0 .. nr - 1.  Ranges are whole
    units of `align` shells (the last unit may be shorter), as even as the units allow, the
    larger ranges first; a rank left without a unit gets an empty range (j0 == j1)."""
    if nr < 1 or world < 1 or align < 1:
        raise ValueError("need nr >= 1, world >= 1 and align >= 1")
    units = (nr + align - 1) // align
    base, extra = divmod(units, world)
    out, u = [], 0
    for rank in range(world):
        n = base + (1 if rank < extra else 0)
        out.append((min(nr, u * align), min(nr, (u + n) * align)))
        u += n
    return out


def _world(group=None) -> tuple[int, int]:
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        return dist.get_rank(group), dist.get_world_size(group)
    return 0, 1


def generate_sharded(partial, nalm: int, names=OUTPUTS, device="cpu", group=None, buf=None):
    """One realisation from per-rank partial sums: `partial(out)` fills `out` (a dict of
    complex128 [nalm] tensors, one per name, all views of one buffer) with this rank's terms, or
    is None for a rank without shells (its terms are zero).  The buffer is then summed over the
    group's ranks by one all-reduce.  Returns the dict of summed outputs (views of the buffer)."""
    import torch
    if buf is None:
        buf = torch.empty((len(names), nalm), dtype=torch.complex128, device=device)
    assert buf.dtype == torch.complex128 and buf.shape == (len(names), nalm) and buf.is_contiguous()
    out = {k: buf[i] for i, k in enumerate(names)}
    if partial is None:
        buf.zero_()
    else:
        partial(out)
    rank, world = _world(group)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(torch.view_as_real(buf), op=dist.ReduceOp.SUM, group=group)
    return out


class ShardedShells:
    """The shard of this rank of an nr-shell configuration (arguments as `fnl.Shells`), and the
    realisation summed over the group's ranks.  Without an initialised process group the rank
    holds every shell and no collective runs."""

    def __init__(self, lmax, nr, ntheta, nphi, r, w, alphaT, alphaE, K=None, cov=None, mu=None, prec="fp64",
                 device=0, group=None, align=8):
        from . import fnl as F
        self.group = group
        self.rank, self.world = _world(group)
        self.range = shell_ranges(nr, self.world, align)[self.rank]
        self.nalm = (lmax + 1) * (lmax + 2) // 2
        self.device = device
        j0, j1 = self.range
        self.shells = None
        if j1 > j0:
            whole = (j0, j1) == (0, nr)
            self.shells = F.Shells(lmax, nr, ntheta, nphi, r, w, alphaT, alphaE, K=K, cov=cov, mu=mu, prec=prec,
                                   device=device, shard=None if whole else (j0, j1))

    def generate(self, seed: int, realisation: int, fnl: float, parts: bool = True, buf=None, stream=None) -> dict:
        """fnl_generate on this rank's shard, then the all-reduce of the outputs (complex128
        [nalm] each: aT, aE and, with parts, aLT, aLE, aNLT, aNLE)."""
        names = OUTPUTS if parts else OUTPUTS[:2]
        sh = self.shells

        def partial(out):
            sh.generate(seed, realisation, fnl, parts=parts, out=out, stream=stream)

        return generate_sharded(partial if sh is not None else None, self.nalm, names,
                                device=f"cuda:{self.device}", group=self.group, buf=buf)

    def close(self):
        if self.shells is not None:
            self.shells.close()
            self.shells = None
