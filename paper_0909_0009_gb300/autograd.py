"""torch.autograd binding of the generator and its hand-written adjoint.

``generate(shells, noise, fnl, seed, realisation)`` returns (a^T, a^E) as complex128
tensors and records a node whose backward calls ``fnl_generate_backward``: dL/dn for the
white noise n_lm(r_j) of Eq. 9 and dL/df_NL for the f_NL of Eq. 3, for field-level
inference.  The backward recomputes the per-shell maps on the ring grid instead of storing
them; it keeps only a^T_NL and a^E_NL of the forward call (2 nalm complex numbers).

PyTorch's gradient of a real loss with respect to a complex tensor is dL/dRe + i dL/dIm,
which is exactly the pair layout the C ABI takes and returns, so no conversion is done.
The imaginary part of every m = 0 noise entry is ignored by the forward and gets a zero
gradient.  Every precision form has an adjoint; the tensor-core forms run it on their
tcgen05 GEMMs (HEALPix objects raise).
"""
from __future__ import annotations

import torch

from . import fnl as _fnl


class _Generate(torch.autograd.Function):
    @staticmethod
    def forward(ctx, noise, fnl, shells, seed, realisation):
        f = float(fnl)
        out = shells.generate(seed, realisation, f, noise=noise, parts=True)
        ctx.shells, ctx.seed, ctx.realisation, ctx.f = shells, seed, realisation, f
        ctx.fnl_meta = (fnl.dtype, fnl.device) if isinstance(fnl, torch.Tensor) else None
        ctx.save_for_backward(noise if noise is not None else torch.empty(0), out["aNLT"], out["aNLE"])
        ctx.has_noise = noise is not None
        return out["aT"], out["aE"]

    @staticmethod
    def backward(ctx, gT, gE):
        noise, aNLT, aNLE = ctx.saved_tensors
        want_noise = ctx.has_noise and ctx.needs_input_grad[0]
        want_fnl = ctx.fnl_meta is not None and ctx.needs_input_grad[1]
        if not (want_noise or want_fnl):
            return None, None, None, None, None
        gT = None if gT is None else gT.contiguous()
        gE = None if gE is None else gE.contiguous()
        gn, gf = ctx.shells.generate_backward(ctx.seed, ctx.realisation, ctx.f, gT=gT, gE=gE,
                                              noise=noise if ctx.has_noise else None, aNLT=aNLT, aNLE=aNLE,
                                              want_noise=want_noise, want_fnl=want_fnl)
        if gf is not None:
            dtype, device = ctx.fnl_meta
            gf = gf.to(dtype=dtype, device=device)
        return gn, gf, None, None, None


def generate(shells: "_fnl.Shells", noise: torch.Tensor | None, fnl, seed: int = 0, realisation: int = 0):
    """Differentiable realisation: (a^T, a^E), complex128 [nalm] each.

    noise: complex128 [nr, nalm] device tensor (differentiable), or None for the Philox draw
    of (seed, realisation) (then only f_NL is differentiable).  fnl: a float or a 0-d tensor
    (differentiable when it requires grad)."""
    return _Generate.apply(noise, fnl, shells, int(seed), int(realisation))


__all__ = ["generate"]
