"""torch.autograd.Function over the C ABI: D = forward(R, m, S_age); backward = the
hand-written straight-through adjoint (App. B of the paper: gradients through the
unrolled day loop, with the Gumbel-softmax relaxation of the infection draw)."""
from __future__ import annotations

import torch

from . import capi


class GabmFunction(torch.autograd.Function):
    """``GabmFunction.apply(ctx, R, m, S_age, n_seed) -> D``.

    R, m: [I, T] float32 CUDA tensors; S_age: [I, 9] float32; n_seed: ints per instance.
    D: [I, T] float64 daily new deaths.  The backward runs ``gabm_backward`` on the
    same ctx, so a ctx serves one forward/backward pair at a time.
    """

    @staticmethod
    def forward(fctx, handle, R, m, S_age, n_seed):
        T = int(R.shape[-1])
        D, _ = capi.gabm_forward(handle, T, R.detach().contiguous(), m.detach().contiguous(),
                                 S_age.detach().contiguous(), n_seed)
        fctx.handle = handle
        fctx.dtypes = (R.dtype, m.dtype, S_age.dtype)
        return D

    @staticmethod
    def backward(fctx, gD):
        dR, dm, dS = capi.gabm_backward(fctx.handle, gD.detach().to(torch.float64).contiguous())
        return None, dR.to(fctx.dtypes[0]), dm.to(fctx.dtypes[1]), dS.to(fctx.dtypes[2]), None
