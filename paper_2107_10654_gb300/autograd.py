"""torch.autograd.Function for the sketched core solve with a frozen sketch.

Forward calls tucker_core_update_sketched with a fixed sample; backward calls
tucker_core_solve_adjoint, which reuses the cached Cholesky factor of the
forward solve for the transposed solve and scatter-adds the Kronecker-row
gradients into dA^(n) in CUDA.  The sample (keys, counts, probabilities) is a
constant of differentiation: it is discrete.
"""
from __future__ import annotations

import torch

from . import tucker as T


class SketchedCoreSolve(torch.autograd.Function):
    """g = SketchedCoreSolve.apply(handle, X, samples, lam, reg, prec, A_1, ..., A_N).

    X is a dense CUDA tensor or a CooTensor; the gradient w.r.t. X is returned
    for a dense X (non-zero only at the sampled entries) and is None for COO.
    """

    @staticmethod
    def forward(ctx, handle, X, samples, lam, reg, prec, *A):
        core, st = T.tucker_core_update_sketched(handle, X, list(A), lam, 0, 0, 0, reg, prec,
                                                 fixed=samples, stats=True)
        ctx.handle, ctx.X, ctx.samples = handle, X, samples
        ctx.lam, ctx.reg, ctx.prec = lam, reg, prec
        ctx.solve_id = st["solve_id"]
        ctx.save_for_backward(core, *A)
        return core

    @staticmethod
    def backward(ctx, gbar):
        core, *A = ctx.saved_tensors
        dA, dx = T.tucker_core_solve_adjoint(ctx.handle, ctx.X, A, ctx.lam, ctx.reg, ctx.prec,
                                             ctx.samples, ctx.solve_id, core,
                                             gbar.contiguous().to(torch.float64))
        dX = None
        if isinstance(ctx.X, torch.Tensor) and ctx.needs_input_grad[1]:
            total = ctx.X.numel()
            keys = ctx.samples.keys[:ctx.samples.n_unique]
            real = keys < total
            dX = torch.zeros(total, dtype=torch.float64, device=ctx.X.device)
            dX[keys[real]] = dx[real]
            dX = dX.view(ctx.X.shape).to(ctx.X.dtype)
        grads = [g.to(a.dtype) for g, a in zip(dA, A)]
        return (None, dX, None, None, None, None, *grads)
