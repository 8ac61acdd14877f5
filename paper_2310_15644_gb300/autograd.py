"""torch.autograd binding of the absorbed-power gradient.

`AbsorbedPower.apply(w, ctx, bm)` returns the absorbed power (Re xJ^H X xM, a
float64 scalar tensor) of the excitation b = bm w; the forward pass already runs
the adjoint solve, inside `bem_grad_weights` (forward solve, adjoint solve
Z^H lambda = dP/d conj(x), grad = bm^H lambda), so backward only scales the stored
gradient.  Argument marshalling only: every step runs in the library.
"""
from __future__ import annotations

import torch

from . import bem as B


class AbsorbedPower(torch.autograd.Function):
    @staticmethod
    def forward(ctx, w, handle, bm):
        """w: complex128 (nw,) weights (any device); handle: assembled bem context;
        bm: device complex128 (nw, 2ne) contiguous -- row i is the right-hand side of
        excitation i (the library's column-major 2ne x nw)."""
        if bm.dtype != torch.complex128 or not bm.is_cuda or not bm.is_contiguous():
            raise ValueError("bm must be a contiguous complex128 CUDA tensor")
        stream = torch.cuda.current_stream(bm.device).cuda_stream
        p, grad, _ = B.bem_grad_weights(handle, bm.data_ptr(), w.detach().cpu().numpy(), stream=stream)
        ctx.save_for_backward(torch.from_numpy(grad).to(w.device))
        return torch.tensor(p, dtype=torch.float64, device=w.device)

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        # PyTorch's gradient of a real loss with respect to complex w is
        # dL/d Re w + j dL/d Im w = 2 dL/d conj(w)
        return 2.0 * grad_out * g, None, None


def absorbed_power(w, handle, bm):
    return AbsorbedPower.apply(w, handle, bm)
