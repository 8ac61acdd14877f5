"""torch.autograd binding of the absorbed-power gradients.

`absorbed_power(w, handle, bm)` returns the absorbed power (Re xJ^H X xM, a float64
scalar tensor) of the excitation b = bm w.  With `eps` (a float64 tensor
[Re eps_r, Im eps_r]) and `k0`, the interior permittivity is an input too: the
context is re-assembled when eps changes, and eps gets its gradient from
`bem_grad_eps` (single body; on a layered context, set up with bem_set_regions,
only the weights are inputs).  The forward pass already runs the adjoint solve, inside
`bem_grad_weights` (forward solve, adjoint solve Z^H lambda = dP/d conj(x),
grad = bm^H lambda), so backward only scales stored gradients.  Argument
marshalling only: every step runs in the library.
"""
from __future__ import annotations

import torch

from . import bem as B

_media = {}  # context handle -> (k0, eps_r) it was last assembled with here


class AbsorbedPower(torch.autograd.Function):
    @staticmethod
    def forward(ctx, w, eps, handle, bm, k0):
        """w: complex128 (nw,) weights; eps: float64 (2,) [Re, Im] of eps_r, or None;
        handle: bem context with its mesh set; bm: device complex128 (nw, 2ne)
        contiguous, row i the right-hand side of excitation i (the library's
        column-major 2ne x nw); k0: exterior wavenumber (with eps)."""
        if bm.dtype != torch.complex128 or not bm.is_cuda or not bm.is_contiguous():
            raise ValueError("bm must be a contiguous complex128 CUDA tensor")
        stream = torch.cuda.current_stream(bm.device).cuda_stream
        key = handle.value if hasattr(handle, "value") else int(handle)
        if eps is not None:
            e = complex(float(eps[0]), float(eps[1]))
            if _media.get(key) != (float(k0), e):
                B.bem_set_media(handle, float(k0), e)
                B.bem_assemble(handle, stream)
                _media[key] = (float(k0), e)
        n = bm.shape[1]
        x = torch.empty(n, dtype=torch.complex128, device=bm.device)
        lam = torch.empty_like(x)
        p, grad, _ = B.bem_grad_weights(handle, bm.data_ptr(), w.detach().cpu().numpy(), x.data_ptr(),
                                        lam.data_ptr(), stream=stream)
        deps = B.bem_grad_eps(handle, x.data_ptr(), lam.data_ptr(), stream=stream) if eps is not None else None
        ctx.save_for_backward(torch.from_numpy(grad).to(w.device),
                              torch.from_numpy(deps) if deps is not None else torch.zeros(2, dtype=torch.float64))
        ctx.has_eps = eps is not None
        ctx.eps_device = eps.device if eps is not None else None
        return torch.tensor(p, dtype=torch.float64, device=w.device)

    @staticmethod
    def backward(ctx, grad_out):
        g, deps = ctx.saved_tensors
        # PyTorch's gradient of a real loss with respect to complex w is
        # dL/d Re w + j dL/d Im w = 2 dL/d conj(w)
        gw = 2.0 * grad_out * g
        ge = (grad_out.cpu() * deps).to(ctx.eps_device) if ctx.has_eps else None
        return gw, ge, None, None, None


def absorbed_power(w, handle, bm, eps=None, k0=None):
    """See the module docstring.  The re-assembly cache is keyed by the context: a
    context whose media are changed outside this function must not be reused here."""
    if eps is not None and k0 is None:
        raise ValueError("k0 is needed with eps")
    if eps is not None and B.bem_num_regions(handle) > 2:
        raise ValueError("eps as an input needs a single-body context; a layered context gets "
                         "one permittivity gradient per region from bem_grad_eps")
    return AbsorbedPower.apply(w, eps, handle, bm, k0)
