"""PyTorch autograd over the C ABI (differentiation extension).

``Energy.apply(m, prob, Hext)`` returns the total energy U(m) (J) of
``mm_energy``; its backward is the library's field kernel through
``mm_energy_gradient`` (dU/dm = -mu0 Ms V H_eff).  ``dmx_dK`` is the implicit
adjoint of <m_x> with respect to the per-cell anisotropy at a converged
minimum (``mm_adjoint_dK``).  Only argument marshalling happens here.
"""
import numpy as np
import torch

from . import mm


class Energy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, m, prob, Hext):
        E = mm.mm_energy(prob, m.detach().contiguous(), Hext)
        ctx.save_for_backward(m)
        ctx.prob, ctx.Hext = prob, Hext
        return torch.tensor(E[4], dtype=torch.float64, device=m.device)

    @staticmethod
    def backward(ctx, grad_out):
        (m,) = ctx.saved_tensors
        G = torch.empty_like(m)
        mm.mm_energy_gradient(ctx.prob, m.detach().contiguous(), ctx.Hext, G, scale=float(grad_out))
        return G, None, None


def dmx_dK(prob, m, Hext, tol=1e-10, max_iter=20000):
    """d<m_x>/dK_i at a converged minimum m (device tensor); returns (dJdK, status, iterations)."""
    dJdm = torch.zeros_like(m)
    n = m[0].numel()
    dJdm[0].fill_(1.0 / n)
    out = torch.empty(m.shape[1:], dtype=torch.float64, device=m.device)
    st, it, _ = mm.mm_adjoint_dK(prob, m, Hext, dJdm, out, tol=tol, max_iter=max_iter)
    return out, st, it
