"""PyTorch autograd wrapper of the receiver misfit (hz_grad).

``misfit(m, solver, src, rec, d)`` returns Phi(m) as a 0-d tensor whose
backward gives dPhi/dm from the adjoint-state gradient computed on the device
in the same call (one forward and one adjoint GMRES solve per batch of
sources).  Each call loads ``m`` into the solver and refactors the slabs.
"""

from __future__ import annotations

import torch


class _Misfit(torch.autograd.Function):
    @staticmethod
    def forward(ctx, m, solver, src, rec, d):
        solver.set_medium(m.detach())
        solver.factor()
        phi, grad, _ = solver.grad(src, rec, d)
        ctx.save_for_backward(grad.to(m.dtype))
        return torch.tensor(phi, dtype=m.dtype, device=m.device)

    @staticmethod
    def backward(ctx, grad_out):
        (grad,) = ctx.saved_tensors
        return grad_out * grad, None, None, None, None


def misfit(m: torch.Tensor, solver, src, rec, d) -> torch.Tensor:
    """Phi(m) = 1/2 sum |u_s(rec) - d_s|^2 with a gradient in m (see hz_grad)."""
    return _Misfit.apply(m, solver, src, rec, d)
