"""The registration energy as a differentiable PyTorch function.

``registration_energy(vt, plan)`` returns E(v~) of Eq. 35 (a float64 scalar on the
device) computed by the library's forward solve (``blr_state``); its backward is
the library's adjoint kernel chain (``blr_gradient_at_state``: adjoint sweeps with
the body force, projection pi and the regulariser term of Eq. 38), so
``E.backward()`` leaves dE/dv~ in ``vt.grad``.  With a plan created with
``ckpt_every=k`` the forward keeps only every k-th state and the backward
recomputes each segment from its checkpoint.  Any plan form works (the
incompressible, non-stationary and deformation-state variants): the backward
is the plan's own gradient at its current point.

Gradients of complex coefficients follow PyTorch's convention for a real loss:
grad = dE/d(Re v~) + i dE/d(Im v~), which is exactly g~ of Eq. 38 under the inner
product <a, b> = Re sum a conj(b).
"""

from __future__ import annotations

import torch


class RegistrationEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vt, plan):
        want = (3,) + tuple(plan.band)
        if plan.params.nonstationary:
            want = (plan.nt,) + want
        if vt.dtype != torch.complex64 or not vt.is_cuda or tuple(vt.shape) != want:
            raise ValueError(f"vt must be a complex64 CUDA tensor of the plan's coefficient "
                             f"shape {want} ((3, B1, B2, B3), or (nt, 3, B1, B2, B3) for a "
                             f"non-stationary plan); got {tuple(vt.shape)} {vt.dtype} on {vt.device}")
        vt = vt.contiguous()
        energy = torch.empty(3, dtype=torch.float64, device=vt.device)
        plan.state(vt, energy=energy)
        ctx.plan = plan
        ctx.point = plan.point
        ctx.save_for_backward(vt)
        return energy[0].clone()

    @staticmethod
    def backward(ctx, grad_energy):
        (vt,) = ctx.saved_tensors
        plan = ctx.plan
        if plan.point != ctx.point:
            # another forward solve moved the plan's current point: redo this one
            plan.state(vt)
        g = torch.empty_like(vt)
        plan.gradient_at_state(g)
        return g * grad_energy.to(torch.float32), None


def registration_energy(vt: torch.Tensor, plan) -> torch.Tensor:
    """E(v~) = 1/2 <L~v~, v~> + sigma^-2 ||m(1) - I1||^2 with a hand-written backward."""
    return RegistrationEnergy.apply(vt, plan)
