"""Differentiable discrete electrostatic energy.

``energy(handle, x, q, phi_b)`` returns U (a float64 scalar tensor) of the
particle-mesh problem of Sec. II.B.1; ``U.backward()`` runs the library's
hand-written adjoint (discos_energy_backward): interpolation for the charge
spreading, gradient-kernel interpolation for the positions and the lift
profile for the wall potentials.  Nothing is saved between the two passes
but the inputs: the backward re-spreads and re-solves.
"""
import torch


class DiscreteEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, q, phi_b, handle):
        ctx.handle = handle
        ctx.save_for_backward(x, q, phi_b)
        return handle.energy(x.contiguous(), q.contiguous(), phi_b=phi_b.detach())

    @staticmethod
    def backward(ctx, gU):
        x, q, phi_b = ctx.saved_tensors
        h = ctx.handle
        need = ctx.needs_input_grad[:3]
        dx, dq, db = h.energy_backward(x.contiguous(), q.contiguous(), gU, phi_b=phi_b.detach(), need=need)
        if db is not None:
            db = db.to(device=phi_b.device, dtype=phi_b.dtype)
        return dx, dq, db, None


def energy(handle, x, q, phi_b=None):
    """U(x, q, phi_b); phi_b defaults to the handle's configured wall potentials."""
    if phi_b is None:
        phi_b = torch.tensor(list(handle.cfg.phi_b), dtype=torch.float64)
    return DiscreteEnergy.apply(x, q, phi_b, handle)
