"""torch.autograd.Function wrappers around the C ABI (argument marshalling only).

* ``MTPEnergy``: per-configuration energies E_k (eq. 1) as a function of the atomic
  positions and of the parameter vector theta.  Its backward pass is one library call,
  mtp_energy_vjp, on the hand-written adjoint kernels: dE_k/dx_i = -F_i for atoms i of
  configuration k (forces from the same call as the energies), and
  dE_k/dtheta = sum_{i in k} b_i with b_i = dV_i/dtheta (eq. 9), contracted with the cotangent
  in the library.
* ``MTPLoss``: the energy/force/stress loss of eq. 7 as a function of theta; its backward
  returns the gradient that mtp_train_step computes (second hand-written kernel).

Positions enter through the batch struct: the forward pass points the batch at the given
position tensor and rebuilds the neighbor list, so a changed position tensor is always seen.
Theta enters through mtp_set_params (host copy of m doubles).
"""
from __future__ import annotations

import torch

from . import api


def _set_theta(model, theta: torch.Tensor):
    api.mtp_set_params(model, theta.detach().to("cpu", torch.float64).numpy())


class MTPEnergy(torch.autograd.Function):
    """E = MTPEnergy.apply(pos, theta, model, batch, prec) -> (n_cfg,) float64.

    ``pos``: (N, 3) float64 CUDA tensor (the batch's positions are replaced by it);
    ``theta``: (m,) float64 tensor (loaded into the model before evaluation).
    The neighbor list is rebuilt inside every forward call."""

    @staticmethod
    def forward(ctx, pos, theta, model, batch, prec="fp64"):
        pos = pos.detach().to(device="cuda", dtype=torch.float64).contiguous()
        if pos.shape != (batch.n_atoms, 3):
            raise ValueError(f"positions must be ({batch.n_atoms}, 3)")
        _set_theta(model, theta)
        batch.pos = pos
        batch.refresh()
        nbr = api.mtp_build_neighbors(model, batch)
        out = api.mtp_energy_forces_stress(model, batch, nbr, prec, want=("energy", "forces"))
        ctx.model, ctx.batch, ctx.nbr, ctx.prec = model, batch, nbr, prec
        ctx.theta_device = theta.device
        ctx.save_for_backward(out["forces"])
        return out["energy"]

    @staticmethod
    def backward(ctx, gE):
        (F,) = ctx.saved_tensors
        g_pos, g_theta = api.mtp_energy_vjp(ctx.model, ctx.batch, ctx.nbr, gE, F, want_pos=ctx.needs_input_grad[0],
                                            want_theta=ctx.needs_input_grad[1], prec=ctx.prec)
        if g_theta is not None:
            g_theta = g_theta.to(ctx.theta_device)
        return g_pos, g_theta, None, None, None


class MTPLoss(torch.autograd.Function):
    """L = MTPLoss.apply(theta, model, batch, nbr, E_ref, F_ref, W_ref, w_e, w_f, w_s, prec).

    Returns the scalar loss of eq. 7 (float64, 0-dim); backward gives dL/dtheta."""

    @staticmethod
    def forward(ctx, theta, model, batch, nbr, E_ref, F_ref, W_ref=None, w_e=1.0, w_f=0.01, w_s=0.0,
                prec="fp64"):
        _set_theta(model, theta)
        loss, grad = api.mtp_train_step(model, batch, nbr, E_ref, F_ref, W_ref, w_e, w_f, w_s, prec)
        ctx.save_for_backward(grad.to(theta.device))
        return loss.reshape(()).to(theta.device)

    @staticmethod
    def backward(ctx, gL):
        (grad,) = ctx.saved_tensors
        return (gL * grad,) + (None,) * 10


def energy(pos, theta, model, batch, prec="fp64"):
    return MTPEnergy.apply(pos, theta, model, batch, prec)


def loss(theta, model, batch, nbr, E_ref, F_ref, W_ref=None, w_e=1.0, w_f=0.01, w_s=0.0, prec="fp64"):
    return MTPLoss.apply(theta, model, batch, nbr, E_ref, F_ref, W_ref, w_e, w_f, w_s, prec)
