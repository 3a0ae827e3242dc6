"""torch.autograd.Function over the library's forward transform and its
hand-written gradient (paper Methods: gradients of the complex farfield
weights propagated forward and backward through the transform).

    E = spot_field(holo, phase, coeff)      # complex64 (N,)

Backward takes torch's complex gradient convention, grad_E = dL/dRe E +
i dL/dIm E, and returns dL/dphase (adjoint pass, ash_grad) and dL/dC (moment
pass with the spot tiles recomputed, ash_grad); nothing of the forward is
stored besides (phase, coeff).
"""
from __future__ import annotations

import torch

from .hologram import Hologram, spot_loss

__all__ = ["SpotField", "SpotIntensityLoss", "spot_field", "spot_intensity_loss"]


class SpotField(torch.autograd.Function):
    @staticmethod
    def forward(ctx, phase: torch.Tensor, coeff: torch.Tensor, holo: Hologram) -> torch.Tensor:
        phase = phase.detach().contiguous()
        coeff = coeff.detach().contiguous()
        E = holo.forward_coeff(coeff, phase)   # sets C and runs the forward in one call
        ctx.save_for_backward(phase, coeff)
        ctx.holo = holo
        ctx.epoch = holo.coeff_epoch
        return E

    @staticmethod
    def backward(ctx, grad_E: torch.Tensor):
        phase, coeff = ctx.saved_tensors
        holo: Hologram = ctx.holo
        want_phase, want_coeff = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        if not (want_phase or want_coeff):
            return None, None, None
        if holo.coeff_epoch != ctx.epoch:
            # the handle was given other coefficients since this forward
            # (an in-place change of `coeff` itself fails autograd's check)
            holo.set_coefficients(coeff)
        dphase, dcoeff = holo.grad(phase, grad_E.contiguous(), want_phase=want_phase, want_coeff=want_coeff)
        return dphase, dcoeff, None


def spot_field(holo: Hologram, phase: torch.Tensor, coeff: torch.Tensor | None = None) -> torch.Tensor:
    """E_n = sum_m A_m exp(i phase_m) exp(-i coeff_n . Z_m), differentiable in
    phase and coeff. `coeff` defaults to the handle's current coefficients
    (then no gradient flows to them)."""
    if coeff is None:
        coeff = holo.coefficients()
    return SpotField.apply(phase, coeff, holo)


class SpotIntensityLoss(torch.autograd.Function):
    """L = sum_n (|E_n|^2 / mean|E|^2 - t_n)^2 with its gradient dL/dE from
    the same library kernel (ash_spot_loss); backward scales it."""

    @staticmethod
    def forward(ctx, E: torch.Tensor, t: torch.Tensor) -> torch.Tensor:
        loss, g = spot_loss(E.detach().contiguous(), t.detach().contiguous(), want_grad=ctx.needs_input_grad[0])
        ctx.save_for_backward(g if g is not None else loss)
        return loss

    @staticmethod
    def backward(ctx, grad_L: torch.Tensor):
        if not ctx.needs_input_grad[0]:
            return None, None
        (g,) = ctx.saved_tensors
        return g * grad_L, None


def spot_intensity_loss(E: torch.Tensor, t: torch.Tensor) -> torch.Tensor:
    """L = sum_n (|E_n|^2 / mean|E|^2 - t_n)^2, differentiable in E (the loss
    and its gradient in one library kernel)."""
    return SpotIntensityLoss.apply(E, t)
