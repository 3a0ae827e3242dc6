"""Conjugate-gradient refinement of the SLM phase (oracle).

Paper, Methods (end of "Computational Scaling"): precision targets such as
very uniform top hats are better refined by conjugate-gradient descent than
by weighted GS, with the gradients propagated forward and backward through
the transform. The paper prints no algorithm. Reading used here: nonlinear
conjugate gradients with the Polak-Ribiere coefficient and its non-negative
restart (PR+, Nocedal & Wright, Numerical Optimization, Sec. 5.2), and a
line search of one trial step with a quadratic fit:

  g_0 = dL/dphi(phi_0) (grad.py's loss and closed-form gradient), d_0 = -g_0
  iteration k:
     s  = g_k . d_k; if s >= 0: d_k = -g_k, s = -g_k . g_k      (restart)
     a0 = theta / max_m |d_k,m|     (the trial changes no phase by more than theta)
     L1 = L(phi_k + a0 d_k)
     c  = (L1 - L_k - s a0) / a0^2   (curvature of the quadratic through
                                      L_k, slope s and L1)
     a  = -s / (2 c) if c > 0 else 2 a0
     phi_{k+1} = phi_k + a d_k;  L_{k+1}, g_{k+1} at phi_{k+1}
     beta = max(0, g_{k+1} . (g_{k+1} - g_k) / (g_k . g_k))
     d_{k+1} = -g_{k+1} + beta d_k
  (a zero gradient stops the descent: a0 = a = 0)

On a quadratic the fit is exact, so the line search is exact and the
iteration is linear CG, which minimises an n-dimensional quadratic in n
steps (the CPU pin).
"""
from __future__ import annotations

import numpy as np

from . import grad, transform


def minimize(fun, fun_grad, x0, iters: int, theta: float):
    """Generic form: fun(x) -> L, fun_grad(x) -> (L, g). Returns (x, [L_0..L_iters])."""
    x = np.array(x0, np.float64, copy=True)
    L, g = fun_grad(x)
    d = -g
    losses = [L]
    for _ in range(iters):
        s = float(g @ d)
        if s >= 0:
            d = -g
            s = -float(g @ g)
        mx = float(np.max(np.abs(d))) if d.size else 0.0
        if mx == 0.0:
            losses.append(L)
            continue
        a0 = theta / mx
        L1 = fun(x + a0 * d)
        c = (L1 - L - s * a0) / (a0 * a0)
        a = -s / (2.0 * c) if c > 0 else 2.0 * a0
        x = x + a * d
        g_old = g
        L, g = fun_grad(x)
        beta = max(0.0, float(g @ (g - g_old)) / float(g_old @ g_old))
        d = -g + beta * d
        losses.append(L)
    return x, losses


def loss_and_phase_grad(amp, phase, C, Z, t, workers: int = 1):
    """(L, dL/dphi) at `phase` (no coefficient gradient)."""
    f = transform.field(amp, phase)
    E = transform.forward(f, C, Z, workers=workers)
    h = transform.adjoint(grad.grad_E(E, t), C, Z, workers=workers)
    return grad.loss_from_E(E, t), -np.imag(f * np.conj(h))


def refine(amp, phase0, C, Z, t, iters: int, theta: float = 0.05, workers: int = 1):
    """`iters` CG iterations on phi for the spot-intensity loss with targets t."""
    amp = np.asarray(amp, np.float64).ravel()

    def fun(ph):
        return grad.loss_from_E(transform.forward(transform.field(amp, ph), C, Z, workers=workers), t)

    def fun_grad(ph):
        return loss_and_phase_grad(amp, ph, C, Z, t, workers)

    return minimize(fun, fun_grad, np.asarray(phase0, np.float64).ravel(), iters, theta)
