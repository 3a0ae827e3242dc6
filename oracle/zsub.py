"""Simulated Zernike-subtraction calibration (oracle).

Paper, Sec. III (Fig. 2b and the calibration text): starting from a baseline
hologram aimed at the target points, one Zernike order Z_d at a time is
superimposed on the SLM with a global amplitude that is swept; a per-spot
figure of merit read at every sweep value gives the local contribution of
that order at each site, which aberration-space holography then subtracts
spot by spot; repeating over the orders up to D converges to a spot array
that cancels the local aberration.

The paper runs this on hardware. Here the optical system is synthetic: a
coefficient matrix C_sys (N x D) is the "true" kernel matrix of the system,
and the model's matrix C_model is what the hologram is computed from.
Readings where the paper is silent:

  baseline  phi = arg K_model^H T (superposition of the target spots'
            kernels with amplitudes T), or `iters` weighted-GS iterations
            on the model (wgs.run) when iters > 0.
  sweep     for every offset delta_k, the SLM phase phi + delta_k Z_d is
            propagated through the system: I_n(delta_k) = |E_n|^2 with
            E = K_sys (A exp(i (phi + delta_k Z_d))). The figure of merit is
            the spot's peak intensity (a relative Strehl ratio).
  estimate  per spot, a least-squares parabola through (delta_k,
            ln max(I_n(delta_k), 1e-37)) -- a Gaussian peak -- and its
            vertex -b / (2 c), clipped to [min delta, max delta]; if the
            fitted curvature c is not negative, the offset of the largest
            sample (the first one on ties).
  update    C_model[n, d] += delta*_n. Since exp(i delta Z_d) exp(-i C Z)
            = exp(-i (C - delta e_d) Z), the spot is brightest when
            C_sys[n, d] - delta = C_model[n, d], so delta* estimates the
            model's error in that order and adding it subtracts it.
  loop      `rounds` passes over `modes` in the given order, the baseline
            hologram recomputed from the current model before every sweep;
            round r sweeps the offsets times shrink^r (shrink = 1: the same
            sweep every round).
"""
from __future__ import annotations

import numpy as np

from . import transform, wgs

TINY = 1e-37


def baseline_phase(amp, C_model, Z, target, iters: int = 0, phase0=None, workers: int = 1) -> np.ndarray:
    """Hologram aimed at the target points through the model's kernels."""
    if iters <= 0:
        g = transform.adjoint(np.asarray(target, np.float64).astype(np.complex128), C_model, Z, workers=workers)
        return np.where(g == 0, 0.0, np.angle(g))
    if phase0 is None:
        phase0 = np.zeros(np.asarray(amp).size)
    return wgs.run(amp, phase0, C_model, Z, target, iters, workers=workers).phase


def sweep(amp, phase, C_sys, Z, mode: int, deltas, workers: int = 1) -> np.ndarray:
    """I[k, n] = |E_n|^2 for the SLM phase phase + deltas[k] Z[mode] through C_sys."""
    phase = np.asarray(phase, np.float64).ravel()
    Z = np.asarray(Z, np.float64)
    out = []
    for dk in np.asarray(deltas, np.float64):
        E = transform.forward(transform.field(amp, phase + dk * Z[mode]), C_sys, Z, workers=workers)
        out.append(np.abs(E) ** 2)
    return np.array(out)


def wavefront_residual(amp, C_model, C_sys, Z) -> float:
    """RMS over spots of the model's phase error (C_model - C_sys) . Z_m
    about its mean, weighted by the SLM intensity A_m^2: what a
    calibration removes (combinations of orders that cancel where the beam
    is are invisible to any spot measurement)."""
    w = np.asarray(amp, np.float64).ravel() ** 2
    w = w / w.sum()
    W = (np.asarray(C_model, np.float64) - np.asarray(C_sys, np.float64)) @ np.asarray(Z, np.float64)
    mu = W @ w
    return float(np.sqrt(np.mean(((W - mu[:, None]) ** 2) @ w)))


def estimate(I, deltas) -> np.ndarray:
    """Per-spot vertex of the least-squares parabola through (delta, ln I)."""
    d = np.asarray(deltas, np.float64)
    L = np.log(np.maximum(np.asarray(I, np.float64), TINY))          # (K, N)
    X = np.stack([np.ones_like(d), d, d * d], axis=1)                  # (K, 3)
    coef = np.linalg.lstsq(X, L, rcond=None)[0]                        # (3, N)
    b, c = coef[1], coef[2]
    out = np.empty(L.shape[1])
    for n in range(L.shape[1]):
        if c[n] < 0:
            out[n] = min(max(-b[n] / (2.0 * c[n]), d.min()), d.max())
        else:
            out[n] = d[int(np.argmax(L[:, n]))]
    return out


def calibrate(amp, C_model0, C_sys, Z, target, modes, deltas, rounds: int = 1, iters: int = 0, shrink: float = 1.0,
              workers: int = 1):
    """The loop: returns the final model matrix and the per-step estimates."""
    C = np.array(C_model0, np.float64, copy=True)
    steps = []
    for r in range(rounds):
        dr = np.asarray(deltas, np.float64) * shrink ** r
        for d in modes:
            phi = baseline_phase(amp, C, Z, target, iters, workers=workers)
            I = sweep(amp, phi, C_sys, Z, d, dr, workers=workers)
            ds = estimate(I, dr)
            C[:, d] += ds
            steps.append((d, ds))
    return C, steps
