"""Weighted Gerchberg-Saxton on the compressed spot transform (oracle).

Paper: Sec. II reduces spot holography to choosing the N complex farfield
weights F_n, solved iteratively as in GS (nearfield and farfield amplitudes
are corrected to the source and target until |F| converges to |G|);
Sec. III uses weighted GS (citing Kim et al. 2019) for the tweezer arrays.
The paper does not print the weighting rule. Reading used here (classic
weighted GS, scale-invariant form, feedback exponent 1, no phase fixing):

  init   w = T (target amplitudes), phase phi^0 given, T^ = T / ||T||_2
  repeat `iters` times:
     f   = A exp(i phi)                       (source amplitude constraint)
     E   = K f                                (forward transform)
     E^  = |E| / ||E||_2
     w   = w * T^ / max(E^, 1e-30);  w = w / ||w||_2
     psi = arg E
     g   = K^H (w exp(i psi))                 (adjoint transform)
     phi = arg g   (0 where g == 0 exactly)
  finally E = K (A exp(i phi)) is the reported field.

Variants (the paper only cites Kim et al. for its WGS): the weight
update with a feedback exponent p, w = w * (T^ / max(E^, 1e-30))^p (p = 1
above; p = 0 keeps w = T^, plain GS), and phase fixing, where psi is held
at given values instead of arg E.

Metrics (the paper reports camera Strehl instead; these are the readings):
  uniformity U = 1 - (max I^ - min I^)/(max I^ + min I^), I^_n = |E_n|^2 / T_n^2
  efficiency eta = sum_n |E_n|^2 / (M sum_m A_m^2)
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import transform


@dataclasses.dataclass
class WGSResult:
    phase: np.ndarray     # (M,) float64, final SLM phase
    weights: np.ndarray   # (N,) float64, final spot weights w
    E: np.ndarray         # (N,) complex128, field of the final phase
    uniformity: float
    efficiency: float
    history: list         # per-iteration uniformity of the forward inside the loop
    psi: np.ndarray = None  # (N,) spot phases used by the last update


def uniformity(E: np.ndarray, target: np.ndarray) -> float:
    I = np.abs(E) ** 2 / np.asarray(target, np.float64) ** 2
    hi, lo = float(I.max()), float(I.min())
    return 1.0 - (hi - lo) / (hi + lo) if hi + lo > 0 else 0.0


def efficiency(E: np.ndarray, amp: np.ndarray) -> float:
    a = np.asarray(amp, np.float64).ravel()
    return float(np.sum(np.abs(E) ** 2) / (a.size * np.sum(a * a)))


def weight_update(E: np.ndarray, w: np.ndarray, target: np.ndarray, feedback: float = 1.0, psi=None):
    """One spot-side update: returns (new w, y = w exp(i psi)).

    w <- w (T^/E^)^feedback, renormalised (feedback 1 is the plain weighted
    GS rule, 0 plain GS with the target amplitudes); psi = arg E unless a
    held phase `psi` is given (phase fixing, after Kim et al.)."""
    t = np.asarray(target, np.float64)
    t_hat = t / np.linalg.norm(t)
    a = np.abs(E)
    nrm = np.linalg.norm(a)
    e_hat = a / nrm if nrm > 0 else a
    w = w * (t_hat / np.maximum(e_hat, 1e-30)) ** feedback
    w = w / np.linalg.norm(w)
    if psi is None:
        psi = transform.phase_of(E)
    return w, w * np.exp(1j * psi)


def run(amp, phase0, C, Z, target, iters: int, weights0=None, workers: int = 1, feedback: float = 1.0,
        fixed_psi=None) -> WGSResult:
    """`iters` WGS iterations and a final forward. `fixed_psi`: hold the spot
    phases at these values (phase fixing); otherwise psi = arg E each time.
    The result's `psi` is the spot phase of the last update."""
    amp = np.asarray(amp, np.float64).ravel()
    phase = np.asarray(phase0, np.float64).ravel().copy()
    w = np.asarray(target if weights0 is None else weights0, np.float64).copy()
    hist = []
    psi = None if fixed_psi is None else np.asarray(fixed_psi, np.float64)
    for _ in range(iters):
        E = transform.forward(transform.field(amp, phase), C, Z, workers=workers)
        hist.append(uniformity(E, target))
        if fixed_psi is None:
            psi = transform.phase_of(E)
        w, y = weight_update(E, w, target, feedback, psi)
        g = transform.adjoint(y, C, Z, workers=workers)
        phase = transform.phase_of(g)
    E = transform.forward(transform.field(amp, phase), C, Z, workers=workers)
    return WGSResult(phase, w, E, uniformity(E, target), efficiency(E, amp), hist, psi)
