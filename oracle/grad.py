"""Spot-intensity loss and its gradient through the transform (oracle).

Paper, Methods ("Computational Scaling"): gradients of the complex farfield
weights are propagated forward and backward through the transform for
gradient-descent refinement of uniform top hats or images. The paper gives
no loss; the reading used here is the normalised spot-intensity loss

  I_n = |E_n|^2,  mu = mean(I),  r_n = I_n / mu - t_n,  L = sum_n r_n^2.

Closed-form gradient (derived from the transform definition
E_n = sum_m f_m K_nm, f_m = A_m exp(i phi_m), K_nm = exp(-i C_n . Z_m)):

  G_k        = dL/dI_k = (2/mu) (r_k - (1/N) sum_n r_n I_n / mu)
  ghat_n     = 2 G_n E_n     (complex gradient in the dL/dRe + i dL/dIm convention)
  dL/dphi_m  = -Im(f_m conj(h_m)),        h = K^H ghat
  dL/dC_nd   = Im(conj(ghat_n) S_nd),     S_nd = sum_m Z_dm f_m K_nm

plus float64 central finite differences of L for checking.
"""
from __future__ import annotations

import numpy as np

from . import transform


def loss_from_E(E: np.ndarray, t: np.ndarray) -> float:
    I = np.abs(E) ** 2
    mu = I.mean()
    r = I / mu - np.asarray(t, np.float64)
    return float(np.sum(r * r))


def loss(amp, phase, C, Z, t) -> float:
    return loss_from_E(transform.forward(transform.field(amp, phase), C, Z), t)


def grad_E(E: np.ndarray, t: np.ndarray) -> np.ndarray:
    """ghat_n = dL/dRe(E_n) + i dL/dIm(E_n) = 2 G_n E_n."""
    I = np.abs(E) ** 2
    N = I.size
    mu = I.mean()
    r = I / mu - np.asarray(t, np.float64)
    G = (2.0 / mu) * (r - np.sum(r * I / mu) / N)
    return 2.0 * G * E


def moments(f: np.ndarray, C: np.ndarray, Z: np.ndarray, chunk: int = transform.CHUNK) -> np.ndarray:
    """S (N, D): S_nd = sum_m Z_dm f_m K_nm."""
    f = np.asarray(f, np.complex128).ravel()
    C = np.asarray(C, np.float64)
    Z = np.asarray(Z, np.float64)
    S = np.zeros(C.shape, np.complex128)
    for m0 in range(0, f.size, chunk):
        m1 = min(f.size, m0 + chunk)
        Kf = np.exp(-1j * (C @ Z[:, m0:m1])) * f[None, m0:m1]   # (N, chunk)
        S += Kf @ Z[:, m0:m1].T
    return S


def backward(amp, phase, C, Z, ghat) -> tuple:
    """(dL/dphi (M,), dL/dC (N, D)) given ghat (N,) complex."""
    f = transform.field(amp, phase)
    h = transform.adjoint(ghat, C, Z)
    dphi = -np.imag(f * np.conj(h))
    dC = np.imag(np.conj(np.asarray(ghat))[:, None] * moments(f, C, Z))
    return dphi, dC


def grad(amp, phase, C, Z, t) -> tuple:
    """Closed-form (L, dL/dphi, dL/dC)."""
    f = transform.field(amp, phase)
    E = transform.forward(f, C, Z)
    ghat = grad_E(E, t)
    dphi, dC = backward(amp, phase, C, Z, ghat)
    return loss_from_E(E, t), dphi, dC


def fd_phase(amp, phase, C, Z, t, idx, h: float = 1e-6) -> np.ndarray:
    """Central finite differences of L with respect to phi at flat indices idx."""
    phase = np.asarray(phase, np.float64).ravel()
    out = np.empty(len(idx))
    for k, m in enumerate(idx):
        p = phase.copy(); p[m] += h
        q = phase.copy(); q[m] -= h
        out[k] = (loss(amp, p, C, Z, t) - loss(amp, q, C, Z, t)) / (2 * h)
    return out


def fd_coeff(amp, phase, C, Z, t, idx, h: float = 1e-6) -> np.ndarray:
    """Central finite differences of L with respect to C at (n, d) pairs idx."""
    C = np.asarray(C, np.float64)
    out = np.empty(len(idx))
    for k, (n, d) in enumerate(idx):
        cp = C.copy(); cp[n, d] += h
        cm = C.copy(); cm[n, d] -= h
        out[k] = (loss(amp, phase, cp, Z, t) - loss(amp, phase, cm, Z, t)) / (2 * h)
    return out
