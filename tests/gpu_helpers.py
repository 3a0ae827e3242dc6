"""Shared helpers for the GPU parity tests (inputs from workloads, reference
values from the oracle, comparisons in float64 on the host)."""
from __future__ import annotations

import numpy as np

from oracle import transform, zernike

# Tolerances of the transform parity (normwise and per-element guard).
REL_TOL = 1e-4
GRAD_TOL = 1e-3
UNIF_TOL = 1e-3


def rel_err(got: np.ndarray, ref: np.ndarray) -> float:
    return float(np.linalg.norm(got - ref) / np.linalg.norm(ref))


def max_guard(got: np.ndarray, ref: np.ndarray) -> float:
    return float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))


def assert_close(got, ref, tol=REL_TOL, what=""):
    got = np.asarray(got, np.complex128).ravel()
    ref = np.asarray(ref, np.complex128).ravel()
    r, g = rel_err(got, ref), max_guard(got, ref)
    assert r <= tol and g <= tol, f"{what}: normwise {r:.3e}, max-guard {g:.3e} (tol {tol:g})"
    return r, g


def oracle_inputs(p):
    Z = zernike.basis(p.nx, p.ny, p.noll)
    return Z, p.coeff.astype(np.float64), p.amp.astype(np.float64).ravel()


def oracle_forward(p, phase, Z=None, idx=None, workers=4):
    if Z is None:
        Z = zernike.basis(p.nx, p.ny, p.noll)
    C = p.coeff.astype(np.float64)
    if idx is not None:
        C = C[idx]
    f = transform.field(p.amp.astype(np.float64), np.asarray(phase, np.float64))
    return transform.forward(f, C, Z, workers=workers)


def basis_at(p, pix):
    """Z columns at flat pixel indices only (for sampled checks at full size)."""
    R = min(p.nx, p.ny) / 2.0
    i = pix % p.nx
    j = pix // p.nx
    x = (i - (p.nx - 1) / 2.0) / R
    y = (j - (p.ny - 1) / 2.0) / R
    rho = np.hypot(x, y)
    th = np.arctan2(y, x)
    out = np.empty((len(p.noll), len(pix)))
    for d, jn in enumerate(p.noll):
        n, m = zernike.noll_to_nm(jn)
        out[d] = zernike.zernike_polar(n, m, rho, th)
    return out
