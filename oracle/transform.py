"""Compressed spot transform and its adjoint (oracle, complex128).

Paper, Sec. II: the DFT restricted to N target points becomes a compressed
sum of per-spot kernels,
    F_n      = sum_m K_n(m) f_m              (near -> far, "overlap integrals"),
    f(m)     = sum_n K_n(m)^* F_n            (far -> near, "summation of kernels"),
with the Zernike kernel K_n(m) = exp(-i sum_d w_d^(n) Z_d(m)) (Sec. II;
Methods "Computational Scaling" builds it from the N x D matrix w_d^(n)).
The paper writes these up to proportionality; the reading used here is the
unnormalised sum (no 1/M or 1/sqrt(M) factor).

Evaluated in pixel chunks (all spots x a block of pixels) so that no N x M
matrix is held; `workers` > 1 spreads chunks over a thread pool (numpy
releases the GIL inside exp and matmul). Chunk partial sums are added in
chunk order, so the result does not depend on `workers`.
"""
from __future__ import annotations

import concurrent.futures as cf

import numpy as np

CHUNK = 4096


def field(amp: np.ndarray, phase: np.ndarray) -> np.ndarray:
    """Nearfield f = A exp(i phi) (phase-only SLM, Sec. II / Fig. 1a)."""
    return np.asarray(amp, np.float64).ravel() * np.exp(1j * np.asarray(phase, np.float64).ravel())


def _chunks(M: int, chunk: int):
    return [(m0, min(M, m0 + chunk)) for m0 in range(0, M, chunk)]


def _map(fn, items, workers: int):
    if workers <= 1:
        return [fn(it) for it in items]
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        return list(ex.map(fn, items))


def forward(f: np.ndarray, C: np.ndarray, Z: np.ndarray, chunk: int = CHUNK, workers: int = 1) -> np.ndarray:
    """E_n = sum_m f_m exp(-i C_n . Z_m).  f (M,), C (N, D), Z (D, M) -> E (N,)."""
    f = np.asarray(f, np.complex128).ravel()
    C = np.asarray(C, np.float64)
    Z = np.asarray(Z, np.float64)

    def part(rng):
        m0, m1 = rng
        theta = C @ Z[:, m0:m1]
        return np.exp(-1j * theta) @ f[m0:m1]

    E = np.zeros(C.shape[0], np.complex128)
    for p in _map(part, _chunks(f.size, chunk), workers):
        E += p
    return E


def adjoint(y: np.ndarray, C: np.ndarray, Z: np.ndarray, chunk: int = CHUNK, workers: int = 1) -> np.ndarray:
    """g_m = sum_n y_n exp(+i C_n . Z_m).  y (N,), C (N, D), Z (D, M) -> g (M,)."""
    y = np.asarray(y, np.complex128).ravel()
    C = np.asarray(C, np.float64)
    Z = np.asarray(Z, np.float64)
    M = Z.shape[1]
    g = np.empty(M, np.complex128)

    def part(rng):
        m0, m1 = rng
        theta = C @ Z[:, m0:m1]
        g[m0:m1] = y @ np.exp(1j * theta)

    _map(part, _chunks(M, chunk), workers)
    return g


def kernel_matrix(C: np.ndarray, Z: np.ndarray) -> np.ndarray:
    """Explicit K (N, M) = exp(-i C Z): the cached-kernel form (Methods), tiny grids only."""
    return np.exp(-1j * (np.asarray(C, np.float64) @ np.asarray(Z, np.float64)))


def phase_of(g: np.ndarray) -> np.ndarray:
    """phi = arg g, with phi = 0 where g == 0 exactly."""
    g = np.asarray(g, np.complex128)
    out = np.angle(g)
    out[g == 0] = 0.0
    return out
