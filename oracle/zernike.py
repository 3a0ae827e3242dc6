"""Zernike basis on the SLM pixel grid (oracle, float64).

Paper: Sec. II writes each kernel's phase as sum_d w_d^(n) Z_d(x, y) with
Zernike polynomials indexed by a single ANSI index d (tilt x ~ Z_2 = Z_1^1,
tilt y ~ Z_1 = Z_1^-1, defocus Z_4 = Z_2^0, spherical Z_12 = Z_4^0).
Methods ("Computational Scaling") evaluates each Z_d per pixel.

Readings (the paper is silent on these):
  * Coordinates: pixel (i, j) -> x = (i - (nx-1)/2)/R, y = (j - (ny-1)/2)/R,
    R = min(nx, ny)/2 (unit disk inscribed in the SLM). Pixels outside the
    disk keep their polynomial values.
  * Polynomial: Z_n^m = R_n^|m|(rho) cos(m theta) for m >= 0 and
    R_n^|m|(rho) sin(|m| theta) for m < 0, textbook radial polynomial,
    no RMS normalisation (peak 1 at rho = 1).
  * Column order of the coefficient matrix is given as Noll indices; Noll
    and ANSI enumerate the same polynomials in different orders.

This module evaluates the radial-polynomial form directly; it deliberately
does not use the monomial expansion the GPU path is built on.
"""
from __future__ import annotations

import math

import numpy as np


def noll_to_nm(j: int) -> tuple:
    """Noll index j >= 1 -> (n, m). Row n holds indices n(n+1)/2+1 .. (n+1)(n+2)/2;
    |m| increases along the row; even j carries cos (m > 0), odd j sin (m < 0)."""
    if j < 1:
        raise ValueError("Noll index starts at 1")
    n = 0
    while (n + 1) * (n + 2) // 2 < j:
        n += 1
    k = j - n * (n + 1) // 2 - 1          # 0-based position within row n
    if n % 2 == 0:
        am = 2 * ((k + 1) // 2)
    else:
        am = 2 * (k // 2) + 1
    if am == 0:
        return n, 0
    return n, (am if j % 2 == 0 else -am)


def ansi_index(n: int, m: int) -> int:
    """ANSI single index of Z_n^m: (n(n+2) + m)/2 (the paper's indexing, Sec. II)."""
    return (n * (n + 2) + m) // 2


def ansi_to_nm(j: int) -> tuple:
    n = int(math.floor((math.sqrt(8 * j + 1) - 1) / 2))
    m = 2 * j - n * (n + 2)
    return n, m


def radial(n: int, am: int, rho: np.ndarray) -> np.ndarray:
    """Textbook radial polynomial R_n^am(rho), am = |m| <= n, n - am even:
    sum_k (-1)^k (n-k)! / (k! ((n+am)/2-k)! ((n-am)/2-k)!) rho^(n-2k)."""
    if am > n or (n - am) % 2:
        raise ValueError("invalid (n, m)")
    out = np.zeros_like(rho, dtype=np.float64)
    for k in range((n - am) // 2 + 1):
        c = ((-1) ** k) * math.factorial(n - k) / (
            math.factorial(k) * math.factorial((n + am) // 2 - k) * math.factorial((n - am) // 2 - k))
        out = out + c * rho ** (n - 2 * k)
    return out


def zernike_polar(n: int, m: int, rho: np.ndarray, theta: np.ndarray) -> np.ndarray:
    r = radial(n, abs(m), rho)
    if m >= 0:
        return r * np.cos(m * theta)
    return r * np.sin(-m * theta)


def pixel_coords(nx: int, ny: int) -> tuple:
    """(x, y) of every pixel, each (ny, nx) float64, per the coordinate reading."""
    R = min(nx, ny) / 2.0
    x = (np.arange(nx, dtype=np.float64) - (nx - 1) / 2.0) / R
    y = (np.arange(ny, dtype=np.float64) - (ny - 1) / 2.0) / R
    return np.broadcast_to(x[None, :], (ny, nx)), np.broadcast_to(y[:, None], (ny, nx))


def basis(nx: int, ny: int, noll) -> np.ndarray:
    """Z of shape (D, M), M = nx*ny, flat pixel index m = j*nx + i."""
    x, y = pixel_coords(nx, ny)
    rho = np.hypot(x, y)
    theta = np.arctan2(y, x)
    out = np.empty((len(noll), nx * ny), dtype=np.float64)
    for d, j in enumerate(noll):
        n, m = noll_to_nm(int(j))
        out[d] = zernike_polar(n, m, rho, theta).ravel()
    return out
