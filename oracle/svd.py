"""Principal isoplanatic modes (oracle).

Paper, Methods ("Anisoplanatic Singular Value Decomposition"): the N x D
aberration matrix W = w_d^(n) is factored as W = U Sigma V^dagger; the
columns of V rotate the Zernike basis into D principal isoplanatic modes,
ordered by singular value. Keeping the K largest singular values gives the
truncated correction Sigma_K. Sec. III reports the normalised singular
values sigma~_i = sigma_i / sum_i sigma_i and their Shannon entropy; the
printed formula has lost its minus sign, the reading here is
H = -sum_i sigma~_i log2 sigma~_i (>= 0).

Since sum_d W_nd Z_d = sum_k (U Sigma)_nk (V^T Z)_k, the rotated problem
has coefficients U Sigma (N x K) and basis rows V^T Z (K x M). The paper
removes the position-defining shear (tilt) terms before the analysis;
`principal_modes` therefore factors only the columns listed in `cols`.
"""
from __future__ import annotations

import numpy as np


def principal_modes(W: np.ndarray, K: int | None = None):
    """Return (U, s, Vt) of W (N x D), truncated to K singular triplets."""
    U, s, Vt = np.linalg.svd(np.asarray(W, np.float64), full_matrices=False)
    if K is not None:
        U, s, Vt = U[:, :K], s[:K], Vt[:K]
    return U, s, Vt


def entropy(s: np.ndarray) -> float:
    p = np.asarray(s, np.float64)
    p = p / p.sum()
    p = p[p > 0]
    return float(-np.sum(p * np.log2(p)))


def rotate(C: np.ndarray, Z: np.ndarray, cols, K: int):
    """Rotate the modes in `cols` of (C, Z) to their K principal modes.

    Returns (C', Z'): the untouched columns first (in order), then K rotated
    columns with coefficients U_K Sigma_K and basis rows V_K^T Z[cols].
    """
    C = np.asarray(C, np.float64)
    Z = np.asarray(Z, np.float64)
    cols = list(cols)
    keep = [d for d in range(C.shape[1]) if d not in cols]
    U, s, Vt = principal_modes(C[:, cols], K)
    C2 = np.concatenate([C[:, keep], U * s[None, :]], axis=1)
    Z2 = np.concatenate([Z[keep], Vt @ Z[cols]], axis=0)
    return C2, Z2
