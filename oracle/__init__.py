"""CPU oracle for aberration-space holography (arXiv 2505.08777).

TEST INFRASTRUCTURE ONLY. Nothing on the product path imports, calls or
executes this package: only tests/, __graft_entry__.smoke() and the
cpu_baseline / reference legs of bench.py use it. The CUDA library never
routes through it and shares no code, table or constant with it.

Plain, slow, obviously-correct numpy in float64 / complex128, following the
paper's definitions:

  zernike   : Zernike basis Z_d on the SLM pixel grid (Sec. II, Noll/ANSI
              indexing; Methods "Computational Scaling", monomial form).
  transform : compressed spot transform F_n = sum_m K_n(m) f_m and its
              adjoint f_m = sum_n K_n(m)^* F_n with Zernike kernels
              K_n(m) = exp(-i sum_d w_d^(n) Z_d(m))   (Sec. II).
  wgs       : weighted Gerchberg-Saxton loop on the compressed transform
              (Sec. II "choose the N complex farfield weights", Sec. III).
  grad      : spot-intensity loss and its gradient with respect to the SLM
              phase and the coefficient matrix (Methods, gradient descent
              through the transform), closed form and finite differences.
  svd       : principal isoplanatic modes W = U Sigma V^dagger (Methods,
              "Anisoplanatic Singular Value Decomposition").
  cg        : conjugate-gradient refinement of the SLM phase on that loss
              (Methods: precision top hats refined by CG through the
              transform's gradients).
  zsub      : simulated Zernike-subtraction calibration (Sec. III,
              calibration by swept global Zernike orders and per-spot
              subtraction) on a synthetic system matrix.

Readings where the paper is silent (coordinates, Zernike normalisation,
transform normalisation, WGS update rule, metrics) are stated in each
module's docstring.
"""
from . import zernike, transform, wgs, grad, svd, zsub, cg  # noqa: F401
