"""Holograms in a basis of principal isoplanatic modes (rotated Zernikes
built by ash_hologram_create_mixed) against the oracle on the rotated
problem (C', Z') = oracle.svd.rotate(C, Z, cols, K)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from gpu_helpers import GRAD_TOL, assert_close  # noqa: E402
from oracle import grad as ograd, svd, transform, zernike  # noqa: E402
from workloads import random_problem  # noqa: E402

pytestmark = pytest.mark.gpu


def _rotated(p, cols, K):
    from paper_2505_08777_gb300 import Hologram, principal_modes
    mix, Cout, sigma = principal_modes(p.coeff, cols, K)
    h = Hologram(torch.from_numpy(p.amp).cuda(), torch.from_numpy(Cout).cuda(), noll=p.noll, mix=mix)
    return h, mix, Cout


@pytest.mark.parametrize("nx,ny,N,noll,K", [(96, 80, 150, list(range(2, 12)), 8), (96, 80, 150, list(range(2, 12)), 3),
                                            (160, 128, 300, list(range(2, 13)), 9), (64, 64, 40, list(range(2, 8)), 2)])
def test_principal_mode_hologram_matches_oracle(nx, ny, N, noll, K):
    p = random_problem(500 + N + K, nx, ny, N, noll, defocus_max=8.0)
    cols = list(range(2, len(noll)))          # rotate everything but the tilts
    h, mix, Cout = _rotated(p, cols, K)
    Z = zernike.basis(p.nx, p.ny, p.noll)
    C2, Z2 = svd.rotate(p.coeff.astype(np.float64), Z, cols, K)
    A = p.amp.astype(np.float64).ravel()
    # the library's rotation and the oracle's agree up to the sign of each
    # principal mode; use the library's coefficients with the oracle's basis
    # rotated by the library's mixing matrix (both exact in FP64)
    Zm = mix @ Z
    C_lib = Cout.astype(np.float64)
    np.testing.assert_allclose(C_lib @ Zm, C2 @ Z2, atol=1e-4 * np.abs(C2 @ Z2).max())
    f = transform.field(A, p.phase0)
    E_ref = transform.forward(f, C_lib, Zm)
    E = h.forward(torch.from_numpy(p.phase0).cuda()).cpu().numpy()
    assert_close(E, E_ref, what="principal-mode forward")
    rng = np.random.default_rng(K)
    y = (rng.normal(size=N) + 1j * rng.normal(size=N)).astype(np.complex64)
    g_ref = transform.adjoint(y.astype(np.complex128), C_lib, Zm)
    g, _ = h.adjoint(torch.from_numpy(y).cuda(), want_field=True, want_phase=False)
    assert_close(g.cpu().numpy(), g_ref, what="principal-mode adjoint")
    # gradients: the rotated modes are still polynomials, so dL/dC takes the
    # tensor-core moment pass with tile polynomials of the mixed monomials
    gE = ograd.grad_E(E_ref, p.target).astype(np.complex64)
    dph, dC = h.grad(torch.from_numpy(p.phase0).cuda(), torch.from_numpy(gE).cuda())
    dph_ref, dC_ref = ograd.backward(A, p.phase0, C_lib, Zm, gE.astype(np.complex128))
    assert np.linalg.norm(dph.cpu().numpy().ravel() - dph_ref) <= GRAD_TOL * np.linalg.norm(dph_ref)
    assert np.linalg.norm(dC.cpu().numpy() - dC_ref) <= GRAD_TOL * np.linalg.norm(dC_ref)
    if N >= 64:
        assert h.launch_info()["kernels"] & 8
    if K == len(cols):
        # full rank: the same transform as the original Zernike problem
        E_orig = transform.forward(f, p.coeff.astype(np.float64), Z)
        assert_close(E, E_orig, what="full-rank rotation = original forward")


def test_principal_modes_keep_the_exact_tilt_layout():
    """D = 11 (Noll 2-12) rotated to 9 principal modes plus the two tilts:
    the tilts stay unit rows, so the tensor-core path keeps one K-atom."""
    p = random_problem(77, 128, 96, 300, list(range(2, 13)), defocus_max=10.0)
    h, mix, Cout = _rotated(p, list(range(2, 11)), 9)
    h.set_variant(2)
    Z = zernike.basis(p.nx, p.ny, p.noll)
    E_ref = transform.forward(transform.field(p.amp.astype(np.float64).ravel(), p.phase0), Cout.astype(np.float64),
                              mix @ Z)
    assert_close(h.forward(torch.from_numpy(p.phase0).cuda()).cpu().numpy(), E_ref, what="tc forward, rotated D=11")
