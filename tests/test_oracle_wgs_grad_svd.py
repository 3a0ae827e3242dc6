"""Pins for the oracle's WGS loop, gradient and SVD (CPU only).

WGS: on integer-bin spots with flat amplitude the compressed transform is
the DFT, so the loop must equal an independent FFT-based implementation
written here; it must also reach near-unit uniformity there, be invariant
to the scale of the weights, and resume bit-for-bit.
Gradient: float64 central finite differences of the loss, and torch
autograd (complex128, CPU) applied to a direct transcription of the
forward definition.
SVD: exact reconstruction, K = D rotation leaves every kernel phase
unchanged, entropy of equal singular values is log2(D).
"""
import math

import numpy as np
import pytest

from oracle import grad, svd, transform, wgs, zernike
from workloads import config_c1, flat_amplitude, random_problem


def _bin_problem(nx, ny, bins):
    R = min(nx, ny) / 2.0
    C = np.array([[2 * math.pi * kx * R / nx, 2 * math.pi * ky * R / ny] for kx, ky in bins])
    return C, zernike.basis(nx, ny, [2, 3])


def _fft_wgs(amp, phase0, bins, nx, ny, target, iters, feedback=1.0, fixed=None):
    """Same update rule, with the transform done by numpy FFTs (DFT special
    case); `feedback` is the weight exponent, `fixed` held spot phases."""
    A = amp.reshape(ny, nx)
    phase = phase0.reshape(ny, nx).copy()
    t = np.asarray(target, np.float64)
    t_hat = t / np.linalg.norm(t)
    w = t.copy()
    cen = np.array([np.exp(1j * math.pi * (kx * (nx - 1) / nx + ky * (ny - 1) / ny)) for kx, ky in bins])
    for _ in range(iters):
        F = np.fft.fft2(A * np.exp(1j * phase))
        E = np.array([F[ky % ny, kx % nx] for kx, ky in bins]) * cen
        e_hat = np.abs(E) / np.linalg.norm(np.abs(E))
        w = w * np.power(t_hat / np.maximum(e_hat, 1e-30), feedback)
        w = w / np.linalg.norm(w)
        y = w * np.exp(1j * (np.angle(E) if fixed is None else fixed))
        spec = np.zeros((ny, nx), np.complex128)
        for (kx, ky), v, c in zip(bins, y, cen):
            spec[ky % ny, kx % nx] += v * np.conj(c)
        g = np.fft.ifft2(spec) * (nx * ny)
        phase = np.where(g == 0, 0.0, np.angle(g))
    return phase.ravel(), w


def test_wgs_matches_fft_implementation_on_integer_bins():
    nx, ny = 24, 20
    bins = [(-5, -4), (-5, 3), (4, -4), (4, 3), (0, 6), (-2, 0), (7, -1)]
    C, Z = _bin_problem(nx, ny, bins)
    rng = np.random.default_rng(3)
    amp = flat_amplitude(nx, ny).astype(np.float64).ravel()
    phase0 = rng.uniform(0, 2 * math.pi, nx * ny)
    target = rng.uniform(0.5, 1.0, len(bins))
    res = wgs.run(amp, phase0, C, Z, target, 6)
    ph_fft, w_fft = _fft_wgs(amp, phase0, bins, nx, ny, target, 6)
    np.testing.assert_allclose(np.exp(1j * res.phase), np.exp(1j * ph_fft), atol=1e-9)
    np.testing.assert_allclose(res.weights, w_fft, rtol=1e-9)


@pytest.mark.parametrize("feedback", [0.0, 0.5, 2.0])
def test_wgs_variants_match_fft_implementation(feedback):
    """Feedback exponent and phase fixing against the FFT implementation; p = 0
    keeps the weights at the normalised targets (plain GS)."""
    nx, ny = 24, 20
    bins = [(-5, -4), (-5, 3), (4, -4), (4, 3), (0, 6), (-2, 0), (7, -1)]
    C, Z = _bin_problem(nx, ny, bins)
    rng = np.random.default_rng(4)
    amp = flat_amplitude(nx, ny).astype(np.float64).ravel()
    phase0 = rng.uniform(0, 2 * math.pi, nx * ny)
    target = rng.uniform(0.5, 1.0, len(bins))
    res = wgs.run(amp, phase0, C, Z, target, 5, feedback=feedback)
    ph_fft, w_fft = _fft_wgs(amp, phase0, bins, nx, ny, target, 5, feedback=feedback)
    np.testing.assert_allclose(np.exp(1j * res.phase), np.exp(1j * ph_fft), atol=1e-9)
    np.testing.assert_allclose(res.weights, w_fft, rtol=1e-9)
    if feedback == 0.0:
        np.testing.assert_allclose(res.weights, target / np.linalg.norm(target), rtol=1e-12)
    psi = rng.uniform(-math.pi, math.pi, len(bins))
    fixed = wgs.run(amp, phase0, C, Z, target, 4, feedback=feedback, fixed_psi=psi)
    ph_fix, w_fix = _fft_wgs(amp, phase0, bins, nx, ny, target, 4, feedback=feedback, fixed=psi)
    np.testing.assert_allclose(np.exp(1j * fixed.phase), np.exp(1j * ph_fix), atol=1e-9)
    np.testing.assert_allclose(fixed.weights, w_fix, rtol=1e-9)
    np.testing.assert_array_equal(fixed.psi, psi)


def test_wgs_reaches_uniformity_on_integer_bins():
    nx, ny = 32, 32
    bins = [(kx, ky) for kx in (-6, -2, 2, 6) for ky in (-6, -2, 2, 6)]
    C, Z = _bin_problem(nx, ny, bins)
    rng = np.random.default_rng(4)
    amp = flat_amplitude(nx, ny).astype(np.float64).ravel()
    res = wgs.run(amp, rng.uniform(0, 2 * math.pi, nx * ny), C, Z, np.ones(len(bins)), 60)
    # not monotone step by step, but rising on average and close to 1 at the end
    assert res.uniformity > 0.995
    assert np.mean(res.history[-10:]) > np.mean(res.history[:10])


def test_wgs_weight_scale_invariance_and_resume():
    p = random_problem(8, 30, 26, 6, range(2, 12))
    Z = zernike.basis(p.nx, p.ny, p.noll)
    C = p.coeff.astype(np.float64)
    T = p.target.astype(np.float64)
    r1 = wgs.run(p.amp, p.phase0, C, Z, T, 4)
    r2 = wgs.run(p.amp, p.phase0, C, Z, T, 4, weights0=3.0 * T)
    np.testing.assert_allclose(np.exp(1j * r1.phase), np.exp(1j * r2.phase), atol=1e-12)
    full = wgs.run(p.amp, p.phase0, C, Z, T, 8)
    half = wgs.run(p.amp, r1.phase, C, Z, T, 4, weights0=r1.weights)
    np.testing.assert_array_equal(full.phase, half.phase)
    np.testing.assert_array_equal(full.weights, half.weights)


def test_efficiency_parseval():
    # All M integer bins targeted: eta = 1 for any phase (Parseval).
    nx, ny = 6, 4
    bins = [(kx, ky) for ky in range(ny) for kx in range(nx)]
    C, Z = _bin_problem(nx, ny, bins)
    rng = np.random.default_rng(0)
    amp = rng.uniform(0.2, 1.0, nx * ny)
    E = transform.forward(transform.field(amp, rng.uniform(0, 6, nx * ny)), C, Z)
    assert abs(wgs.efficiency(E, amp) - 1.0) < 1e-12


def test_uniformity_definition():
    E = np.array([1.0, 2.0, 1.0 + 0j])
    T = np.array([1.0, 2.0, 0.5])
    # I^ = [1, 1, 4] -> U = 1 - 3/5
    assert abs(wgs.uniformity(E, T) - 0.4) < 1e-15


@pytest.mark.slow
def test_c1_wgs_uniformity_recorded():
    p = config_c1(1)
    Z = zernike.basis(p.nx, p.ny, p.noll)
    res = wgs.run(p.amp, p.phase0, p.coeff, Z, p.target, p.iters, workers=4)
    # expected behaviour (not a number the paper prints): WGS drives 16 spots to > 0.95 uniformity
    assert res.uniformity > 0.95


def _grad_problem():
    p = random_problem(12, 9, 7, 5, range(2, 12), defocus_max=3.0, target_range=(0.5, 1.5))
    Z = zernike.basis(p.nx, p.ny, p.noll)
    return p, Z


def test_gradient_matches_finite_differences():
    p, Z = _grad_problem()
    C = p.coeff.astype(np.float64)
    phase = p.phase0.astype(np.float64).ravel()
    L, dphi, dC = grad.grad(p.amp, phase, C, Z, p.target)
    idx = list(range(0, p.M, 5))
    fd = grad.fd_phase(p.amp, phase, C, Z, p.target, idx, h=1e-6)
    np.testing.assert_allclose(dphi[idx], fd, rtol=1e-5, atol=1e-7 * np.abs(fd).max())
    pairs = [(n, d) for n in range(p.N) for d in range(p.D)]
    fdc = grad.fd_coeff(p.amp, phase, C, Z, p.target, pairs, h=1e-6)
    got = np.array([dC[n, d] for n, d in pairs])
    np.testing.assert_allclose(got, fdc, rtol=1e-5, atol=1e-7 * np.abs(fdc).max())


def test_gradient_matches_torch_autograd():
    torch = pytest.importorskip("torch")
    p, Z = _grad_problem()
    C = p.coeff.astype(np.float64)
    phase = p.phase0.astype(np.float64).ravel()
    L, dphi, dC = grad.grad(p.amp, phase, C, Z, p.target)
    tph = torch.tensor(phase, dtype=torch.float64, requires_grad=True)
    tC = torch.tensor(C, dtype=torch.float64, requires_grad=True)
    tZ = torch.tensor(Z, dtype=torch.float64)
    tA = torch.tensor(p.amp.astype(np.float64).ravel())
    f = tA * torch.exp(1j * tph)
    K = torch.exp(-1j * (tC @ tZ))
    E = K @ f
    I = E.abs() ** 2
    r = I / I.mean() - torch.tensor(p.target.astype(np.float64))
    loss = (r * r).sum()
    loss.backward()
    assert abs(loss.item() - L) < 1e-12 * abs(L)
    np.testing.assert_allclose(tph.grad.numpy(), dphi, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(tC.grad.numpy(), dC, rtol=1e-10, atol=1e-12)


def test_svd_reconstruction_and_full_rotation():
    p = random_problem(5, 20, 16, 30, range(2, 12), defocus_max=5.0)
    Z = zernike.basis(p.nx, p.ny, p.noll)
    C = p.coeff.astype(np.float64)
    cols = list(range(2, 10))
    U, s, Vt = svd.principal_modes(C[:, cols])
    np.testing.assert_allclose(U @ np.diag(s) @ Vt, C[:, cols], atol=1e-12)
    assert np.all(np.diff(s) <= 0)
    C2, Z2 = svd.rotate(C, Z, cols, len(cols))
    np.testing.assert_allclose(C2 @ Z2, C @ Z, atol=1e-10)
    C3, Z3 = svd.rotate(C, Z, cols, 3)
    assert C3.shape == (p.N, 5) and Z3.shape == (5, p.M)
    # truncation error equals the discarded singular values (Eckart-Young)
    Ct = (U[:, :3] * s[:3]) @ Vt[:3]
    assert abs(np.linalg.norm(Ct - C[:, cols]) - math.sqrt(np.sum(s[3:] ** 2))) < 1e-9


def test_svd_entropy():
    assert abs(svd.entropy(np.ones(8)) - 3.0) < 1e-15
    assert svd.entropy(np.array([1.0, 0.0, 0.0])) == 0.0
