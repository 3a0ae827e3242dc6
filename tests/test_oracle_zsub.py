"""Pins for the oracle's simulated Zernike-subtraction calibration (CPU).

Estimator: exact on Gaussian peaks (ln I is then a parabola), the argmax
fallback when the fit has no maximum, and clipping to the sweep range.
Sweep: superimposing delta Z_d on the SLM phase must equal propagating the
unperturbed phase through the coefficient matrix shifted by -delta in
column d (an identity of the kernel definition, here between two different
constructions). Single spot: the baseline phase is the exact conjugate of
the model's kernel, so the swept intensity is symmetric about the model's
error a in that order and, on a grid symmetric about a, the vertex is a
itself: this fixes the signs of the sweep and of the update. Loop: with one
spot it must converge to the system's coefficients; with nine, one round
must remove most of the intensity-weighted wavefront error and brighten the
spots.
"""
import numpy as np

from oracle import transform, zernike, zsub
from workloads import ZSUB_DELTAS, config_zsub, zsub_model0


def test_estimate_is_exact_on_gaussian_peaks():
    d = np.linspace(-1.5, 1.5, 7)
    peaks = np.array([-1.2, -0.3, 0.0, 0.41, 1.49])
    I = 3.0 * np.exp(-2.0 * (d[:, None] - peaks[None, :]) ** 2)
    assert np.allclose(zsub.estimate(I, d), peaks, atol=1e-12)


def test_estimate_fallback_and_clip():
    d = np.linspace(-1.0, 1.0, 5)
    # convex in ln I (no maximum): the largest sample's offset
    I_convex = np.exp(np.array([1.0, 0.2, 0.0, 0.3, 0.9]))[:, None]
    # a peak beyond the range: clipped to the end
    I_far = np.exp(-(d - 3.0) ** 2)[:, None]
    # an intensity of exactly 0 is read as 1e-37
    I_zero = np.array([0.0, 1.0, 2.0, 1.0, 0.0])[:, None]
    out = zsub.estimate(np.hstack([I_convex, I_far, I_zero]), d)
    assert out[0] == -1.0
    assert out[1] == 1.0
    assert abs(out[2]) < 1e-12


def test_sweep_equals_shifted_coefficients():
    p = config_zsub(3, 40, 36, 2)
    Z = zernike.basis(p.nx, p.ny, p.noll)
    C = p.coeff.astype(np.float64)
    amp = p.amp.astype(np.float64).ravel()
    phase = p.phase0.astype(np.float64).ravel()
    d = np.array([-0.7, 0.25, 1.1])
    for mode in (2, 5, 9):
        I = zsub.sweep(amp, phase, C, Z, mode, d)
        for k, dk in enumerate(d):
            Cs = C.copy()
            Cs[:, mode] -= dk
            ref = np.abs(transform.forward(transform.field(amp, phase), Cs, Z)) ** 2
            assert np.allclose(I[k], ref, rtol=1e-10, atol=0)


def test_single_spot_vertex_is_the_model_error():
    nx, ny = 48, 40
    noll = [2, 3, 4, 5, 6, 7, 8]
    Z = zernike.basis(nx, ny, noll)
    amp = np.ones(nx * ny)
    rng = np.random.default_rng(4)
    C_model = rng.normal(0.0, 0.4, size=(1, len(noll)))
    for mode, a in ((2, 0.37), (4, -0.52), (6, 0.11)):
        C_sys = C_model.copy()
        C_sys[0, mode] += a
        phi = zsub.baseline_phase(amp, C_model, Z, np.ones(1))
        # the superposition of one kernel is its conjugate phase
        assert np.allclose(np.exp(1j * phi), np.exp(1j * (C_model @ Z)[0]), atol=1e-12)
        grid = a + np.linspace(-0.9, 0.9, 7)
        I = zsub.sweep(amp, phi, C_sys, Z, mode, grid)
        assert abs(zsub.estimate(I, grid)[0] - a) < 1e-9


def test_single_spot_calibration_converges_to_the_system():
    p = config_zsub(2, 128, 112, 1)
    Z = zernike.basis(p.nx, p.ny, p.noll)
    amp = p.amp.astype(np.float64).ravel()
    C_sys = p.coeff.astype(np.float64)
    C0 = zsub_model0(p).astype(np.float64)
    modes = [k for k, j in enumerate(p.noll) if j >= 4]
    C1, _ = zsub.calibrate(amp, C0, C_sys, Z, p.target, modes, ZSUB_DELTAS, rounds=4)
    e0 = np.linalg.norm((C0 - C_sys)[:, modes])
    assert np.linalg.norm((C1 - C_sys)[:, modes]) < 0.01 * e0
    assert zsub.wavefront_residual(amp, C1, C_sys, Z) < 0.01 * zsub.wavefront_residual(amp, C0, C_sys, Z)


def test_one_round_reduces_the_wavefront_residual():
    # nine spots: the phase-only superposition couples them, so the loop
    # settles at a residual set by that crosstalk; one round removes most
    # of the aberration and makes the spots brighter
    p = config_zsub(2, 64, 56, 3)
    Z = zernike.basis(p.nx, p.ny, p.noll)
    amp = p.amp.astype(np.float64).ravel()
    C_sys = p.coeff.astype(np.float64)
    C0 = zsub_model0(p).astype(np.float64)
    modes = [k for k, j in enumerate(p.noll) if j >= 4]
    C1, steps = zsub.calibrate(amp, C0, C_sys, Z, p.target, modes, ZSUB_DELTAS, rounds=1)
    assert [d for d, _ in steps] == modes
    r0 = zsub.wavefront_residual(amp, C0, C_sys, Z)
    r1 = zsub.wavefront_residual(amp, C1, C_sys, Z)
    assert r1 < 0.35 * r0, (r0, r1)

    def brightness(C):
        phi = zsub.baseline_phase(amp, C, Z, p.target)
        return np.mean(np.abs(transform.forward(transform.field(amp, phi), C_sys, Z)) ** 2)

    assert brightness(C1) > 1.2 * brightness(C0)
