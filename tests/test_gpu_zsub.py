"""GPU parity of the simulated Zernike-subtraction calibration.

Sweep: the library evaluates the swept SLM phase as a forward through the
system's coefficients with one column shifted; the oracle adds delta Z_d to
the phase itself. The intensities must agree within the transform's parity
bar (|E|^2 carries twice the field's relative error), in both kernel
families, and the handle's coefficients must be untouched afterwards.
Estimate: on the same float32 intensities both sides fit in float64, so the
per-spot vertices agree to rounding. Loop: one round over Noll 4-11 from
the superposition baseline, the model's final coefficients against the
oracle's, and the intensity-weighted wavefront residual reduced as the
oracle's is.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from gpu_helpers import REL_TOL, assert_close, oracle_inputs  # noqa: E402
from oracle import transform, zernike, zsub  # noqa: E402
from workloads import ZSUB_DELTAS, config_zsub, zsub_model0  # noqa: E402

pytestmark = pytest.mark.gpu


def _holo(p, coeff):
    from paper_2505_08777_gb300 import Hologram
    return Hologram(torch.from_numpy(p.amp).cuda(), torch.from_numpy(np.ascontiguousarray(coeff)).cuda(), noll=p.noll)


@pytest.mark.parametrize("variant", [1, 2])
@pytest.mark.parametrize("nx,ny,grid", [(96, 80, 4), (130, 97, 9)])
def test_sweep_matches_oracle(nx, ny, grid, variant):
    p = config_zsub(5, nx, ny, grid)
    Z, C, A = oracle_inputs(p)
    h = _holo(p, p.coeff)
    h.set_variant(variant)
    ph = torch.from_numpy(p.phase0).cuda()
    E0 = h.forward(ph).clone()
    for mode in (2, 6, 9):
        I = h.zsub_sweep(ph, mode, ZSUB_DELTAS).cpu().numpy().astype(np.float64)
        ref = zsub.sweep(A, p.phase0.astype(np.float64).ravel(), C, Z, mode, ZSUB_DELTAS, workers=4)
        assert I.shape == ref.shape
        assert_close(I, ref, 2 * REL_TOL, f"sweep mode {mode}")
    # coefficients and operand images restored: the same forward, bit for bit
    assert torch.equal(h.forward(ph), E0)


def test_estimate_matches_oracle_and_updates_coefficients():
    from paper_2505_08777_gb300 import zsub_estimate
    p = config_zsub(6, 96, 80, 4)
    Z, C, A = oracle_inputs(p)
    d = np.linspace(-1.2, 1.0, 9)
    I = zsub.sweep(A, p.phase0.astype(np.float64).ravel(), C, Z, 3, d, workers=4).astype(np.float32)
    # a spot with a convex profile and one with zeros exercise the fallback
    I[:, 0] = np.exp(np.linspace(1.0, 0.0, 9) ** 2).astype(np.float32)
    I[:, 1] = np.array([0, 0, 1, 2, 3, 2, 1, 0, 0], np.float32)
    ref = zsub.estimate(I.astype(np.float64), d.astype(np.float32).astype(np.float64))
    coeff = torch.from_numpy(p.coeff.copy()).cuda()
    got = zsub_estimate(torch.from_numpy(I).cuda(), d, coeff, 3).cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got - ref)) <= 1e-6 * (d.max() - d.min())
    want = p.coeff.copy()
    want[:, 3] += got.astype(np.float32)
    assert np.array_equal(coeff.cpu().numpy(), want)


def test_calibration_round_matches_oracle():
    from paper_2505_08777_gb300 import zernike_subtraction
    p = config_zsub(2, 96, 80, 3)
    Z, C_sys, A = oracle_inputs(p)
    C0 = zsub_model0(p)
    modes = [k for k, j in enumerate(p.noll) if j >= 4]
    system = _holo(p, p.coeff)
    model = _holo(p, C0)
    T = torch.from_numpy(p.target).cuda()
    C_gpu, steps = zernike_subtraction(model, system, T, modes, ZSUB_DELTAS, rounds=1)
    C_gpu = C_gpu.cpu().numpy().astype(np.float64)
    C_ref, _ = zsub.calibrate(A, C0.astype(np.float64), C_sys, Z, p.target, modes, ZSUB_DELTAS, rounds=1, workers=4)
    assert [d for d, _ in steps] == modes
    assert np.max(np.abs(C_gpu - C_ref)) <= 2e-3, np.max(np.abs(C_gpu - C_ref))
    r0 = zsub.wavefront_residual(A, C0, C_sys, Z)
    r_gpu = zsub.wavefront_residual(A, C_gpu, C_sys, Z)
    r_ref = zsub.wavefront_residual(A, C_ref, C_sys, Z)
    assert r_gpu < 0.35 * r0 and abs(r_gpu - r_ref) <= 1e-3 * r0
    assert np.array_equal(model.coefficients().cpu().numpy(), C_gpu.astype(np.float32))


def test_zsub_arguments_rejected_on_the_host():
    from paper_2505_08777_gb300 import _lib
    lib = _lib.load()
    p = config_zsub(1, 64, 64, 2)
    h = _holo(p, p.coeff)
    ph = torch.zeros((p.ny, p.nx), dtype=torch.float32, device="cuda")
    I = torch.empty((3, p.N), dtype=torch.float32, device="cuda")
    d3 = (ctypes.c_float * 3)(-1.0, 0.0, 1.0)
    assert lib.ash_zsub_sweep(h.handle, ctypes.c_void_p(ph.data_ptr()), p.coeff.shape[1], d3, 3,
                              ctypes.c_void_p(I.data_ptr()), None) != 0
    assert lib.ash_zsub_sweep(h.handle, ctypes.c_void_p(ph.data_ptr()), 0, d3, 0,
                              ctypes.c_void_p(I.data_ptr()), None) != 0
    same = (ctypes.c_float * 3)(0.5, 0.5, 0.5)
    out = torch.empty(p.N, dtype=torch.float32, device="cuda")
    assert lib.ash_zsub_estimate(ctypes.c_void_p(I.data_ptr()), same, 3, p.N, ctypes.c_void_p(out.data_ptr()),
                                 None, 0, 0, None) != 0
