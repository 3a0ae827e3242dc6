"""GPU parity of the WGS loop and of the hand-written gradient.

WGS: final spot uniformity within 1e-3 absolute of the oracle's after the
full loop (trajectories drift apart slowly in FP32, so only the final metric
is compared), the metrics the kernel reports against the oracle's formula on
the GPU's own final field, and bitwise resume (k + k iterations == 2k).
Gradient: dL/dphase and dL/dC against the oracle's closed form on the same
grad_E at 1e-3 normwise, and the oracle's closed form is itself pinned to
float64 finite differences in the CPU tests.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from gpu_helpers import GRAD_TOL, UNIF_TOL, assert_close, oracle_inputs  # noqa: E402
from oracle import grad as ograd  # noqa: E402
from oracle import transform, wgs  # noqa: E402
from workloads import config_c1, random_problem  # noqa: E402

pytestmark = pytest.mark.gpu


def _holo(p):
    from paper_2505_08777_gb300 import Hologram
    return Hologram(torch.from_numpy(p.amp).cuda(), torch.from_numpy(p.coeff).cuda(), noll=p.noll)


def _run_wgs(h, p, iters, phase=None, w=None):
    ph = torch.from_numpy(p.phase0 if phase is None else phase).cuda().clone()
    ww = torch.from_numpy(p.target if w is None else w).cuda().clone()
    T = torch.from_numpy(p.target).cuda()
    E, met = h.wgs(ph, ww, T, iters)
    torch.cuda.synchronize()
    return ph, ww, E, met


def test_wgs_c1_uniformity_matches_oracle():
    p = config_c1(1)
    h = _holo(p)
    ph, ww, E, met = _run_wgs(h, p, p.iters)
    Z, C, A = oracle_inputs(p)
    res = wgs.run(A, p.phase0, C, Z, p.target, p.iters, workers=4)
    met = met.cpu().numpy()
    assert abs(float(met[0]) - res.uniformity) <= UNIF_TOL, (met[0], res.uniformity)
    # reported metrics equal the oracle formulas on the GPU's own final field
    E = E.cpu().numpy().astype(np.complex128)
    assert abs(met[0] - wgs.uniformity(E, p.target)) <= 1e-5
    assert abs(met[1] - wgs.efficiency(E, p.amp)) <= 1e-5 * max(1.0, wgs.efficiency(E, p.amp))
    # and the final field is the oracle forward of the GPU's final phase
    E_ref = transform.forward(transform.field(A, ph.cpu().numpy()), C, Z)
    assert_close(E, E_ref, what="final field")


@pytest.mark.parametrize("N,noll,flat", [(37, list(range(2, 13)), True), (300, list(range(2, 12)), False)])
def test_wgs_random_uniformity(N, noll, flat):
    p = random_problem(N, 96, 80, N, noll, defocus_max=8.0, flat=flat, target_range=(0.5, 1.0))
    h = _holo(p)
    _, _, _, met = _run_wgs(h, p, 12)
    Z, C, A = oracle_inputs(p)
    res = wgs.run(A, p.phase0, C, Z, p.target, 12, workers=4)
    assert abs(float(met[0].item()) - res.uniformity) <= UNIF_TOL, (met[0].item(), res.uniformity)


@pytest.mark.parametrize("feedback", [0.0, 0.7, 2.0])
def test_wgs_variants_match_oracle(feedback):
    """Feedback exponent p, then phase fixing: 6 plain iterations store the
    spot phases, 6 fixed ones hold them; final uniformity vs the oracle."""
    p = random_problem(41, 96, 80, 37, list(range(2, 12)), defocus_max=6.0, target_range=(0.5, 1.0))
    h = _holo(p)
    Z, C, A = oracle_inputs(p)
    h.set_wgs_options(feedback=feedback)
    ph, ww, _, met = _run_wgs(h, p, 6)
    res = wgs.run(A, p.phase0, C, Z, p.target, 6, workers=4, feedback=feedback)
    assert abs(float(met[0].item()) - res.uniformity) <= UNIF_TOL, (met[0].item(), res.uniformity)
    h.set_wgs_options(feedback=feedback, fix_phase=True)
    _, _, _, met2 = _run_wgs(h, p, 6, phase=ph.cpu().numpy(), w=ww.cpu().numpy())
    res2 = wgs.run(A, ph.cpu().numpy().astype(np.float64), C, Z, p.target, 6, weights0=ww.cpu().numpy(), workers=4,
                   feedback=feedback, fixed_psi=res.psi)
    assert abs(float(met2[0].item()) - res2.uniformity) <= UNIF_TOL, (met2[0].item(), res2.uniformity)
    h.set_wgs_options()   # back to the plain rule


def test_wgs_resume_is_bitwise():
    p = random_problem(3, 128, 128, 64, list(range(2, 12)))
    h = _holo(p)
    ph_a, w_a, E_a, _ = _run_wgs(h, p, 6)
    ph_b, w_b, _, _ = _run_wgs(h, p, 3)
    ph_c, w_c, E_c, _ = _run_wgs(h, p, 3, phase=ph_b.cpu().numpy(), w=w_b.cpu().numpy())
    assert torch.equal(ph_a, ph_c) and torch.equal(w_a, w_c) and torch.equal(E_a, E_c)
    # iters = 0 and 1 (non-graph path) agree with the graph path's prefix
    ph_1, w_1, _, _ = _run_wgs(h, p, 1)
    ph_2, w_2, _, _ = _run_wgs(h, p, 1, phase=ph_1.cpu().numpy(), w=w_1.cpu().numpy())
    ph_g, w_g, _, _ = _run_wgs(h, p, 2)
    assert torch.equal(ph_2, ph_g) and torch.equal(w_2, w_g)


@pytest.mark.parametrize("nx,ny,N,noll", [(72, 56, 40, list(range(2, 12))), (130, 97, 600, list(range(2, 13))),
                                          (64, 64, 9, [2, 3, 4, 5, 6])])
def test_grad_matches_oracle(nx, ny, N, noll):
    _check_grad(nx, ny, N, noll)


# Both kernel families of the coefficient-gradient moments: odd and even D
# (the tensor-core pass packs modes in pairs), the tilt-exact operand layout
# (D = 11 with Noll 2, 3), a partial last block of 128 spots, spot blocks
# split between CTAs (many units) and tiny ranges (2 units per CTA).
@pytest.mark.parametrize("variant", [1, 2])
@pytest.mark.parametrize("nx,ny,N,noll", [(96, 80, 200, list(range(2, 12))), (130, 97, 600, list(range(2, 13))),
                                          (32, 32, 64, [4, 5, 6, 7]), (100, 70, 130, [2, 3, 4, 5, 6]),
                                          (200, 150, 1000, [4, 5])])
def test_grad_coeff_both_families(nx, ny, N, noll, variant):
    tc = _check_grad(nx, ny, N, noll, variant=variant)
    assert tc == (variant == 2)


def _check_grad(nx, ny, N, noll, variant=0):
    p = random_problem(nx + N, nx, ny, N, noll, defocus_max=5.0, target_range=(0.5, 1.5))
    h = _holo(p)
    if variant:
        h.set_variant(variant)
    Z, C, A = oracle_inputs(p)
    phase = p.phase0.astype(np.float64).ravel()
    E = transform.forward(transform.field(A, phase), C, Z)
    gE = ograd.grad_E(E, p.target).astype(np.complex64)
    dph_ref, dC_ref = ograd.backward(A, phase, C, Z, gE.astype(np.complex128))
    dph, dC = h.grad(torch.from_numpy(p.phase0).cuda(), torch.from_numpy(gE).cuda())
    dph = dph.cpu().numpy().astype(np.float64).ravel()
    dC = dC.cpu().numpy().astype(np.float64)
    r1 = np.linalg.norm(dph - dph_ref) / np.linalg.norm(dph_ref)
    r2 = np.linalg.norm(dC - dC_ref) / np.linalg.norm(dC_ref)
    assert r1 <= GRAD_TOL and r2 <= GRAD_TOL, (r1, r2)
    return bool(h.launch_info()["kernels"] & 8)


def test_grad_tensor_cores_at_large_local_phases():
    """The gradient's tensor-core passes feed the MUFU the tile-local phase
    unreduced (they run once per gradient, not inside a loop): strong tilts
    (0.45 Nyquist), defocus up to 20 rad and larger higher modes give the
    largest local phases per 32 x 32 tile, where that error is largest. It
    stays a decade inside the gradient tolerance."""
    p = random_problem(77, 256, 224, 300, list(range(2, 13)), aberr_sigma=2.0, defocus_max=20.0,
                       target_range=(0.5, 1.5))
    h = _holo(p)
    h.set_variant(2)
    Z, C, A = oracle_inputs(p)
    phase = p.phase0.astype(np.float64).ravel()
    E = transform.forward(transform.field(A, phase), C, Z)
    gE = ograd.grad_E(E, p.target).astype(np.complex64)
    dph_ref, dC_ref = ograd.backward(A, phase, C, Z, gE.astype(np.complex128))
    dph, dC = h.grad(torch.from_numpy(p.phase0).cuda(), torch.from_numpy(gE).cuda())
    assert h.launch_info()["kernels"] & 10 == 10   # tensor-core adjoint and moment pass
    dph = dph.cpu().numpy().astype(np.float64).ravel()
    dC = dC.cpu().numpy().astype(np.float64)
    r1 = np.linalg.norm(dph - dph_ref) / np.linalg.norm(dph_ref)
    r2 = np.linalg.norm(dC - dC_ref) / np.linalg.norm(dC_ref)
    print(f"large local phases: dL/dphi {r1:.3g}, dL/dC {r2:.3g}, max |C.Z| {np.abs(C @ Z).max():.3g}")
    assert r1 <= 0.1 * GRAD_TOL and r2 <= 0.1 * GRAD_TOL, (r1, r2)
