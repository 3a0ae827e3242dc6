"""GPU parity of the conjugate-gradient phase refinement.

From the same float32 start (the oracle's WGS phase) the device loop must
follow the oracle's iteration: the loss history agrees closely over the
first iterations (both sides take the same line-search and PR+ decisions)
and the refined phase after one iteration agrees as unit phasors; over a
longer run fp32 and fp64 trajectories separate, so the final loss is
compared loosely and both must have lowered it. Both kernel families; zero
iterations report the loss only; a replayed graph is bitwise repeatable.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cg, grad, transform, wgs, zernike  # noqa: E402
from workloads import random_problem  # noqa: E402

pytestmark = pytest.mark.gpu


def _setup(seed=21, nx=96, ny=80, N=24):
    from paper_2505_08777_gb300 import Hologram
    p = random_problem(seed, nx, ny, N, [2, 3, 4, 5, 6, 7], aberr_sigma=0.4, target_range=(1.0, 1.0))
    Z = zernike.basis(p.nx, p.ny, p.noll)
    C = p.coeff.astype(np.float64)
    A = p.amp.astype(np.float64).ravel()
    res = wgs.run(A, p.phase0.astype(np.float64).ravel(), C, Z, p.target, 8, workers=4)
    phi0 = res.phase.astype(np.float32)
    t = (p.target.astype(np.float64) ** 2 / np.mean(p.target.astype(np.float64) ** 2)).astype(np.float32)
    h = Hologram(torch.from_numpy(p.amp).cuda(), torch.from_numpy(p.coeff).cuda(), noll=p.noll)
    return p, Z, C, A, phi0, t, h


@pytest.mark.parametrize("variant", [1, 2])
def test_cg_follows_the_oracle(variant):
    p, Z, C, A, phi0, t, h = _setup()
    h.set_variant(variant)
    ph = torch.from_numpy(phi0.reshape(p.ny, p.nx).copy()).cuda()
    L1 = h.cg_refine(ph, torch.from_numpy(t).cuda(), 1).cpu().numpy().astype(np.float64)
    phi_ref, Lr = cg.refine(A, phi0.astype(np.float64), C, Z, t.astype(np.float64), 1, theta=0.05, workers=4)
    assert np.allclose(L1, Lr, rtol=2e-4), (L1, Lr)
    w = A * A
    dphi = np.angle(np.exp(1j * (ph.cpu().numpy().astype(np.float64).ravel() - phi_ref)))
    assert np.sqrt(np.sum(w * dphi ** 2) / np.sum(w)) < 1e-3
    # a longer run: the same early history, a similar end point
    ph = torch.from_numpy(phi0.reshape(p.ny, p.nx).copy()).cuda()
    L = h.cg_refine(ph, torch.from_numpy(t).cuda(), 12).cpu().numpy().astype(np.float64)
    _, Lr = cg.refine(A, phi0.astype(np.float64), C, Z, t.astype(np.float64), 12, theta=0.05, workers=4)
    assert np.allclose(L[:3], Lr[:3], rtol=2e-3), (L[:3], Lr[:3])
    assert L[-1] < 0.5 * L[0] and Lr[-1] < 0.5 * Lr[0]
    assert abs(L[-1] - Lr[-1]) <= 0.25 * Lr[-1] + 1e-3 * Lr[0], (L[-1], Lr[-1])
    # the reported loss is the loss of the returned phase
    E = transform.forward(transform.field(A, ph.cpu().numpy().astype(np.float64).ravel()), C, Z)
    assert abs(grad.loss_from_E(E, t.astype(np.float64)) - L[-1]) <= 1e-3 * L[0]
    assert wgs.uniformity(E, p.target) > wgs.uniformity(transform.forward(transform.field(A, phi0), C, Z), p.target)


def test_cg_zero_iterations_and_replay():
    p, Z, C, A, phi0, t, h = _setup(seed=5)
    td = torch.from_numpy(t).cuda()
    ph = torch.from_numpy(phi0.reshape(p.ny, p.nx).copy()).cuda()
    L0 = h.cg_refine(ph, td, 0).cpu().numpy()
    assert torch.equal(ph.cpu(), torch.from_numpy(phi0.reshape(p.ny, p.nx)))
    ref = grad.loss(A, phi0.astype(np.float64), C, Z, t.astype(np.float64))
    assert abs(L0[0] - ref) <= 2e-4 * ref
    outs = []
    for _ in range(2):
        ph = torch.from_numpy(phi0.reshape(p.ny, p.nx).copy()).cuda()
        L = h.cg_refine(ph, td, 5)
        outs.append((ph.clone(), L.clone()))
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])
