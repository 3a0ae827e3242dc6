"""The FMA-pipe kernels' register-image basis (4 D bytes per pixel) is
released when every transform of a handle runs on the tensor cores, and
rebuilt from the monomial tables when a later kernel choice needs it; a
handle made from a caller's basis keeps it. Results stay equal to the
oracle's either way."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from gpu_helpers import assert_close, oracle_forward  # noqa: E402
from oracle import zernike  # noqa: E402
from workloads import random_problem  # noqa: E402

pytestmark = pytest.mark.gpu


def test_basis_image_released_and_rebuilt():
    from paper_2505_08777_gb300 import Hologram
    p = random_problem(61, 256, 192, 300, list(range(2, 12)), defocus_max=5.0)
    amp, coeff = torch.from_numpy(p.amp).cuda(), torch.from_numpy(p.coeff).cuda()
    h = Hologram(amp, coeff, noll=p.noll)
    assert h.launch_info()["kernels"] & 14 == 14          # tensor-core forward, adjoint, moments
    image = (256 // 32) * (192 // 32) * 1024 * p.D * 4     # tiles x pixels x D fp32
    lean = h.workspace_bytes()
    phase = torch.from_numpy(p.phase0).cuda()
    Z = zernike.basis(p.nx, p.ny, p.noll)
    E_ref = oracle_forward(p, p.phase0, Z)
    assert_close(h.forward(phase).cpu().numpy(), E_ref, what="tensor-core forward")
    h.set_variant(1)                                      # FMA-pipe kernels: the image is rebuilt
    assert h.workspace_bytes() == lean + image
    assert_close(h.forward(phase).cpu().numpy(), E_ref, what="FMA forward on the rebuilt image")
    h.set_variant(0)
    assert_close(h.forward(phase).cpu().numpy(), E_ref, what="back to automatic")
    # a caller's basis cannot be rebuilt, so its image is kept
    basis = torch.from_numpy(Z.astype(np.float32).reshape(p.D, p.ny, p.nx)).cuda()
    hb = Hologram(amp, coeff, basis=basis)
    assert not hb.launch_info()["kernels"] & 8            # FMA-pipe moments on a caller's basis
    assert_close(hb.forward(phase).cpu().numpy(), E_ref, what="caller's basis")
    gE = torch.from_numpy((np.random.default_rng(1).normal(size=p.N) * 1e-3).astype(np.complex64)).cuda()
    _, dC = hb.grad(phase, gE)
    assert torch.isfinite(dC).all()
