"""GPU parity at the size limits, on sampled outputs.

An 8192 x 8192 grid (its tensor-core pixel-row image is 8.6 GB, past every
32-bit byte offset) with a ragged N = 130, and N = 2^20 spots (the largest
the handle accepts) on a 32 x 32 grid. Forward fields of sampled spots are
summed by the oracle over all pixels in chunks (the basis evaluated per
chunk); adjoint values at sampled pixels need the basis there only.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from gpu_helpers import assert_close, basis_at  # noqa: E402
from workloads import random_problem  # noqa: E402

pytestmark = pytest.mark.gpu


def _holo(p):
    from paper_2505_08777_gb300 import Hologram
    return Hologram(torch.from_numpy(p.amp).cuda(), torch.from_numpy(p.coeff).cuda(), noll=p.noll)


def _forward_ref(p, phase, spots, chunk=1 << 21):
    """E at the sampled spots, summed over every pixel in chunks (complex128)."""
    M = p.nx * p.ny
    C = p.coeff.astype(np.float64)[spots]
    A = p.amp.astype(np.float64).ravel()
    ph = np.asarray(phase, np.float64).ravel()
    E = np.zeros(len(spots), np.complex128)
    for m0 in range(0, M, chunk):
        pix = np.arange(m0, min(M, m0 + chunk))
        Z = basis_at(p, pix)
        E += np.exp(-1j * (C @ Z)) @ (A[pix] * np.exp(1j * ph[pix]))
    return E


def _adjoint_ref(p, y, pix):
    Z = basis_at(p, pix)
    return np.exp(1j * (p.coeff.astype(np.float64) @ Z)).T @ y.astype(np.complex128)


@pytest.mark.parametrize("nx,ny,N", [(8192, 8192, 130), (32, 32, 1 << 20)], ids=["grid_8192x8192_N130", "N_2^20"])
def test_size_limits_sampled(nx, ny, N):
    p = random_problem(11, nx, ny, N, list(range(2, 12)), defocus_max=5.0)
    h = _holo(p)
    ph = torch.from_numpy(p.phase0).cuda()
    E = h.forward(ph).cpu().numpy()
    rng = np.random.default_rng(3)
    spots = np.unique(np.concatenate([[0, N - 1], rng.integers(0, N, 6)]))
    assert_close(E[spots], _forward_ref(p, p.phase0, spots), what=f"forward {nx}x{ny} N={N}")
    y = (rng.normal(size=N) + 1j * rng.normal(size=N)).astype(np.complex64)
    g, _ = h.adjoint(torch.from_numpy(y).cuda())
    g = g.cpu().numpy().ravel()
    pix = np.unique(np.concatenate([[0, nx * ny - 1], rng.integers(0, nx * ny, 200)]))
    assert_close(g[pix], _adjoint_ref(p, y, pix), what=f"adjoint {nx}x{ny} N={N}")
    del h
    torch.cuda.empty_cache()
