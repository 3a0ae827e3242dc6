"""Pixel-sharded transforms on band handles (Methods, "Computational
Scaling": each pixel's kernel values depend only on that pixel and the
global N x D matrix, so the forward is a sum over pixel blocks and the
adjoint is local per pixel).

Two or three band handles of one grid on one device stand for the ranks of
a multi-GPU run. Their forwards summed must equal the full grid's handle
and the oracle; their adjoints must tile the full grid's adjoint; their
coefficient gradients summed must equal the full gradient (moment pass
over tile polynomials in the full grid's coordinates); and a sharded WGS
(summed forwards, replicated update, local adjoints) must reach the
oracle's final uniformity. The grids are chosen so that the band's own
rows would give another unit-disk radius and centre than the full grid's
(nx > ny_full and nx < ny_full), and the D = 11 cases use the tilt-exact
operand layout, whose spot rows carry tilt / R.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from gpu_helpers import GRAD_TOL, UNIF_TOL, assert_close, oracle_inputs  # noqa: E402
from oracle import grad as ograd  # noqa: E402
from oracle import transform, wgs  # noqa: E402
from workloads import random_problem  # noqa: E402

pytestmark = pytest.mark.gpu

CASES = [  # nx, ny_full, N, noll, ranks, variant
    (256, 160, 300, list(range(2, 12)), 3, 0),
    (150, 200, 300, list(range(2, 12)), 2, 1),
    (150, 200, 300, list(range(2, 13)), 3, 2),
    (96, 130, 40, list(range(2, 13)), 2, 0),
]


def _setup(nx, ny, N, noll, ranks, variant):
    from paper_2505_08777_gb300 import Hologram
    from paper_2505_08777_gb300.shard import band_holograms, row_blocks
    p = random_problem(nx + 7 * N, nx, ny, N, noll, defocus_max=6.0, target_range=(0.5, 1.0))
    amp = torch.from_numpy(p.amp).cuda()
    coeff = torch.from_numpy(p.coeff).cuda()
    full = Hologram(amp, coeff, noll=p.noll)
    blocks = row_blocks(ny, ranks)
    bands = band_holograms(amp, coeff, p.noll, ny, blocks)
    for h in [full] + bands:
        if variant:
            h.set_variant(variant)
    return p, full, bands, [b for b in blocks if b[1] > b[0]]


@pytest.mark.parametrize("nx,ny,N,noll,ranks,variant", CASES)
def test_band_transforms_sum_and_tile_to_the_full_grid(nx, ny, N, noll, ranks, variant):
    p, full, bands, blocks = _setup(nx, ny, N, noll, ranks, variant)
    for h, (r0, r1) in zip(bands, blocks):
        assert h.band_info()[:2] == (r0, ny)
    assert abs(sum(h.band_info()[2] for h in bands) - full.band_info()[2]) <= 1e-6 * full.band_info()[2]
    Z, C, A = oracle_inputs(p)
    phase = torch.from_numpy(p.phase0).cuda()
    # forward: partial fields over each band's rows sum to the full field
    E = sum(h.forward(phase[r0:r1].contiguous()).cpu().numpy().astype(np.complex128)
            for h, (r0, r1) in zip(bands, blocks))
    E_full = full.forward(phase).cpu().numpy()
    E_ref = transform.forward(transform.field(A, p.phase0), C, Z)
    assert_close(E, E_ref, what="summed band forwards vs oracle")
    assert_close(E, E_full, what="summed band forwards vs full handle")
    # adjoint: each band's output is its rows of the full adjoint
    rng = np.random.default_rng(N)
    y = (rng.normal(size=N) + 1j * rng.normal(size=N)).astype(np.complex64)
    yt = torch.from_numpy(y).cuda()
    g_full, _ = full.adjoint(yt)
    g = torch.cat([h.adjoint(yt)[0] for h in bands], 0).cpu().numpy()
    g_ref = transform.adjoint(y.astype(np.complex128), C, Z)
    assert_close(g, g_ref, what="tiled band adjoints vs oracle")
    assert_close(g, g_full.cpu().numpy(), what="tiled band adjoints vs full handle")
    # gradient: dphase tiles, dC sums over the bands
    gE = ograd.grad_E(E_ref, p.target).astype(np.complex64)
    gEt = torch.from_numpy(gE).cuda()
    dph_ref, dC_ref = ograd.backward(A, p.phase0, C, Z, gE.astype(np.complex128))
    parts = [h.grad(phase[r0:r1].contiguous(), gEt) for h, (r0, r1) in zip(bands, blocks)]
    dph = torch.cat([a for a, _ in parts], 0).cpu().numpy().astype(np.float64).ravel()
    dC = sum(b.cpu().numpy().astype(np.float64) for _, b in parts)
    r1 = np.linalg.norm(dph - dph_ref) / np.linalg.norm(dph_ref)
    r2 = np.linalg.norm(dC - dC_ref) / np.linalg.norm(dC_ref)
    assert r1 <= GRAD_TOL and r2 <= GRAD_TOL, (r1, r2)
    for h in bands:
        h.check()


@pytest.mark.parametrize("nx,ny,N,noll,ranks,variant", CASES[:2] + CASES[3:])
def test_sharded_wgs_matches_oracle(nx, ny, N, noll, ranks, variant):
    from paper_2505_08777_gb300.shard import sharded_wgs
    p, full, bands, blocks = _setup(nx, ny, N, noll, ranks, variant)
    iters = 8
    ph0 = torch.from_numpy(p.phase0).cuda()
    phases = [ph0[r0:r1].clone() for r0, r1 in blocks]
    w = torch.from_numpy(p.target).cuda().clone()
    T = torch.from_numpy(p.target).cuda()
    sum_a2 = sum(h.band_info()[2] for h in bands)
    E, met = sharded_wgs(bands, phases, w, T, iters, sum_a2=sum_a2)
    torch.cuda.synchronize()
    Z, C, A = oracle_inputs(p)
    res = wgs.run(A, p.phase0, C, Z, p.target, iters, workers=4)
    met = met.cpu().numpy().astype(np.float64)
    assert abs(met[0] - res.uniformity) <= UNIF_TOL, (met[0], res.uniformity)
    # the reported metrics are the oracle formulas on the sharded loop's own field and phase
    Eg = E.cpu().numpy().astype(np.complex128)
    assert abs(met[0] - wgs.uniformity(Eg, p.target)) <= 1e-5
    assert abs(met[1] - wgs.efficiency(Eg, p.amp)) <= 1e-5 * max(1.0, wgs.efficiency(Eg, p.amp))
    ph = torch.cat(phases, 0).cpu().numpy()
    assert_close(Eg, transform.forward(transform.field(A, ph), C, Z), what="final field vs oracle of final phase")
