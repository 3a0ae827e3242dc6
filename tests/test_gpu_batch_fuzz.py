"""Randomised parity of the batched form: weighted GS (Sec. II; Methods) for
seeded batches of 2-8 uneven holograms in one CUDA graph.

Each batch draws its members (grids 8..159 px a side with aspect ratio at
most 3, 1..399 spots, a Noll set, Gaussian or flat illumination, a defocus
range); a kernel family (automatic, FMA pipe, tensor cores) and a
standalone threshold go with the batch (both by batch index). The batch
runs ITERS - 1 iterations, then one more, and every member is checked
  * against one oracle WGS iteration from the GPU's state after ITERS - 1
    (phase and weights): uniformity within 1e-3, efficiency and sum |E|^2
    within 1e-3 relative. One iteration at a time, because the weight
    feedback and arg g amplify fp32 against fp64 differences from one
    iteration to the next on dense problems (N close to M), so
    multi-iteration trajectories have no fixed tolerance;
  * for self-consistency: the reported uniformity equals the oracle formula
    on the field of the GPU's own final phase, within 1e-4;
  * standalone members (N M at or above the threshold) bit for bit against
    the single-hologram loop of the same family on their own handle, run
    as the same two calls.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from gpu_helpers import UNIF_TOL, oracle_inputs  # noqa: E402
from oracle import transform, wgs  # noqa: E402
from workloads import random_problem  # noqa: E402

pytestmark = pytest.mark.gpu

N_BATCHES = 8
ITERS = 3
DEFAULT_SOLO_TERMS = 1 << 22


def _member(rng, seed):
    while True:
        nx, ny = int(rng.integers(8, 160)), int(rng.integers(8, 160))
        if max(nx, ny) <= 3 * min(nx, ny):
            break
    N = int(rng.integers(1, 400))
    if rng.random() < 0.5:
        noll = sorted(rng.choice(np.arange(2, 13), size=int(rng.integers(1, 11)), replace=False).tolist())
    else:
        noll = list(range(2, 2 + int(rng.integers(1, 11))))
    return random_problem(seed, nx, ny, N, noll, defocus_max=float(rng.uniform(0, 6)), flat=bool(rng.random() < 0.3),
                          target_range=(0.5, 1.0))


def _case(k):
    rng = np.random.default_rng([20261204, k])
    ps = [_member(rng, 9000 + 100 * k + i) for i in range(int(rng.integers(2, 9)))]
    # family and threshold kind by batch index, so that 8 batches cover them
    return ps, k % 3, [None, 0, 1 << 20][(k // 3) % 3]


def _tensors(p):
    return torch.from_numpy(p.amp).cuda(), torch.from_numpy(p.coeff).cuda(), p.noll


@pytest.mark.parametrize("k", range(N_BATCHES))
def test_batch_fuzz(k):
    from paper_2505_08777_gb300 import Batch, Hologram
    from paper_2505_08777_gb300._lib import AshError
    ps, variant, solo_terms = _case(k)
    b = Batch([_tensors(p) for p in ps], **({} if solo_terms is None else {"solo_terms": solo_terms}))
    if variant:
        try:
            b.set_variant(variant)
        except AshError:
            # only the tensor-core family can be refused: some member has no
            # tensor-core images with the batch's K-atom count
            assert variant == 2
            variant = 0
    thr = DEFAULT_SOLO_TERMS if solo_terms is None else solo_terms
    solo = [p.N * p.nx * p.ny >= thr for p in ps]
    assert b.info()["standalone"] == sum(solo)

    ph = [torch.from_numpy(p.phase0).cuda().clone() for p in ps]
    w = [torch.from_numpy(p.target).cuda().clone() for p in ps]
    T = [torch.from_numpy(p.target).cuda() for p in ps]
    b.wgs(ph, w, T, ITERS - 1)
    mid = [(x.cpu().numpy().astype(np.float64), v.cpu().numpy().astype(np.float64)) for x, v in zip(ph, w)]
    met = b.wgs(ph, w, T, 1).cpu().numpy()

    for i, p in enumerate(ps):
        Z, C, A = oracle_inputs(p)
        what = f"member {i}: {p.nx}x{p.ny} N={p.N} noll={p.noll} variant={variant} solo={solo[i]}"
        assert float(np.abs(C @ Z).max()) <= 2.5e3, what
        res = wgs.run(A, mid[i][0], C, Z, p.target, 1, weights0=mid[i][1], workers=4)
        assert abs(met[i, 0] - res.uniformity) <= UNIF_TOL, (what, met[i, 0], res.uniformity)
        assert abs(met[i, 1] - res.efficiency) <= 1e-3 * res.efficiency, (what, met[i, 1], res.efficiency)
        s2 = float(np.sum(np.abs(res.E) ** 2))
        assert abs(met[i, 2] - s2) <= 1e-3 * s2, (what, met[i, 2], s2)
        E_own = transform.forward(transform.field(A, ph[i].cpu().numpy()), C, Z, workers=4)
        assert abs(met[i, 0] - wgs.uniformity(E_own, p.target)) <= 1e-4, what
        if solo[i]:
            h = Hologram(*_tensors(p))
            if variant:
                h.set_variant(variant)
            ph1 = torch.from_numpy(p.phase0).cuda().clone()
            w1 = torch.from_numpy(p.target).cuda().clone()
            h.wgs(ph1, w1, T[i], ITERS - 1)
            _, met1 = h.wgs(ph1, w1, T[i], 1)
            torch.cuda.synchronize()
            assert torch.equal(ph[i], ph1) and torch.equal(w[i], w1), what
            assert np.array_equal(met[i], met1.cpu().numpy()), what


def test_batch_fuzz_draw_covers_families_and_thresholds():
    """The seeded draw spans every family, every threshold kind and both
    standalone and persistent members."""
    variants, thresholds, n_solo, n_group = set(), set(), 0, 0
    for k in range(N_BATCHES):
        ps, variant, solo_terms = _case(k)
        variants.add(variant)
        thresholds.add(solo_terms)
        thr = DEFAULT_SOLO_TERMS if solo_terms is None else solo_terms
        for p in ps:
            if p.N * p.nx * p.ny >= thr:
                n_solo += 1
            else:
                n_group += 1
    assert variants == {0, 1, 2} and thresholds == {None, 0, 1 << 20}
    assert n_solo > 0 and n_group > 0
