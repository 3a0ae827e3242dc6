"""Batched uneven form (ash_batch_*), in both kernel families (1: FMA-pipe
kernels, 2: tensor-core kernels): parity with the oracle and with the
per-hologram path of the same family, determinism, launch-shape
independence, autotuner cache."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from gpu_helpers import UNIF_TOL, oracle_inputs  # noqa: E402
from oracle import transform, wgs  # noqa: E402
from workloads import random_problem  # noqa: E402

pytestmark = pytest.mark.gpu

SHAPES = [  # (nx, ny, N, noll, flat)
    (96, 64, 37, list(range(2, 12)), False),
    (40, 72, 5, [2, 3, 4, 5, 6], True),
    (130, 97, 300, list(range(2, 13)), True),
    (64, 64, 12, [2, 3], False),
    (33, 45, 70, list(range(2, 10)), False),
]


def _problems(seed0=30):
    return [random_problem(seed0 + k, nx, ny, N, noll, defocus_max=6.0, flat=flat, target_range=(0.5, 1.0))
            for k, (nx, ny, N, noll, flat) in enumerate(SHAPES)]


VARIANTS = [1, 2]


def _batch(ps, variant=0):
    from paper_2505_08777_gb300 import Batch
    b = Batch([(torch.from_numpy(p.amp).cuda(), torch.from_numpy(p.coeff).cuda(), p.noll) for p in ps])
    if variant:
        b.set_variant(variant)
    return b


def _state(ps):
    ph = [torch.from_numpy(p.phase0).cuda().clone() for p in ps]
    w = [torch.from_numpy(p.target).cuda().clone() for p in ps]
    T = [torch.from_numpy(p.target).cuda() for p in ps]
    return ph, w, T


@pytest.mark.parametrize("variant", VARIANTS)
def test_batch_wgs_matches_oracle_per_hologram(variant):
    ps = _problems()
    b = _batch(ps, variant)
    ph, w, T = _state(ps)
    met = b.wgs(ph, w, T, 10).cpu().numpy()
    for k, p in enumerate(ps):
        Z, C, A = oracle_inputs(p)
        res = wgs.run(A, p.phase0, C, Z, p.target, 10)
        assert abs(met[k, 0] - res.uniformity) <= UNIF_TOL, (k, met[k, 0], res.uniformity)
        # the reported metric is the oracle formula on the GPU's own final phase
        E = transform.forward(transform.field(A, ph[k].cpu().numpy()), C, Z)
        assert abs(met[k, 0] - wgs.uniformity(E, p.target)) <= 1e-4


@pytest.mark.parametrize("variant", VARIANTS)
def test_batch_one_iteration_equals_single_path(variant):
    from paper_2505_08777_gb300 import Hologram
    ps = _problems(50)
    b = _batch(ps, variant)
    ph, w, T = _state(ps)
    b.wgs(ph, w, T, 1)
    for k, p in enumerate(ps):
        h = Hologram(torch.from_numpy(p.amp).cuda(), torch.from_numpy(p.coeff).cuda(), noll=p.noll)
        h.set_variant(variant)   # same kernel family: the same sums up to summation order
        ph1 = torch.from_numpy(p.phase0).cuda().clone()
        w1 = torch.from_numpy(p.target).cuda().clone()
        h.wgs(ph1, w1, T[k], 1)
        torch.cuda.synchronize()
        np.testing.assert_allclose(w[k].cpu().numpy(), w1.cpu().numpy(), rtol=1e-5)
        amp = p.amp.ravel()
        u = np.exp(1j * ph[k].cpu().numpy().ravel().astype(np.float64))
        u1 = np.exp(1j * ph1.cpu().numpy().ravel().astype(np.float64))
        assert np.linalg.norm(amp * (u - u1)) <= 1e-4 * np.linalg.norm(amp)


@pytest.mark.parametrize("variant", VARIANTS)
def test_batch_deterministic_and_grid_independent(variant):
    ps = _problems(70)
    b = _batch(ps, variant)
    outs = []
    for grid in (None, None, 7, 1, 3 * b.info()["resident_ctas"]):
        if grid is not None:
            b.set_grid(grid)
        ph, w, T = _state(ps)
        met = b.wgs(ph, w, T, 3)
        outs.append(([x.clone() for x in ph], met.clone()))
    # same launch shape twice: bitwise
    assert all(torch.equal(a, c) for a, c in zip(outs[0][0], outs[1][0]))
    assert torch.equal(outs[0][1], outs[1][1])
    # other launch shapes: same up to fp32 summation order
    for ph_g, met_g in outs[2:]:
        assert torch.allclose(met_g[:, 0], outs[0][1][:, 0], atol=1e-4)
        for a, c, p in zip(ph_g, outs[0][0], ps):
            amp = torch.from_numpy(p.amp).cuda()
            d = amp * (torch.polar(torch.ones_like(a), a) - torch.polar(torch.ones_like(c), c))
            assert float(d.abs().norm() / amp.norm()) <= 1e-3


@pytest.mark.parametrize("variant", VARIANTS)
def test_batch_autotuner_picks_and_caches(tmp_path, variant):
    ps = _problems(90)
    b = _batch(ps, variant)
    ph, _, _ = _state(ps)
    cache = str(tmp_path / "tune.txt")
    g = b.tune(ph, cache)
    assert g >= 0 and os.path.exists(cache)
    lines = [line.split() for line in open(cache).read().split("\n") if line]
    assert len(lines) == 1 and int(lines[0][3]) == g and int(lines[0][2]) == variant
    solo = int(lines[0][1])
    assert b.info()["standalone"] == sum(p.N * p.nx * p.ny >= solo for p in ps)
    b2 = _batch(ps, variant)
    assert b2.tune(ph, cache) == g            # read from the cache
    assert b2.info()["grid"] == g and b2.info()["standalone"] == b.info()["standalone"]
    if g == 0:
        return
    if variant == 1:   # forward + reduction, update, adjoint (+ fix-up); final forward, metrics
        assert b.launches(5) in (5 * 4 + 3, 5 * 5 + 3)
    else:              # nearfield images and forward (+ reduction) once, then update, adjoint (+ fix-up), forward (+ reduction)
        assert b.launches(5) in [2 + f + 5 * (1 + a + f) for f in (1, 2) for a in (1, 2)]


def test_batch_automatic_family_is_tensor_core():
    b = _batch(_problems(110))
    info = b.info()
    b.set_variant(2)
    assert b.info()["resident_ctas"] == info["resident_ctas"]


def test_batch_rejects_large_D():
    from paper_2505_08777_gb300 import Batch
    p = random_problem(1, 32, 32, 4, list(range(2, 16)))
    with pytest.raises(Exception):
        Batch([(torch.from_numpy(p.amp).cuda(), torch.from_numpy(p.coeff).cuda(), p.noll)])


@pytest.mark.parametrize("solo_terms", [0, 200_000])
def test_batch_standalone_members(solo_terms):
    # members at or above the threshold run the single-hologram loop inside
    # the batch's graph: bit for bit the result of ash_wgs_iterate on their
    # own handle; the others stay in the persistent group
    from paper_2505_08777_gb300 import Batch, Hologram, _lib
    ps = _problems(90)
    b = Batch([(torch.from_numpy(p.amp).cuda(), torch.from_numpy(p.coeff).cuda(), p.noll) for p in ps],
              solo_terms=solo_terms)
    solo = [p.N * p.nx * p.ny >= solo_terms for p in ps]
    assert 0 < sum(solo) and (solo_terms == 0 or not all(solo))
    info = b.info()
    assert info["count"] == len(ps) and info["standalone"] == sum(solo)
    if all(solo):
        assert info["grid"] == 0
        # the tuner may regroup (it chooses the standalone threshold); its grid is the batch's
        assert b.tune([torch.from_numpy(p.phase0).cuda() for p in ps]) == b.info()["grid"]
        b = Batch([(torch.from_numpy(p.amp).cuda(), torch.from_numpy(p.coeff).cuda(), p.noll) for p in ps],
                  solo_terms=solo_terms)
    ph, w, T = _state(ps)
    met = b.wgs(ph, w, T, 4)
    lib = _lib.load()
    n_solo_launches = 0
    for k, p in enumerate(ps):
        h = Hologram(torch.from_numpy(p.amp).cuda(), torch.from_numpy(p.coeff).cuda(), noll=p.noll)
        ph1 = torch.from_numpy(p.phase0).cuda().clone()
        w1 = torch.from_numpy(p.target).cuda().clone()
        _, met1 = h.wgs(ph1, w1, T[k], 4)
        torch.cuda.synchronize()
        if solo[k]:
            assert torch.equal(ph[k], ph1) and torch.equal(w[k], w1) and torch.equal(met[k], met1)
            n_solo_launches += int(lib.ash_wgs_launches(h.handle, 4))
        else:
            assert abs(float(met[k, 0]) - float(met1[0])) <= UNIF_TOL
    if all(solo):
        assert b.launches(4) == n_solo_launches
    else:
        assert b.launches(4) > n_solo_launches


def test_batch_rejects_negative_threshold():
    from paper_2505_08777_gb300 import Batch
    from paper_2505_08777_gb300._lib import AshError
    p = _problems(95)[0]
    with pytest.raises(AshError):
        Batch([(torch.from_numpy(p.amp).cuda(), torch.from_numpy(p.coeff).cuda(), p.noll)], solo_terms=-1)


def test_batch_autotuner_tunes_family_and_grouping(tmp_path):
    # automatic family: the tuner chooses the grouping, the persistent
    # group's kernel family and its CTA count; the tuned batch still solves
    # every member as the oracle does
    ps = _problems(95)
    b = _batch(ps)
    ph, w, T = _state(ps)
    cache = str(tmp_path / "tune.txt")
    g = b.tune(ph, cache)
    key, solo, fam, grid = open(cache).read().split()
    assert key.startswith("sm") and int(fam) in (0, 1) and int(grid) == g
    assert b.info()["standalone"] == sum(p.N * p.nx * p.ny >= int(solo) for p in ps)
    ph, w, T = _state(ps)
    met = b.wgs(ph, w, T, 10).cpu().numpy()
    for k, p in enumerate(ps):
        Z, C, A = oracle_inputs(p)
        res = wgs.run(A, p.phase0, C, Z, p.target, 10, workers=4)
        assert abs(float(met[k, 0]) - res.uniformity) <= UNIF_TOL, (k, met[k, 0], res.uniformity)
