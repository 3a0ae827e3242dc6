"""The kernel-launch counts the library reports (ash_wgs_launches,
ash_batch_wgs_launches: the gpu_launches of bench.py) against the kernel
nodes of the CUDA graphs it actually captured for the same calls
(ash_graph_kernels, ash_batch_graph_kernels), over both kernel families and
shapes with and without split reductions and fix-ups."""
import pytest

torch = pytest.importorskip("torch")

from workloads import random_problem  # noqa: E402

pytestmark = pytest.mark.gpu

CASES = [  # (nx, ny, N, noll)
    (96, 64, 37, list(range(2, 12))),
    (300, 200, 700, list(range(2, 13))),
    (1024, 1024, 400, list(range(2, 12))),
    (64, 64, 5, [2, 3]),
]


def _holo(p, variant):
    from paper_2505_08777_gb300 import Hologram
    h = Hologram(torch.from_numpy(p.amp).cuda(), torch.from_numpy(p.coeff).cuda(), noll=p.noll)
    h.set_variant(variant)
    return h


def _state(p):
    return (torch.from_numpy(p.phase0).cuda().clone(), torch.from_numpy(p.target).cuda().clone(),
            torch.from_numpy(p.target).cuda())


@pytest.mark.parametrize("variant", [0, 1, 2])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_wgs_launch_count_is_the_captured_graph(case, variant):
    nx, ny, N, noll = CASES[case]
    p = random_problem(700 + case, nx, ny, N, noll, defocus_max=4.0)
    h = _holo(p, variant)
    for iters in (2, 7):
        assert h.graph_kernels(iters) == -1
        h.wgs(*_state(p), iters)
        assert h.graph_kernels(iters) == h.wgs_launches(iters) > 0, (iters, h.launch_info())
    h.set_wgs_options(0.7, True)          # drops the cached graphs
    assert h.graph_kernels(7) == -1
    h.wgs(*_state(p), 7)
    assert h.graph_kernels(7) == h.wgs_launches(7)


def test_cg_graph_grows_by_a_fixed_count_per_iteration():
    p = random_problem(720, 128, 96, 50, list(range(2, 12)))
    h = _holo(p, 0)
    t = torch.ones(p.N, device="cuda")
    counts = []
    for iters in (1, 3, 5):
        h.cg_refine(torch.from_numpy(p.phase0).cuda().clone(), t, iters)
        counts.append(h.graph_kernels(-iters))
    assert counts[0] > 0 and counts[2] - counts[1] == counts[1] - counts[0] > 0, counts


@pytest.mark.parametrize("variant", [1, 2])
@pytest.mark.parametrize("solo_terms", [None, 1 << 16])
def test_batch_launch_count_is_the_captured_graph(variant, solo_terms):
    from paper_2505_08777_gb300 import Batch
    ps = [random_problem(740 + k, nx, ny, N, noll, defocus_max=4.0) for k, (nx, ny, N, noll) in enumerate(CASES)]
    kw = {} if solo_terms is None else {"solo_terms": solo_terms}
    b = Batch([(torch.from_numpy(p.amp).cuda(), torch.from_numpy(p.coeff).cuda(), p.noll) for p in ps], **kw)
    b.set_variant(variant)
    states = [_state(p) for p in ps]
    b.wgs([s[0] for s in states], [s[1] for s in states], [s[2] for s in states], 4)
    assert b.graph_kernels(4) == b.launches(4) > 0, (b.info(), b.graph_kernels(4), b.launches(4))
    if solo_terms is not None:
        assert b.info()["standalone"] > 0
