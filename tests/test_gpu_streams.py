"""Handles used at the same time: several holograms, each on its own CUDA
stream, enqueued interleaved from one host thread and from several host
threads at once, give bit for bit the results of running them one at a
time on the default stream. Each handle owns its workspace and its loop
graphs (captured in thread-local mode), and every kernel is deterministic,
so nothing but a shared buffer or a capture conflict could change a bit."""
import threading

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from workloads import random_problem  # noqa: E402

pytestmark = pytest.mark.gpu

SHAPES = [  # (nx, ny, N, noll)
    (256, 192, 300, list(range(2, 12))),
    (200, 200, 128, [2, 3, 4, 5, 6, 7]),
    (320, 240, 500, list(range(2, 13))),
    (96, 160, 40, list(range(2, 10))),
]


def _problems():
    return [random_problem(800 + k, *shape, defocus_max=3.0) for k, shape in enumerate(SHAPES)]


def _inputs(p, k):
    rng = np.random.default_rng(900 + k)
    y = (rng.normal(size=p.N) + 1j * rng.normal(size=p.N)).astype(np.complex64)
    return (torch.from_numpy(p.phase0).cuda(), torch.from_numpy(y).cuda(), torch.from_numpy(p.target).cuda())


def _holo(p):
    from paper_2505_08777_gb300 import Hologram
    return Hologram(torch.from_numpy(p.amp).cuda(), torch.from_numpy(p.coeff).cuda(), noll=p.noll)


def _run(h, inputs, stream=None):
    """Forward, adjoint, a 4-iteration WGS loop (a graph) and both gradients;
    allocations, copies and library calls all on `stream` (or the current
    stream)."""
    phase, y, T = inputs
    with torch.cuda.stream(stream if stream is not None else torch.cuda.current_stream()):
        out = [h.forward(phase)]
        out += list(h.adjoint(y, want_field=True, want_phase=True))
        ph, w = phase.clone(), T.clone()
        E, met = h.wgs(ph, w, T, 4)
        out += [ph, w, E, met]
        out += list(h.grad(phase, y))
    return out


def _reference(ps, ins):
    refs = []
    for p, x in zip(ps, ins):
        refs.append([t.clone() for t in _run(_holo(p), x)])
    torch.cuda.synchronize()
    return refs


def _assert_same(got, ref, what):
    assert len(got) == len(ref)
    for i, (a, b) in enumerate(zip(got, ref)):
        assert torch.equal(a, b), f"{what}: output {i} differs"


def test_interleaved_streams_one_thread():
    ps = _problems()
    ins = [_inputs(p, k) for k, p in enumerate(ps)]
    refs = _reference(ps, ins)
    hs = [_holo(p) for p in ps]
    streams = [torch.cuda.Stream() for _ in ps]
    torch.cuda.synchronize()
    # two rounds, so that the second one replays the graphs the first captured
    for _ in range(2):
        outs = [_run(h, x, s) for h, x, s in zip(hs, ins, streams)]
        torch.cuda.synchronize()
        for k, (o, r) in enumerate(zip(outs, refs)):
            _assert_same(o, r, f"hologram {k}")


def test_host_threads_each_with_its_own_handle_and_stream():
    ps = _problems()
    ins = [_inputs(p, k) for k, p in enumerate(ps)]
    refs = _reference(ps, ins)
    hs = [_holo(p) for p in ps]
    streams = [torch.cuda.Stream() for _ in ps]
    torch.cuda.synchronize()
    results, errors = [None] * len(ps), []
    start = threading.Barrier(len(ps))

    def worker(k):
        try:
            start.wait()
            o = [_run(hs[k], ins[k], streams[k]) for _ in range(3)]
            streams[k].synchronize()
            results[k] = o
        except Exception as e:   # noqa: BLE001 -- reported below
            errors.append((k, e))

    threads = [threading.Thread(target=worker, args=(k,)) for k in range(len(ps))]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=300)
    assert not errors, errors
    for k, rounds in enumerate(results):
        assert rounds is not None, f"thread {k} did not finish"
        for i, o in enumerate(rounds):
            _assert_same(o, refs[k], f"thread {k}, round {i}")
