"""The allocation-free forward entry point, called through the C ABI.

ash_forward_noalloc serves callers that cannot allocate device memory (a
host framework that owns all device memory, a real-time control loop that
must not allocate, a plugin handed only pre-allocated buffers). It keeps its
scratch in a fixed array inside the library, shared by every call.

Checked here, each against the oracle's forward (complex128 definition) and
against the handle-based ash_forward on the same inputs and basis:
  * two calls in a row -- a larger problem, then a smaller one, so stale
    scratch from the first call would show up in the second;
  * more tiles than resident CTAs, so each CTA accumulates several tiles
    into its scratch rows (the `*dst + out` chains);
  * N at the scratch limit (131072), where the grid is clamped to the few
    CTAs whose rows fit the fixed array, each walking many tiles (the
    oracle on sampled spots);
  * D in 13..16 (4 pixels per thread, 8 warps per CTA);
  * strong tilts and defocus (large per-tile anchor phases).
The file sorts last so a run stopped at its first failure has already run
every other test.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from gpu_helpers import assert_close, oracle_forward  # noqa: E402
from oracle import zernike  # noqa: E402
from workloads import random_problem  # noqa: E402

pytestmark = pytest.mark.gpu

MAX_SPOTS = 131072


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _noalloc(p, basis, coeff=None, N=None):
    from paper_2505_08777_gb300 import _lib
    lib = _lib.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    coeff = torch.from_numpy(p.coeff).cuda() if coeff is None else coeff
    N = p.N if N is None else N
    amp = torch.from_numpy(p.amp).cuda()
    phase = torch.from_numpy(p.phase0).cuda()
    E = torch.full((N,), float("nan"), dtype=torch.complex64, device="cuda")
    st = lib.ash_forward_noalloc(p.nx, p.ny, _p(amp), _p(phase), p.D, _p(basis), N, _p(coeff), _p(E), stream)
    _lib.check(st, "ash_forward_noalloc")
    torch.cuda.synchronize()
    return E.cpu().numpy()


def _basis(p):
    Z = zernike.basis(p.nx, p.ny, p.noll)
    return Z, torch.from_numpy(Z.astype(np.float32).reshape(p.D, p.ny, p.nx)).cuda()


def _handle_forward(p, basis):
    from paper_2505_08777_gb300 import Hologram
    h = Hologram(torch.from_numpy(p.amp).cuda(), torch.from_numpy(p.coeff).cuda(), basis=basis)
    E = h.forward(torch.from_numpy(p.phase0).cuda()).cpu().numpy()
    h.close()
    return E


def test_noalloc_forward_matches_oracle_and_handle_on_two_calls():
    cases = [(21, 150, 97, 300, list(range(2, 12)), 10.0), (22, 70, 64, 37, list(range(2, 13)), 20.0)]
    for seed, nx, ny, N, noll, dmax in cases:
        p = random_problem(seed, nx, ny, N, noll, defocus_max=dmax)
        Z, basis = _basis(p)
        E = _noalloc(p, basis)
        assert_close(E, oracle_forward(p, p.phase0, Z), what=f"noalloc vs oracle ({nx}x{ny}, N={N})")
        assert_close(E, _handle_forward(p, basis), what=f"noalloc vs ash_forward ({nx}x{ny}, N={N})")


def test_noalloc_more_tiles_than_resident_ctas():
    # 2048 x 2048 = 4096 tiles: every CTA sums several tiles into its rows
    p = random_problem(23, 2048, 2048, 16, list(range(2, 12)), defocus_max=5.0)
    Z, basis = _basis(p)
    E = _noalloc(p, basis)
    assert_close(E, oracle_forward(p, p.phase0, Z, workers=8), what="noalloc 2048^2 vs oracle")
    assert_close(E, _handle_forward(p, basis), what="noalloc 2048^2 vs ash_forward")


@pytest.mark.parametrize("N", [20000, MAX_SPOTS])
def test_noalloc_at_the_scratch_bound(N):
    # 256 x 256 = 64 tiles; at N = 131072 only 8 scratch rows fit (two CTAs
    # of four warps), at N = 20000 thirteen CTAs: each walks many tiles
    p = random_problem(24 + N, 256, 256, N, list(range(2, 12)), defocus_max=5.0)
    Z, basis = _basis(p)
    E = _noalloc(p, basis)
    assert np.all(np.isfinite(E))
    idx = np.random.default_rng(N).choice(N, 64, replace=False)
    assert_close(E[idx], oracle_forward(p, p.phase0, Z, idx=idx), what=f"noalloc N={N} vs oracle (64 spots)")
    assert_close(E, _handle_forward(p, basis), what=f"noalloc N={N} vs ash_forward")


@pytest.mark.parametrize("D", [13, 16])
def test_noalloc_many_modes(D):
    p = random_problem(25 + D, 150, 97, 300, list(range(2, 2 + D)), defocus_max=5.0, aberr_sigma=0.3)
    Z, basis = _basis(p)
    E = _noalloc(p, basis)
    assert_close(E, oracle_forward(p, p.phase0, Z), what=f"noalloc D={D} vs oracle")
    assert_close(E, _handle_forward(p, basis), what=f"noalloc D={D} vs ash_forward")


def test_noalloc_strong_tilt_and_defocus():
    # tilts up to 0.45 Nyquist on 1024^2 (|C Z| ~ 720 rad at the edge) and
    # defocus up to 20 rad: large anchor phases, split into turns in fp32
    p = random_problem(26, 1024, 1024, 64, list(range(2, 12)), tilt_span=0.45, defocus_max=20.0)
    Z, basis = _basis(p)
    E = _noalloc(p, basis)
    assert_close(E, oracle_forward(p, p.phase0, Z, workers=8), what="noalloc strong phases vs oracle")
    assert_close(E, _handle_forward(p, basis), what="noalloc strong phases vs ash_forward")


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_2505_08777_gb300 import _lib
    lib = _lib.load()
    one = torch.zeros(8, device="cuda")
    st = lib.ash_forward_noalloc(2, 2, _p(one), _p(one), 1, _p(one), MAX_SPOTS + 1, _p(one), _p(one), None)
    assert st == 1
    assert b"131072" in lib.ash_last_error()
