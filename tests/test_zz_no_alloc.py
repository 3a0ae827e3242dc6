"""The allocation-free forward entry point, called through the C ABI.

ash_forward_noalloc serves callers that cannot allocate device memory (a
host framework that owns all device memory, a real-time control loop that
must not allocate, a plugin handed only pre-allocated buffers). It keeps its
scratch in a fixed array inside the library, shared by every call. This
test checks two calls in a row -- a larger problem, then a smaller one, so
stale scratch from the first call would show up in the second -- against the
handle-based ash_forward on the same inputs and basis, at the tolerance of
the other parity tests. The file sorts last so a run stopped at its first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from gpu_helpers import assert_close  # noqa: E402
from oracle import zernike  # noqa: E402
from workloads import random_problem  # noqa: E402

pytestmark = pytest.mark.gpu


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_forward_matches_handle_forward_on_two_calls():
    from paper_2505_08777_gb300 import Hologram, _lib
    lib = _lib.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    cases = [(21, 150, 97, 300, list(range(2, 12)), 10.0), (22, 70, 64, 37, list(range(2, 13)), 20.0)]
    for seed, nx, ny, N, noll, dmax in cases:
        p = random_problem(seed, nx, ny, N, noll, defocus_max=dmax)
        basis = torch.from_numpy(zernike.basis(nx, ny, noll).astype(np.float32).reshape(len(noll), ny, nx)).cuda()
        amp = torch.from_numpy(p.amp).cuda()
        coeff = torch.from_numpy(p.coeff).cuda()
        phase = torch.from_numpy(p.phase0).cuda()
        ref = Hologram(amp, coeff, basis=basis).forward(phase)
        E = torch.full((N,), float("nan"), dtype=torch.complex64, device="cuda")
        st = lib.ash_forward_noalloc(nx, ny, _p(amp), _p(phase), len(noll), _p(basis), N, _p(coeff), _p(E), stream)
        _lib.check(st, "ash_forward_noalloc")
        torch.cuda.synchronize()
        assert_close(E.cpu().numpy(), ref.cpu().numpy(), what=f"noalloc vs ash_forward ({nx}x{ny}, N={N})")


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_2505_08777_gb300 import _lib
    lib = _lib.load()
    one = torch.zeros(8, device="cuda")
    st = lib.ash_forward_noalloc(2, 2, _p(one), _p(one), 1, _p(one), 131073, _p(one), _p(one), None)
    assert st == 1
    assert b"131072" in lib.ash_last_error()
