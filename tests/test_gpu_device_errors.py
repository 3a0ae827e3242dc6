"""Device-side failure detection without a fault: every spin-wait of the
tensor-core kernels is bounded, and on reaching its limit a kernel records a
timeout in the handle's error word and returns. Here one such wait is made
to run out (a fresh mbarrier that nothing arrives on); the host reads the
status through ash_hologram_check, the word is cleared, and the handle keeps
computing the same results."""
import ctypes

import pytest

torch = pytest.importorskip("torch")

from workloads import random_problem  # noqa: E402

pytestmark = pytest.mark.gpu

ASH_OK, ASH_ERR_INVALID_ARG, ASH_ERR_TIMEOUT = 0, 1, 4


def test_bounded_wait_times_out_and_the_handle_stays_usable():
    from paper_2505_08777_gb300 import Hologram, _lib
    lib = _lib.load()
    p = random_problem(61, 128, 96, 200, list(range(2, 12)))
    h = Hologram(torch.from_numpy(p.amp).cuda(), torch.from_numpy(p.coeff).cuda(), noll=p.noll)
    phase = torch.from_numpy(p.phase0).cuda()
    s = torch.cuda.current_stream()
    sp = ctypes.c_void_p(s.cuda_stream)
    E0 = h.forward(phase).clone()
    assert lib.ash_hologram_check(h.handle, sp) == ASH_OK
    assert lib.ash_debug_wait_timeout(h.handle, 0, sp) == ASH_ERR_INVALID_ARG
    assert lib.ash_debug_wait_timeout(h.handle, 4096, sp) == ASH_OK
    assert lib.ash_hologram_check(h.handle, sp) == ASH_ERR_TIMEOUT
    assert b"bounded wait" in lib.ash_last_error()
    assert lib.ash_hologram_check(h.handle, sp) == ASH_OK          # the word was cleared
    E1 = h.forward(phase)
    assert torch.equal(E0, E1)
    _, met = h.wgs(phase.clone(), torch.from_numpy(p.target).cuda(), torch.from_numpy(p.target).cuda(), 3)
    assert lib.ash_hologram_check(h.handle, sp) == ASH_OK
    assert bool(torch.isfinite(met).all())


def test_python_check_raises_on_a_recorded_timeout():
    from paper_2505_08777_gb300 import Hologram, _lib
    lib = _lib.load()
    p = random_problem(62, 64, 64, 20, [2, 3, 4])
    h = Hologram(torch.from_numpy(p.amp).cuda(), torch.from_numpy(p.coeff).cuda(), noll=p.noll)
    sp = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.ash_debug_wait_timeout(h.handle, 64, sp) == ASH_OK
    with pytest.raises(_lib.AshError):
        h.check()
    h.check()                                                      # cleared: no error now
