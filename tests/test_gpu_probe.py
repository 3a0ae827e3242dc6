"""The pipe-rate probe behind the roofline: it runs on every SM and returns
per-clock rates inside the ranges any recent NVIDIA SM allows (MUFU 4..64
sin/cos per clock, FP32 64..512 lane results per clock), and the MUFU rate
is far below the FP32 rate (the reason a sin/cos share on the FP32 pipe
pays). Absolute values are recorded by `bench.py --config peaks`."""
import ctypes

import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def test_probe_rates_are_plausible():
    from paper_2505_08777_gb300 import _lib
    lib = _lib.load()
    out = (ctypes.c_double * 6)()
    _lib.check(lib.ash_probe_rates(out, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)), "ash_probe_rates")
    sincos, ffma, ffma2, ex2, mhz, sms = list(out)
    assert sms == torch.cuda.get_device_properties(0).multi_processor_count
    assert 4 <= sincos <= 64 and 4 <= ex2 <= 128
    assert 64 <= ffma <= 512 and 64 <= ffma2 <= 512
    assert ffma > 4 * sincos
    assert 200 <= mhz <= 4000
