"""Accuracy of the transforms' two sin / cos evaluations on the GPU against
float64: the MUFU approximations and the FP32-pipe polynomial that takes a
share of the pixel pairs (half-angle reduction, degree-4 polynomials in r^2).

The polynomial must stay within 1e-6 absolute on |x| <= pi, the range of the
anchored local phases, and within 1e-6 + 1.2e-7 |x| beyond it (the float32
product x / (2 pi) carries a relative rounding error of about 6e-8, the same
for both paths).
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _run(lib, x, path):
    xd = torch.from_numpy(x).cuda()
    s = torch.empty_like(xd)
    c = torch.empty_like(xd)
    st = lib.ash_debug_sincos(ctypes.c_void_p(xd.data_ptr()), x.size, ctypes.c_void_p(s.data_ptr()),
                              ctypes.c_void_p(c.data_ptr()), path, None)
    assert st == 0
    torch.cuda.synchronize()
    return s.cpu().numpy().astype(np.float64), c.cpu().numpy().astype(np.float64)


def test_polynomial_sincos_error_bounds():
    from paper_2505_08777_gb300 import _lib
    lib = _lib.load()
    rng = np.random.default_rng(11)
    special = np.array([0.0, np.pi / 2, -np.pi / 2, np.pi, -np.pi, np.pi / 4, 3 * np.pi / 4, 1e-30, -1e-7,
                        2 * np.pi, 100 * np.pi + 0.5])
    near = rng.uniform(-np.pi, np.pi, 400001)
    wide = rng.uniform(-300.0, 300.0, 400000)
    x = np.concatenate([special, near, wide]).astype(np.float32)
    xe = x.astype(np.float64)
    ref_s, ref_c = np.sin(xe), np.cos(xe)
    bound = np.where(np.abs(xe) <= np.pi, 1e-6, 1e-6 + 1.2e-7 * np.abs(xe))
    s1, c1 = _run(lib, x, 1)
    assert np.all(np.abs(s1 - ref_s) <= bound), float(np.max(np.abs(s1 - ref_s) - bound))
    assert np.all(np.abs(c1 - ref_c) <= bound), float(np.max(np.abs(c1 - ref_c) - bound))
    # the MUFU path on the same inputs (the transforms' other path): the two
    # agree to the sum of their errors on the anchored range
    s0, c0 = _run(lib, x, 0)
    m = np.abs(xe) <= np.pi
    assert np.max(np.abs(s0[m] - s1[m])) <= 3e-6
    assert np.max(np.abs(c0[m] - c1[m])) <= 3e-6


def test_debug_sincos_rejects_bad_arguments():
    from paper_2505_08777_gb300 import _lib
    lib = _lib.load()
    assert lib.ash_debug_sincos(None, 4, None, None, 1, None) != 0
