"""The C ABI library: loads, exports every symbol include/ash.h declares, and
rejects bad arguments on the host before touching the GPU (CPU only)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ash.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(ash_[a-z_0-9]+)\s*\(", text))
    return sorted(n for n in names if not n.endswith("_fn"))


@pytest.fixture(scope="module")
def lib():
    import paper_2505_08777_gb300 as P
    lib_path = os.path.join(ROOT, "paper_2505_08777_gb300", "libash.so")
    if not os.path.exists(lib_path):
        P.build()
    return P.load_library()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    from paper_2505_08777_gb300 import _lib
    assert set(_lib.SIGNATURES) == set(names)


def test_abi_version_and_status_strings(lib):
    assert lib.ash_abi_version() == 1
    assert lib.ash_status_string(0) == b"ASH_OK"
    assert lib.ash_status_string(1) == b"ASH_ERR_INVALID_ARG"
    assert lib.ash_status_string(99) == b"ASH_ERR_UNKNOWN"


def _create(lib, nx, ny, D, N, noll=True, amp=1, coeff=1, basis=0):
    h = ctypes.c_void_p(0)
    arr = (ctypes.c_int * max(D, 1))(*([2] * max(D, 1))) if noll else None
    st = lib.ash_hologram_create(ctypes.byref(h), nx, ny, ctypes.c_void_p(amp), D, arr, ctypes.c_void_p(basis), N,
                                 ctypes.c_void_p(coeff), None)
    return st, h


def test_invalid_arguments_rejected_without_gpu(lib):
    # argument checks run before any CUDA call, so they work on a CPU-only host
    assert _create(lib, 0, 8, 2, 4)[0] == 1
    assert _create(lib, 8, 20000, 2, 4)[0] == 1
    assert _create(lib, 8, 8, 0, 4)[0] == 1
    assert _create(lib, 8, 8, 17, 4)[0] == 1
    assert _create(lib, 8, 8, 2, 0)[0] == 1
    assert _create(lib, 8, 8, 2, 4, amp=0)[0] == 1
    assert _create(lib, 8, 8, 2, 4, noll=False)[0] == 1          # neither noll nor basis
    assert _create(lib, 8, 8, 2, 4, noll=True, basis=64)[0] == 1  # both
    assert b"exactly one" in lib.ash_last_error()
    bad = (ctypes.c_int * 2)(2, 0)
    h = ctypes.c_void_p(0)
    st = lib.ash_hologram_create(ctypes.byref(h), 8, 8, ctypes.c_void_p(1), 2, bad, None, 4, ctypes.c_void_p(1), None)
    assert st == 1 and b"Noll" in lib.ash_last_error()
    for fn, args in [("ash_forward", (None, None, None, None)), ("ash_adjoint", (None, None, None, None, None)),
                     ("ash_wgs_iterate", (None, None, None, None, 1, None, None, None)),
                     ("ash_grad", (None, None, None, None, None, None)), ("ash_hologram_check", (None, None))]:
        assert getattr(lib, fn)(*args) == 1, fn
    assert lib.ash_debug_fail_after(-1) == 1


def test_later_entry_points_reject_bad_arguments_without_gpu(lib):
    # CG, calibration, batch, launch counts, no-alloc forward, mixed bases,
    # sin/cos check: each returns ASH_ERR_INVALID_ARG (or -1 for the counts)
    # from its host-side checks, before any CUDA call
    vp, INV = ctypes.c_void_p, 1
    one = vp(1)
    d3 = (ctypes.c_float * 3)(-1.0, 0.0, 1.0)
    same = (ctypes.c_float * 3)(0.5, 0.5, 0.5)
    assert lib.ash_cg_refine(None, one, one, 5, 0.05, None, None) == INV
    assert lib.ash_zsub_sweep(None, one, 0, d3, 3, one, None) == INV
    assert lib.ash_zsub_estimate(one, d3, 2, 4, one, None, 0, 0, None) == INV      # K < 3
    assert lib.ash_zsub_estimate(one, d3, 33, 4, one, None, 0, 0, None) == INV     # K > 32
    assert lib.ash_zsub_estimate(one, same, 3, 4, one, None, 0, 0, None) == INV    # one distinct offset
    assert b"distinct" in lib.ash_last_error()
    assert lib.ash_zsub_estimate(None, d3, 3, 4, one, None, 0, 0, None) == INV
    for fn in ("ash_wgs_launches", "ash_graph_kernels", "ash_batch_wgs_launches", "ash_batch_graph_kernels"):
        assert getattr(lib, fn)(None, 4) == -1, fn
    assert lib.ash_batch_standalone(None) == -1
    assert lib.ash_debug_wait_timeout(None, 16, None) == INV
    assert lib.ash_get_coefficients(None, one, None) == INV
    b = ctypes.c_void_p(0)
    assert lib.ash_batch_create(ctypes.byref(b), 0, None, None) == INV
    assert lib.ash_batch_create_ex(ctypes.byref(b), 1, one, -1, None) == INV
    assert lib.ash_set_kernel_variant(None, 1) == INV
    assert lib.ash_wgs_set_options(None, 1.0, 0) == INV
    assert lib.ash_debug_sincos(one, -1, one, one, 0, None) == INV
    assert lib.ash_debug_sincos(one, 4, one, one, 2, None) == INV
    E = one
    assert lib.ash_forward_noalloc(0, 8, one, one, 2, one, 4, one, E, None) == INV
    assert lib.ash_forward_noalloc(8, 8, one, one, 2, one, 131073, one, E, None) == INV
    assert lib.ash_forward_noalloc(8, 8, None, one, 2, one, 4, one, E, None) == INV
    noll = (ctypes.c_int * 2)(2, 3)
    mix = (ctypes.c_double * 4)(1, 0, 0, 1)
    h = ctypes.c_void_p(0)
    assert lib.ash_hologram_create_mixed(ctypes.byref(h), 8, 8, one, 0, noll, 2, mix, 4, one, None) == INV
    assert lib.ash_hologram_create_mixed(ctypes.byref(h), 8, 8, one, 65, noll, 2, mix, 4, one, None) == INV


def test_fault_injection_counts_calls(lib):
    # the n-th launching call fails with ASH_ERR_INJECTED; argument errors are not counted
    assert lib.ash_debug_fail_after(1) == 0
    st, _ = _create(lib, 8, 8, 2, 4)
    assert st == 6 and b"injected" in lib.ash_last_error()
    assert lib.ash_debug_fail_after(0) == 0


def test_allocator_hook_validation(lib):
    from paper_2505_08777_gb300 import _lib
    alloc = _lib.ALLOC_FN(lambda ctx, n, s: None)
    assert lib.ash_set_allocator(alloc, _lib.FREE_FN(0), None) == 1
    assert lib.ash_set_allocator(_lib.ALLOC_FN(0), _lib.FREE_FN(0), None) == 0


def test_python_binding_rejects_cpu_tensors():
    torch = pytest.importorskip("torch")
    from paper_2505_08777_gb300 import Hologram
    with pytest.raises(ValueError):
        Hologram(torch.ones(4, 4), torch.zeros(2, 3), noll=[2, 3, 4])


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    # no CPU fallback: without libash.so the binding raises instead of computing
    from paper_2505_08777_gb300 import _lib
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(ImportError, match="not built"):
        _lib.load(str(tmp_path / "libash.so"))


def test_probe_rejects_null_output(lib):
    assert lib.ash_probe_rates(None, None) == 1


def test_band_arguments_rejected_without_gpu(lib):
    h = ctypes.c_void_p(0)
    arr = (ctypes.c_int * 2)(2, 3)

    def band(nx, nyf, r0, r1):
        return lib.ash_hologram_create_band(ctypes.byref(h), nx, nyf, r0, r1, ctypes.c_void_p(1), 2, arr, None, 4,
                                            ctypes.c_void_p(1), None)
    assert band(64, 100, 16, 64) == 1       # not on a 32-row tile boundary
    assert band(64, 100, 0, 40) == 1        # ends inside a tile row that is not the last
    assert band(64, 100, 64, 64) == 1       # empty
    assert band(64, 100, 64, 101) == 1      # past the grid
    assert band(0, 100, 0, 32) == 1
    assert b"tile" in lib.ash_last_error() or b"grid" in lib.ash_last_error()
    assert lib.ash_spot_update(None, None, None, None, None, None) == 1
    assert lib.ash_spot_metrics(None, None, None, 0.0, None, None) == 1


def test_loss_and_fused_forward_reject_bad_arguments(lib):
    assert lib.ash_spot_loss(None, None, 4, None, None, None) == 1
    assert lib.ash_spot_loss(ctypes.c_void_p(8), ctypes.c_void_p(8), 0, ctypes.c_void_p(8), None, None) == 1
    assert lib.ash_forward_coeff(None, None, None, None, None) == 1
