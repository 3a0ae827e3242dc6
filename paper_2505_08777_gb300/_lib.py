"""ctypes loader for libash.so (the C ABI declared in include/ash.h).

Loading never falls back to anything: if the shared library is missing or
does not export the ABI, an error is raised.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libash.so")

c_int, c_float_p, c_void_p = ctypes.c_int, ctypes.POINTER(ctypes.c_float), ctypes.c_void_p
c_int_p = ctypes.POINTER(ctypes.c_int)
c_size_t = ctypes.c_size_t

ALLOC_FN = ctypes.CFUNCTYPE(c_void_p, c_void_p, c_size_t, c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, c_void_p, c_void_p, c_void_p)

# name -> (restype, argtypes); every name here is declared in include/ash.h
SIGNATURES = {
    "ash_abi_version": (c_int, []),
    "ash_status_string": (ctypes.c_char_p, [c_int]),
    "ash_last_error": (ctypes.c_char_p, []),
    "ash_set_allocator": (c_int, [ALLOC_FN, FREE_FN, c_void_p]),
    "ash_debug_fail_after": (c_int, [c_int]),
    "ash_debug_sincos": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_int, c_void_p]),
    "ash_probe_rates": (c_int, [ctypes.POINTER(ctypes.c_double), c_void_p]),
    "ash_zsub_sweep": (c_int, [c_void_p, c_void_p, c_int, c_float_p, c_int, c_void_p, c_void_p]),
    "ash_cg_refine": (c_int, [c_void_p, c_void_p, c_void_p, c_int, ctypes.c_float, c_void_p, c_void_p]),
    "ash_zsub_estimate": (c_int, [c_void_p, c_float_p, c_int, c_int, c_void_p, c_void_p, c_int, c_int, c_void_p]),
    "ash_hologram_create": (c_int, [ctypes.POINTER(c_void_p), c_int, c_int, c_void_p, c_int, c_int_p, c_void_p,
                                    c_int, c_void_p, c_void_p]),
    "ash_hologram_create_mixed": (c_int, [ctypes.POINTER(c_void_p), c_int, c_int, c_void_p, c_int, c_int_p, c_int,
                                          ctypes.POINTER(ctypes.c_double), c_int, c_void_p, c_void_p]),
    "ash_hologram_create_band": (c_int, [ctypes.POINTER(c_void_p), c_int, c_int, c_int, c_int, c_void_p, c_int,
                                         c_int_p, c_void_p, c_int, c_void_p, c_void_p]),
    "ash_hologram_band": (c_int, [c_void_p, c_int_p, c_int_p, ctypes.POINTER(ctypes.c_double)]),
    "ash_spot_update": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "ash_spot_metrics": (c_int, [c_void_p, c_void_p, c_void_p, ctypes.c_double, c_void_p, c_void_p]),
    "ash_principal_modes": (c_int, [c_int, c_int, ctypes.POINTER(ctypes.c_float), c_int, c_int_p, c_int,
                                    ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_float),
                                    ctypes.POINTER(ctypes.c_double)]),
    "ash_wgs_set_options": (c_int, [c_void_p, ctypes.c_float, c_int]),
    "ash_batch_set_variant": (c_int, [c_void_p, c_int]),
    "ash_hologram_destroy": (None, [c_void_p]),
    "ash_hologram_info": (c_int, [c_void_p, c_int_p, c_int_p, c_int_p, c_int_p, ctypes.POINTER(c_size_t)]),
    "ash_set_coefficients": (c_int, [c_void_p, c_void_p, c_void_p]),
    "ash_set_amplitude": (c_int, [c_void_p, c_void_p, c_void_p]),
    "ash_forward": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "ash_forward_field": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "ash_forward_coeff": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "ash_spot_loss": (c_int, [c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_void_p]),
    "ash_adjoint": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "ash_wgs_iterate": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_void_p]),
    "ash_grad": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "ash_hologram_check": (c_int, [c_void_p, c_void_p]),
    "ash_wgs_launches": (c_int, [c_void_p, c_int]),
    "ash_graph_kernels": (c_int, [c_void_p, c_int]),
    "ash_get_coefficients": (c_int, [c_void_p, c_void_p, c_void_p]),
    "ash_debug_wait_timeout": (c_int, [c_void_p, ctypes.c_uint, c_void_p]),
    "ash_set_kernel_variant": (c_int, [c_void_p, c_int]),
    "ash_hologram_launch_info": (c_int, [c_void_p, c_int_p]),
    "ash_profile": (c_int, [c_void_p, c_void_p, c_void_p, c_float_p, c_void_p]),
    "ash_batch_create": (c_int, [ctypes.POINTER(c_void_p), c_int, c_void_p, c_void_p]),
    "ash_batch_create_ex": (c_int, [ctypes.POINTER(c_void_p), c_int, c_void_p, ctypes.c_longlong, c_void_p]),
    "ash_batch_standalone": (c_int, [c_void_p]),
    "ash_batch_destroy": (None, [c_void_p]),
    "ash_batch_info": (c_int, [c_void_p, c_int_p, c_int_p, c_int_p, ctypes.POINTER(ctypes.c_longlong)]),
    "ash_batch_set_grid": (c_int, [c_void_p, c_int]),
    "ash_batch_wgs_launches": (c_int, [c_void_p, c_int]),
    "ash_batch_graph_kernels": (c_int, [c_void_p, c_int]),
    "ash_batch_wgs": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_void_p]),
    "ash_batch_tune": (c_int, [c_void_p, c_void_p, ctypes.c_char_p, c_int_p, c_void_p]),
    "ash_forward_noalloc": (c_int, [c_int, c_int, c_void_p, c_void_p, c_int, c_void_p, c_int, c_void_p, c_void_p,
                                    c_void_p]),
}



class HologramDesc(ctypes.Structure):
    """ash_hologram_desc (include/ash.h)."""
    _fields_ = [("nx", c_int), ("ny", c_int), ("amp", c_void_p), ("D", c_int), ("noll", c_int_p),
                ("basis", c_void_p), ("N", c_int), ("coeff", c_void_p)]


_lib = None


class AshError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: {status_name(status)}: {message}")
        self.status = status


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libash.so not built at {path}; run __graft_entry__.build() "
                          "(python -m paper_2505_08777_gb300.build)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)   # AttributeError if the ABI is incomplete
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def status_name(status: int) -> str:
    lib = load()
    return lib.ash_status_string(status).decode()


def check(status: int, where: str) -> None:
    if status != 0:
        lib = load()
        raise AshError(status, where, lib.ash_last_error().decode())
