"""GB300-native aberration-space holography (arXiv 2505.08777).

The compute path is the CUDA library libash.so (C ABI in include/ash.h);
this package holds its sources (csrc/), the build script and a thin torch
binding. Importing the package does not load the library; constructing a
Hologram does, and fails loudly if it is missing.
"""
from __future__ import annotations

__all__ = ["Hologram", "Batch", "principal_modes", "zsub_estimate", "zernike_subtraction", "build", "load_library"]


def load_library():
    from . import _lib
    return _lib.load()


def build(**kw):
    from .build import build as _build
    return _build(**kw)


def __getattr__(name):
    if name == "Hologram":
        from .hologram import Hologram
        return Hologram
    if name == "Batch":
        from .hologram import Batch
        return Batch
    if name in ("principal_modes", "zsub_estimate", "zernike_subtraction"):
        from . import hologram
        return getattr(hologram, name)
    if name == "autograd":
        from . import autograd
        return autograd
    raise AttributeError(name)
