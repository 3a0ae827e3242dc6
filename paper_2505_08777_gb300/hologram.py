"""Thin torch-facing binding over the C ABI (include/ash.h).

Argument marshalling only: tensors are checked for device, dtype and
contiguity, then their device pointers and torch's current CUDA stream are
handed to libash. Every step of the computation runs in the library's CUDA
kernels; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes

import numpy as np

import torch

from . import _lib

__all__ = ["Hologram", "Batch", "spot_loss", "zsub_estimate", "zernike_subtraction"]


def _stream_ptr(stream=None) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t: torch.Tensor | None) -> ctypes.c_void_p:
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _need(t: torch.Tensor, dtype, shape, name: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def spot_loss(E: torch.Tensor, t: torch.Tensor, want_grad: bool = True, stream=None):
    """Spot-intensity loss L = sum_n (|E_n|^2 / mean |E|^2 - t_n)^2 (0-dim float32
    tensor) and, if asked, dL/dRe E + i dL/dIm E (complex64 (N,)), in one
    library kernel."""
    lib = _lib.load()
    N = int(E.shape[0]) if E.dim() == 1 else -1
    _need(E, torch.complex64, (N,), "E")
    _need(t, torch.float32, (N,), "t")
    loss = torch.empty((), dtype=torch.float32, device=E.device)
    g = torch.empty_like(E) if want_grad else None
    _lib.check(lib.ash_spot_loss(_ptr(E), _ptr(t), N, _ptr(loss), _ptr(g), _stream_ptr(stream)), "ash_spot_loss")
    return loss, g


class Hologram:
    """One hologram: SLM grid (ny, nx), illumination amplitude, basis and the
    N x D coefficient matrix (paper Sec. II / Methods). Owns a libash handle."""

    def __init__(self, amp: torch.Tensor, coeff: torch.Tensor, noll=None, basis: torch.Tensor | None = None,
                 mix=None, stream=None, row0: int | None = None, ny_full: int | None = None):
        """`noll`: Noll indices of the modes (one per column of coeff), or of
        the input Zernikes when `mix` is given; `mix` (D x len(noll), float64):
        output mode k = sum_d mix[k, d] Z_noll[d] (e.g. from principal_modes);
        `basis`: a caller basis (D, ny, nx) instead of Noll modes.
        `row0`, `ny_full`: a band of a larger grid -- this hologram holds rows
        [row0, row0 + ny) of an nx x ny_full grid (amp, basis and every phase
        or field are the band's rows), in the full grid's coordinates."""
        self._lib = _lib.load()
        self._h = ctypes.c_void_p(0)
        self.coeff_epoch = 0   # counts set_coefficients calls
        if amp.dim() != 2:
            raise ValueError("amp must be (ny, nx)")
        self.ny, self.nx = int(amp.shape[0]), int(amp.shape[1])
        if coeff.dim() != 2:
            raise ValueError("coeff must be (N, D)")
        self.N, self.D = int(coeff.shape[0]), int(coeff.shape[1])
        _need(amp, torch.float32, (self.ny, self.nx), "amp")
        _need(coeff, torch.float32, (self.N, self.D), "coeff")
        noll_arr = None
        if noll is not None:
            noll = [int(v) for v in noll]
            if mix is None and len(noll) != self.D:
                raise ValueError("noll must list one index per column of coeff")
            noll_arr = (ctypes.c_int * len(noll))(*noll)
        if basis is not None:
            _need(basis, torch.float32, (self.D, self.ny, self.nx), "basis")
        self.noll = noll
        self.device = amp.device
        self.row0, self.ny_full = 0, self.ny
        if mix is not None:
            if noll is None or basis is not None:
                raise ValueError("mix needs noll (and no basis)")
            mix = np.ascontiguousarray(np.asarray(mix, dtype=np.float64))
            if mix.shape != (self.D, len(noll)):
                raise ValueError("mix must be (D, len(noll))")
            self.mix = mix
            st = self._lib.ash_hologram_create_mixed(
                ctypes.byref(self._h), self.nx, self.ny, _ptr(amp), len(noll), noll_arr, self.D,
                mix.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), self.N, _ptr(coeff), _stream_ptr(stream))
            _lib.check(st, "ash_hologram_create_mixed")
            return
        if row0 is not None or ny_full is not None:
            if row0 is None or ny_full is None:
                raise ValueError("a band needs both row0 and ny_full")
            self.row0, self.ny_full = int(row0), int(ny_full)
            st = self._lib.ash_hologram_create_band(ctypes.byref(self._h), self.nx, self.ny_full, self.row0,
                                                    self.row0 + self.ny, _ptr(amp), self.D, noll_arr, _ptr(basis),
                                                    self.N, _ptr(coeff), _stream_ptr(stream))
            _lib.check(st, "ash_hologram_create_band")
            return
        st = self._lib.ash_hologram_create(ctypes.byref(self._h), self.nx, self.ny, _ptr(amp), self.D,
                                           noll_arr, _ptr(basis), self.N, _ptr(coeff), _stream_ptr(stream))
        _lib.check(st, "ash_hologram_create")

    # -- lifetime ---------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            torch.cuda.current_stream().synchronize()
            self._lib.ash_hologram_destroy(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self) -> ctypes.c_void_p:
        return self._h

    @property
    def M(self) -> int:
        return self.nx * self.ny

    def workspace_bytes(self) -> int:
        b = ctypes.c_size_t(0)
        _lib.check(self._lib.ash_hologram_info(self._h, None, None, None, None, ctypes.byref(b)), "ash_hologram_info")
        return int(b.value)

    # -- state ------------------------------------------------------------
    def set_coefficients(self, coeff: torch.Tensor, stream=None):
        """Replace C; `coeff_epoch` counts these calls (made through this
        object), so a caller can tell whether C changed since it set it."""
        _need(coeff, torch.float32, (self.N, self.D), "coeff")
        _lib.check(self._lib.ash_set_coefficients(self._h, _ptr(coeff), _stream_ptr(stream)), "ash_set_coefficients")
        self.coeff_epoch += 1

    def coefficients(self, stream=None) -> torch.Tensor:
        """A copy of the coefficient matrix the handle currently holds (N, D)."""
        out = torch.empty((self.N, self.D), dtype=torch.float32, device=self.device)
        _lib.check(self._lib.ash_get_coefficients(self._h, _ptr(out), _stream_ptr(stream)), "ash_get_coefficients")
        return out

    def set_amplitude(self, amp: torch.Tensor, stream=None):
        _need(amp, torch.float32, (self.ny, self.nx), "amp")
        _lib.check(self._lib.ash_set_amplitude(self._h, _ptr(amp), _stream_ptr(stream)), "ash_set_amplitude")

    # -- transforms -------------------------------------------------------
    def forward(self, phase: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """E_n = sum_m A_m exp(i phase_m) exp(-i C_n . Z_m) -> complex64 (N,)."""
        _need(phase, torch.float32, (self.ny, self.nx), "phase")
        E = out if out is not None else torch.empty(self.N, dtype=torch.complex64, device=phase.device)
        _need(E, torch.complex64, (self.N,), "out")
        _lib.check(self._lib.ash_forward(self._h, _ptr(phase), _ptr(E), _stream_ptr(stream)), "ash_forward")
        return E

    def forward_coeff(self, coeff: torch.Tensor, phase: torch.Tensor, out: torch.Tensor | None = None,
                      stream=None) -> torch.Tensor:
        """Set the coefficients to `coeff` and run the forward, in one library
        call (counts as a set_coefficients call for coeff_epoch)."""
        _need(coeff, torch.float32, (self.N, self.D), "coeff")
        _need(phase, torch.float32, (self.ny, self.nx), "phase")
        E = out if out is not None else torch.empty(self.N, dtype=torch.complex64, device=phase.device)
        _need(E, torch.complex64, (self.N,), "out")
        _lib.check(self._lib.ash_forward_coeff(self._h, _ptr(coeff), _ptr(phase), _ptr(E), _stream_ptr(stream)),
                   "ash_forward_coeff")
        self.coeff_epoch += 1
        return E

    def forward_field(self, field: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """E_n = sum_m field_m exp(-i C_n . Z_m) for a complex64 (ny, nx) field."""
        _need(field, torch.complex64, (self.ny, self.nx), "field")
        E = out if out is not None else torch.empty(self.N, dtype=torch.complex64, device=field.device)
        _need(E, torch.complex64, (self.N,), "out")
        _lib.check(self._lib.ash_forward_field(self._h, _ptr(field), _ptr(E), _stream_ptr(stream)), "ash_forward_field")
        return E

    def adjoint(self, y: torch.Tensor, want_field: bool = True, want_phase: bool = False, stream=None,
                phase_out: torch.Tensor | None = None):
        """g_m = sum_n y_n exp(+i C_n . Z_m); returns (g complex64 (ny, nx) or None,
        phase float32 (ny, nx) or None); `phase_out`: write arg g there."""
        _need(y, torch.complex64, (self.N,), "y")
        g = torch.empty((self.ny, self.nx), dtype=torch.complex64, device=y.device) if want_field else None
        if phase_out is not None:
            ph = _need(phase_out, torch.float32, (self.ny, self.nx), "phase_out")
        else:
            ph = torch.empty((self.ny, self.nx), dtype=torch.float32, device=y.device) if want_phase else None
        _lib.check(self._lib.ash_adjoint(self._h, _ptr(y), _ptr(g), _ptr(ph), _stream_ptr(stream)), "ash_adjoint")
        return g, ph

    def wgs(self, phase: torch.Tensor, weights: torch.Tensor, target: torch.Tensor, iters: int,
            E_out: torch.Tensor | None = None, metrics_out: torch.Tensor | None = None, stream=None):
        """Weighted GS, in place on (phase, weights). Returns (E, metrics) where
        metrics = [uniformity, efficiency, sum |E|^2, min |E|^2/T^2]."""
        _need(phase, torch.float32, (self.ny, self.nx), "phase")
        _need(weights, torch.float32, (self.N,), "weights")
        _need(target, torch.float32, (self.N,), "target")
        E = E_out if E_out is not None else torch.empty(self.N, dtype=torch.complex64, device=phase.device)
        met = metrics_out if metrics_out is not None else torch.empty(4, dtype=torch.float32, device=phase.device)
        _lib.check(self._lib.ash_wgs_iterate(self._h, _ptr(phase), _ptr(weights), _ptr(target), int(iters), _ptr(E),
                                             _ptr(met), _stream_ptr(stream)), "ash_wgs_iterate")
        return E, met

    def spot_update(self, E: torch.Tensor, weights: torch.Tensor, target: torch.Tensor,
                    out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """The weighted-GS spot update alone: weights updated in place from E,
        returns y = w exp(i arg E) (complex64 (N,)), the adjoint's input."""
        _need(E, torch.complex64, (self.N,), "E")
        _need(weights, torch.float32, (self.N,), "weights")
        _need(target, torch.float32, (self.N,), "target")
        y = out if out is not None else torch.empty(self.N, dtype=torch.complex64, device=E.device)
        _need(y, torch.complex64, (self.N,), "out")
        _lib.check(self._lib.ash_spot_update(self._h, _ptr(E), _ptr(weights), _ptr(target), _ptr(y),
                                             _stream_ptr(stream)), "ash_spot_update")
        return y

    def spot_metrics(self, E: torch.Tensor, target: torch.Tensor, sum_a2: float = 0.0,
                     out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """[uniformity, efficiency, sum |E|^2, min |E|^2/T^2] of E; `sum_a2`:
        the whole grid's sum of A^2 (0: this handle's own)."""
        _need(E, torch.complex64, (self.N,), "E")
        _need(target, torch.float32, (self.N,), "target")
        met = out if out is not None else torch.empty(4, dtype=torch.float32, device=E.device)
        _need(met, torch.float32, (4,), "out")
        _lib.check(self._lib.ash_spot_metrics(self._h, _ptr(E), _ptr(target), float(sum_a2), _ptr(met),
                                              _stream_ptr(stream)), "ash_spot_metrics")
        return met

    def band_info(self) -> tuple[int, int, float]:
        """(first row, rows of the full grid, sum of A^2 over this handle's pixels)."""
        r0, nyf, sa = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_double(0.0)
        _lib.check(self._lib.ash_hologram_band(self._h, ctypes.byref(r0), ctypes.byref(nyf), ctypes.byref(sa)),
                   "ash_hologram_band")
        return int(r0.value), int(nyf.value), float(sa.value)

    def grad(self, phase: torch.Tensor, grad_E: torch.Tensor, want_phase: bool = True, want_coeff: bool = True,
             stream=None):
        """(dL/dphase (ny, nx) or None, dL/dC (N, D) or None) from grad_E = dL/dRe E + i dL/dIm E."""
        _need(phase, torch.float32, (self.ny, self.nx), "phase")
        _need(grad_E, torch.complex64, (self.N,), "grad_E")
        dph = torch.empty((self.ny, self.nx), dtype=torch.float32, device=phase.device) if want_phase else None
        dC = torch.empty((self.N, self.D), dtype=torch.float32, device=phase.device) if want_coeff else None
        _lib.check(self._lib.ash_grad(self._h, _ptr(phase), _ptr(grad_E), _ptr(dph), _ptr(dC), _stream_ptr(stream)),
                   "ash_grad")
        return dph, dC

    def cg_refine(self, phase: torch.Tensor, t: torch.Tensor, iters: int, theta: float = 0.05,
                  loss_out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """Conjugate-gradient refinement of `phase` (in place) on the spot-intensity
        loss with targets t; returns the losses (iters + 1,)."""
        _need(phase, torch.float32, (self.ny, self.nx), "phase")
        _need(t, torch.float32, (self.N,), "t")
        L = loss_out if loss_out is not None else torch.empty(iters + 1, dtype=torch.float32, device=phase.device)
        _need(L, torch.float32, (iters + 1,), "loss_out")
        _lib.check(self._lib.ash_cg_refine(self._h, _ptr(phase), _ptr(t), int(iters), float(theta), _ptr(L),
                                           _stream_ptr(stream)), "ash_cg_refine")
        return L

    def zsub_sweep(self, phase: torch.Tensor, mode: int, deltas, out: torch.Tensor | None = None,
                   stream=None) -> torch.Tensor:
        """Calibration sweep with this hologram as the optical system:
        I[k, n] = |E_n|^2 for the SLM phase phase + deltas[k] Z_mode (K, N)."""
        _need(phase, torch.float32, (self.ny, self.nx), "phase")
        d = [float(v) for v in deltas]
        I = out if out is not None else torch.empty((len(d), self.N), dtype=torch.float32, device=phase.device)
        _need(I, torch.float32, (len(d), self.N), "out")
        dk = (ctypes.c_float * len(d))(*d)
        _lib.check(self._lib.ash_zsub_sweep(self._h, _ptr(phase), int(mode), dk, len(d), _ptr(I),
                                            _stream_ptr(stream)), "ash_zsub_sweep")
        return I

    def set_wgs_options(self, feedback: float = 1.0, fix_phase: bool = False):
        """WGS variants for later wgs() calls: weight-update exponent p
        (w <- w (T^/E^)^p) and phase fixing (hold each spot's phase at its value
        from the last update made without fixing)."""
        _lib.check(self._lib.ash_wgs_set_options(self._h, float(feedback), int(bool(fix_phase))), "ash_wgs_set_options")

    def launch_info(self) -> dict:
        out = (ctypes.c_int * 8)()
        _lib.check(self._lib.ash_hologram_launch_info(self._h, out), "ash_hologram_launch_info")
        keys = ["grid", "fwd_ctas_per_sm", "adj_ctas_per_sm", "tc_adj_grid", "tc_fwd_grid", "split_flags",
                "kernels", "pixels_per_thread"]
        return dict(zip(keys, list(out)))

    def wgs_launches(self, iters: int) -> int:
        """Kernel launches of one wgs() call with `iters` iterations."""
        return int(self._lib.ash_wgs_launches(self._h, int(iters)))

    def graph_kernels(self, key: int) -> int:
        """Kernel nodes of the cached loop graph: key = iters of a wgs() call
        (iters >= 2), -iters of a cg_refine() call; -1 if none is cached."""
        return int(self._lib.ash_graph_kernels(self._h, int(key)))

    def set_variant(self, variant: int):
        """0 = automatic, 1 = FMA-pipe kernels, 2 = tensor-core phase contraction (any D)."""
        _lib.check(self._lib.ash_set_kernel_variant(self._h, int(variant)), "ash_set_kernel_variant")

    def check(self, stream=None):
        _lib.check(self._lib.ash_hologram_check(self._h, _stream_ptr(stream)), "ash_hologram_check")


class Batch:
    """Many holograms solved together (ash_batch_*): the loop as one CUDA
    graph; members with N*M below `solo_terms` share one launch per WGS phase
    over their (tile, spot) work units, larger ones run their own
    single-hologram kernels inside the graph."""

    def __init__(self, problems, stream=None, solo_terms: int | None = None):
        """problems: list of (amp (ny, nx), coeff (N, D), noll list) CUDA tensors / lists;
        solo_terms: the standalone threshold (None: the library default)."""
        self._lib = _lib.load()
        self._b = ctypes.c_void_p(0)
        self.shapes = []
        self._keep = []
        descs = (_lib.HologramDesc * len(problems))()
        for i, (amp, coeff, noll) in enumerate(problems):
            ny, nx = int(amp.shape[0]), int(amp.shape[1])
            N, D = int(coeff.shape[0]), int(coeff.shape[1])
            _need(amp, torch.float32, (ny, nx), "amp")
            _need(coeff, torch.float32, (N, D), "coeff")
            arr = (ctypes.c_int * D)(*[int(v) for v in noll])
            self._keep.append(arr)
            descs[i] = _lib.HologramDesc(nx, ny, amp.data_ptr(), D, ctypes.cast(arr, _lib.c_int_p), None, N,
                                         coeff.data_ptr())
            self.shapes.append((ny, nx, N, D))
        if solo_terms is None:
            _lib.check(self._lib.ash_batch_create(ctypes.byref(self._b), len(problems), descs, _stream_ptr(stream)),
                       "ash_batch_create")
        else:
            _lib.check(self._lib.ash_batch_create_ex(ctypes.byref(self._b), len(problems), descs, int(solo_terms),
                                                     _stream_ptr(stream)), "ash_batch_create_ex")

    def close(self):
        if getattr(self, "_b", None) is not None and self._b.value:
            torch.cuda.current_stream().synchronize()
            self._lib.ash_batch_destroy(self._b)
            self._b = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def count(self) -> int:
        return len(self.shapes)

    def info(self) -> dict:
        c, g, r = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        u = ctypes.c_longlong()
        _lib.check(self._lib.ash_batch_info(self._b, ctypes.byref(c), ctypes.byref(g), ctypes.byref(r),
                                            ctypes.byref(u)), "ash_batch_info")
        return {"count": c.value, "grid": g.value, "resident_ctas": r.value, "units": u.value,
                "standalone": int(self._lib.ash_batch_standalone(self._b))}

    def set_grid(self, grid: int):
        _lib.check(self._lib.ash_batch_set_grid(self._b, int(grid)), "ash_batch_set_grid")

    def set_variant(self, variant: int):
        """0 automatic, 1 FMA-pipe kernels, 2 tensor-core kernels."""
        _lib.check(self._lib.ash_batch_set_variant(self._b, int(variant)), "ash_batch_set_variant")

    def launches(self, iters: int) -> int:
        return int(self._lib.ash_batch_wgs_launches(self._b, int(iters)))

    def graph_kernels(self, iters: int) -> int:
        """Kernel nodes of the graph captured for `iters` (-1 if none is cached)."""
        return int(self._lib.ash_batch_graph_kernels(self._b, int(iters)))

    def _ptrs(self, tensors, dtype, shapes, name):
        if len(tensors) != self.count:
            raise ValueError(f"{name}: need {self.count} tensors")
        for t, shp in zip(tensors, shapes):
            _need(t, dtype, shp, name)
        return (ctypes.c_void_p * self.count)(*[t.data_ptr() for t in tensors])

    def wgs(self, phases, weights, targets, iters: int, metrics_out: torch.Tensor | None = None, stream=None):
        """In place on phases / weights; returns metrics (count, 4)."""
        ph = self._ptrs(phases, torch.float32, [(s[0], s[1]) for s in self.shapes], "phases")
        w = self._ptrs(weights, torch.float32, [(s[2],) for s in self.shapes], "weights")
        T = self._ptrs(targets, torch.float32, [(s[2],) for s in self.shapes], "targets")
        met = metrics_out if metrics_out is not None else torch.empty((self.count, 4), dtype=torch.float32,
                                                                       device=phases[0].device)
        _need(met, torch.float32, (self.count, 4), "metrics_out")
        _lib.check(self._lib.ash_batch_wgs(self._b, ph, w, T, int(iters), _ptr(met), _stream_ptr(stream)),
                   "ash_batch_wgs")
        return met

    def tune(self, phases, cache_path: str | None = None, stream=None) -> int:
        ph = self._ptrs(phases, torch.float32, [(s[0], s[1]) for s in self.shapes], "phases")
        g = ctypes.c_int()
        path = cache_path.encode() if cache_path else None
        _lib.check(self._lib.ash_batch_tune(self._b, ph, path, ctypes.byref(g), _stream_ptr(stream)), "ash_batch_tune")
        return g.value


def principal_modes(coeff, cols, K: int):
    """Principal isoplanatic modes (paper, Methods "Anisoplanatic Singular
    Value Decomposition"): rotate the modes at positions `cols` of the N x D
    coefficient matrix to their K leading principal modes (host FP64 SVD in
    the library). Returns (mix, coeff_out, sigma): mix (D', D) float64 for
    Hologram(..., noll=noll, mix=mix), coeff_out (N, D') float32 with
    D' = D - len(cols) + K, and all len(cols) singular values."""
    c = np.ascontiguousarray(np.asarray(coeff.detach().cpu() if isinstance(coeff, torch.Tensor) else coeff,
                                        dtype=np.float32))
    if c.ndim != 2:
        raise ValueError("coeff must be (N, D)")
    N, D = c.shape
    cols = [int(v) for v in cols]
    Dout = D - len(cols) + int(K)
    mix = np.zeros((max(Dout, 0), D), np.float64)
    out = np.zeros((N, max(Dout, 0)), np.float32)
    sigma = np.zeros(len(cols), np.float64)
    lib = _lib.load()
    cols_arr = (ctypes.c_int * max(len(cols), 1))(*cols)
    st = lib.ash_principal_modes(N, D, c.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), len(cols), cols_arr, int(K),
                                 mix.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                 out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                 sigma.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    _lib.check(st, "ash_principal_modes")
    return mix, out, sigma


def zsub_estimate(intensity: torch.Tensor, deltas, coeff: torch.Tensor | None = None, mode: int = 0,
                  stream=None) -> torch.Tensor:
    """Per-spot vertex of the log-parabola through a sweep (K, N); with
    `coeff` (N, D) the estimates are also added to its column `mode`."""
    d = [float(v) for v in deltas]
    K = len(d)
    if intensity.dim() != 2 or intensity.shape[0] != K:
        raise ValueError("intensity must have shape (K, N)")
    N = int(intensity.shape[1])
    _need(intensity, torch.float32, (K, N), "intensity")
    D = 0
    if coeff is not None:
        D = int(coeff.shape[1]) if coeff.dim() == 2 else 0
        _need(coeff, torch.float32, (N, D), "coeff")
    out = torch.empty(N, dtype=torch.float32, device=intensity.device)
    dk = (ctypes.c_float * K)(*d)
    lib = _lib.load()
    _lib.check(lib.ash_zsub_estimate(_ptr(intensity), dk, K, N, _ptr(out), _ptr(coeff), D, int(mode),
                                     _stream_ptr(stream)), "ash_zsub_estimate")
    return out


def zernike_subtraction(model: Hologram, system: Hologram, target: torch.Tensor, modes, deltas, rounds: int = 1,
                        wgs_iters: int = 0, shrink: float = 1.0, stream=None):
    """Simulated Zernike-subtraction calibration (paper Sec. III): for each
    round and each column d in `modes`, a baseline hologram from the model
    (superposition arg K^H T, or `wgs_iters` weighted-GS iterations from a
    zero phase), a sweep of deltas * shrink^round through the system, the
    per-spot estimates, and their subtraction into the model's column d.
    Returns the model's final coefficients (N, D) and the estimates of every
    step [(d, delta_star)]."""
    _need(target, torch.float32, (model.N,), "target")
    if (system.nx, system.ny, system.N, system.D) != (model.nx, model.ny, model.N, model.D):
        raise ValueError("model and system must have the same grid, spots and modes")
    C = model.coefficients().clone()
    y = target.to(torch.complex64)
    steps = []
    for r in range(rounds):
        dr = [float(v) * shrink ** r for v in deltas]
        for d in modes:
            if wgs_iters > 0:
                phi = torch.zeros((model.ny, model.nx), dtype=torch.float32, device=target.device)
                model.wgs(phi, target.clone(), target, wgs_iters, stream=stream)
            else:
                _, phi = model.adjoint(y, want_field=False, want_phase=True, stream=stream)
            I = system.zsub_sweep(phi, d, dr, stream=stream)
            ds = zsub_estimate(I, dr, C, d, stream=stream)
            model.set_coefficients(C, stream=stream)
            steps.append((d, ds))
    return C, steps
