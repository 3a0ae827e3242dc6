"""Seeded synthetic inputs shaped like the paper's workloads.

This module produces INPUTS only (illumination amplitude, initial phase,
per-spot coefficient matrix, target amplitudes). It holds none of the
method's arithmetic: no basis evaluation, no transform, no update rule.
Both the CPU oracle tests and the GPU path draw their inputs from here.

Shapes follow the paper's experiments:
  * 2D tweezer grids with per-spot tilts (Sec. III, Fig. 3),
  * 50 isoplanatic patches x 8 aberration modes (abstract; Sec. III),
  * 3D lattices with per-spot defocus (Sec. IV, Fig. 4).
The paper's experimental data are not public (Data availability), so these
synthetic fields stand in for the measured aberration maps.

Conventions (shared with the readings documented for the oracle):
  * pixel (i, j): i = column in [0, nx), j = row in [0, ny); flat m = j*nx + i.
  * modes are Zernike polynomials in Noll order; mode list "noll" gives the
    Noll index of each column of C.
  * a spot at Nyquist fraction (u, v) has x/y tilt coefficients
    (u*pi*R, v*pi*R) radians of edge phase, R = min(nx, ny)/2.
All arrays are float32 (the GPU path's input precision); the oracle promotes
them exactly to float64.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Problem", "gaussian_amplitude", "flat_amplitude", "random_phase",
    "config_c1", "config_c2", "config_c3", "config_c4", "config_c5", "config_c5_small",
    "make_config", "random_problem", "CONFIG_NAMES", "pixel_sample", "masked_amplitude",
]


@dataclasses.dataclass
class Problem:
    """One hologram: grid, amplitude, initial phase, coefficients, target."""
    name: str
    nx: int
    ny: int
    amp: np.ndarray      # float32 (ny, nx)
    phase0: np.ndarray   # float32 (ny, nx)
    noll: list           # Noll index per column of C
    coeff: np.ndarray    # float32 (N, D), radians of edge phase per mode
    target: np.ndarray   # float32 (N,) target amplitudes
    iters: int

    @property
    def N(self) -> int:
        return int(self.coeff.shape[0])

    @property
    def D(self) -> int:
        return int(self.coeff.shape[1])

    @property
    def M(self) -> int:
        return self.nx * self.ny


def _radius(nx: int, ny: int) -> float:
    return min(nx, ny) / 2.0


def gaussian_amplitude(nx: int, ny: int, waist_frac: float = 0.4) -> np.ndarray:
    """Gaussian illumination A ~ exp(-r^2/w^2), w = waist_frac*min(nx, ny)
    pixels (1/e^2 intensity radius), normalised to unit power sum(A^2) = 1."""
    w = waist_frac * min(nx, ny)
    ii = np.arange(nx, dtype=np.float64) - (nx - 1) / 2.0
    jj = np.arange(ny, dtype=np.float64) - (ny - 1) / 2.0
    r2 = jj[:, None] ** 2 + ii[None, :] ** 2
    a = np.exp(-r2 / (w * w))
    a /= math.sqrt(float(np.sum(a * a)))
    return a.astype(np.float32)


def flat_amplitude(nx: int, ny: int) -> np.ndarray:
    """Flat-top illumination over the whole rectangle, unit power."""
    return np.full((ny, nx), 1.0 / math.sqrt(nx * ny), dtype=np.float32)


def random_phase(rng: np.random.Generator, nx: int, ny: int) -> np.ndarray:
    return rng.uniform(0.0, 2.0 * math.pi, size=(ny, nx)).astype(np.float32)


def _grid_uv(g: int, span: float) -> np.ndarray:
    """g x g lattice of Nyquist fractions in [-span, span], row-major (v outer)."""
    t = np.linspace(-span, span, g) if g > 1 else np.zeros(1)
    uu, vv = np.meshgrid(t, t)  # vv varies along rows
    return np.stack([uu.ravel(), vv.ravel()], axis=1)


def _quadratic_field(rng: np.random.Generator, n_modes: int, sigma: float, nvars: int):
    """Random smooth field a_d(p) = sum_{|k| <= 2} alpha_{d,k} p^k over nvars
    normalised coordinates; returns (exponent list, alpha matrix)."""
    exps = []
    for total in range(3):
        if nvars == 2:
            for p in range(total, -1, -1):
                exps.append((p, total - p))
        else:
            for p in range(total, -1, -1):
                for q in range(total - p, -1, -1):
                    exps.append((p, q, total - p - q))
    alpha = rng.normal(0.0, sigma, size=(n_modes, len(exps)))
    return exps, alpha


def _eval_field(exps, alpha, pts: np.ndarray) -> np.ndarray:
    """Evaluate the smooth field at points (P, nvars) -> (P, n_modes)."""
    mono = np.ones((pts.shape[0], len(exps)))
    for k, e in enumerate(exps):
        for v, power in enumerate(e):
            mono[:, k] *= pts[:, v] ** power
    return mono @ alpha.T


def _tilts(uv: np.ndarray, R: float) -> np.ndarray:
    return (uv * math.pi * R).astype(np.float64)


def config_c1(seed: int = 1) -> Problem:
    """Plain WGS: 256x256, Gaussian A, 4x4 spots within +-0.4 Nyquist, D=10
    (Noll 2-11), defocus 0, aberrations quadratic(u, v) + N(0, 0.2), T = 1."""
    rng = np.random.default_rng(seed)
    nx = ny = 256
    R = _radius(nx, ny)
    uv = _grid_uv(4, 0.4)
    N = uv.shape[0]
    noll = list(range(2, 12))
    C = np.zeros((N, len(noll)))
    C[:, 0:2] = _tilts(uv, R)
    exps, alpha = _quadratic_field(rng, 7, 0.5, 2)
    C[:, 3:10] = _eval_field(exps, alpha, uv / 0.4) + rng.normal(0.0, 0.2, size=(N, 7))
    phase0 = random_phase(rng, nx, ny)
    return Problem("c1_plain_256x256_N16_D10", nx, ny, gaussian_amplitude(nx, ny), phase0,
                   noll, C.astype(np.float32), np.ones(N, np.float32), 20)


def _patch_coeffs(rng, uv_norm: np.ndarray, n_modes: int, n_patches: int, sigma: float):
    """Piecewise-constant smooth field: 50 patch centres uniform in the field
    box, each spot takes the nearest centre's coefficients."""
    centres = rng.uniform(-1.0, 1.0, size=(n_patches, 2))
    exps, alpha = _quadratic_field(rng, n_modes, sigma, 2)
    patch_vals = _eval_field(exps, alpha, centres)
    d2 = ((uv_norm[:, None, :] - centres[None, :, :]) ** 2).sum(-1)
    nearest = np.argmin(d2, axis=1)
    return patch_vals[nearest], nearest


def config_c2(seed: int = 1, nx: int = 1024, ny: int = 1024, grid: int = 20) -> Problem:
    """Anisoplanatic 2D tweezer array: Gaussian A, grid x grid spots over
    +-0.45 Nyquist, 50 isoplanatic patches (nearest centre), Noll 4-11 from a
    smooth field with sigma 0.5 rad, per-spot tilts, D=10, T = 1, 50 iters."""
    rng = np.random.default_rng(seed)
    R = _radius(nx, ny)
    uv = _grid_uv(grid, 0.45)
    N = uv.shape[0]
    noll = list(range(2, 12))
    C = np.zeros((N, len(noll)))
    C[:, 0:2] = _tilts(uv, R)
    vals, _ = _patch_coeffs(rng, uv / 0.45, 8, 50, 0.5)
    C[:, 2:10] = vals
    phase0 = random_phase(rng, nx, ny)
    return Problem(f"c2_aniso2d_{nx}x{ny}_N{N}_D10_50patches", nx, ny, gaussian_amplitude(nx, ny),
                   phase0, noll, C.astype(np.float32), np.ones(N, np.float32), 50)


def config_c3(seed: int = 1, nx: int = 1920, ny: int = 1152, grid: int = 20, planes: int = 5) -> Problem:
    """3D volume: flat-top A, grid x grid lateral lattice over +-0.45 Nyquist
    times `planes` defocus planes evenly in [-20, 20] rad edge phase, D=11
    (Noll 2-12), aberrations (Noll 5-12) = quadratic(u, v, z) + N(0, 0.3),
    T ~ U[0.5, 1], 100 iters."""
    rng = np.random.default_rng(seed)
    R = _radius(nx, ny)
    uv = _grid_uv(grid, 0.45)
    zs = np.linspace(-20.0, 20.0, planes) if planes > 1 else np.zeros(1)
    pts = np.array([(u, v, z) for z in zs for (u, v) in uv])
    N = pts.shape[0]
    noll = list(range(2, 13))
    C = np.zeros((N, len(noll)))
    C[:, 0:2] = _tilts(pts[:, :2], R)
    C[:, 2] = pts[:, 2]
    norm = np.stack([pts[:, 0] / 0.45, pts[:, 1] / 0.45, pts[:, 2] / 20.0], axis=1)
    exps, alpha = _quadratic_field(rng, 8, 0.5, 3)
    C[:, 3:11] = _eval_field(exps, alpha, norm) + rng.normal(0.0, 0.3, size=(N, 8))
    target = rng.uniform(0.5, 1.0, size=N)
    phase0 = random_phase(rng, nx, ny)
    return Problem(f"c3_volume3d_{nx}x{ny}_N{N}_D11", nx, ny, flat_amplitude(nx, ny), phase0,
                   noll, C.astype(np.float32), target.astype(np.float32), 100)


def config_c4(seed: int = 1, nx: int = 1024, ny: int = 1024, grid: int = 32) -> Problem:
    """One hologram of the differentiable batch: c2 recipe with a grid x grid
    lattice (N = 1024 at grid 32); target t ~ U[0.5, 1.5] (spot-intensity
    loss targets)."""
    p = config_c2(seed, nx, ny, grid)
    rng = np.random.default_rng(10_000 + seed)
    p.target = rng.uniform(0.5, 1.5, size=p.N).astype(np.float32)
    p.name = f"c4_autograd_{nx}x{ny}_N{p.N}_D10"
    p.iters = 200
    return p


def config_zsub(seed: int = 1, nx: int = 1024, ny: int = 1024, grid: int = 20) -> Problem:
    """Simulated Zernike-subtraction calibration: the c2 system (its
    coefficient matrix is the synthetic optical system's, with the smooth
    anisoplanatic aberration in Noll 4-11) seen by a model that knows only
    the spot positions (zsub_model0). Sweep: 7 offsets in [-1.5, 1.5] rad
    over Noll 4-11, one round, superposition baseline."""
    p = config_c2(seed, nx, ny, grid)
    p.name = f"zsub_{nx}x{ny}_N{p.N}_D10"
    p.iters = 0
    return p


def zsub_model0(p: Problem) -> np.ndarray:
    """The model's starting coefficients: the system's tilts, no aberration."""
    C = np.zeros_like(p.coeff)
    for k, j in enumerate(p.noll):
        if j in (2, 3):
            C[:, k] = p.coeff[:, k]
    return C


ZSUB_DELTAS = np.linspace(-1.5, 1.5, 7)


C5_SIZES = [(512, 512), (1024, 1024), (1920, 1152)]


def config_c5(seed: int = 1, count: int = 64, sizes=None, max_spots: int = 5000) -> list:
    """Batched uneven form: `count` holograms; size uniform over `sizes`;
    N = round(exp U[ln 10, ln max_spots]); D uniform over {5, 10, 11}
    (Noll 2-6 / 2-11 / 2-12); coefficients as the 2D (D = 5, 10) or 3D
    (D = 11) recipes; 50 iterations each."""
    rng = np.random.default_rng(seed)
    sizes = sizes or C5_SIZES
    out = []
    for h in range(count):
        nx, ny = sizes[int(rng.integers(len(sizes)))]
        N = int(round(math.exp(rng.uniform(math.log(10.0), math.log(max_spots)))))
        D = [5, 10, 11][int(rng.integers(3))]
        R = _radius(nx, ny)
        g = int(math.ceil(math.sqrt(N)))
        if D == 11:
            g = int(math.ceil(math.sqrt(N / 5.0)))
        uv = _grid_uv(max(g, 1), 0.45)
        noll = list(range(2, 2 + D))
        C = np.zeros((N, D))
        if D == 11:
            zs = np.linspace(-20.0, 20.0, 5)
            pts = np.array([(u, v, z) for z in zs for (u, v) in uv])[:N]
            C[:, 0:2] = _tilts(pts[:, :2], R)
            C[:, 2] = pts[:, 2]
            norm = np.stack([pts[:, 0] / 0.45, pts[:, 1] / 0.45, pts[:, 2] / 20.0], axis=1)
            exps, alpha = _quadratic_field(rng, 8, 0.5, 3)
            C[:, 3:11] = _eval_field(exps, alpha, norm) + rng.normal(0.0, 0.3, size=(N, 8))
            target = rng.uniform(0.5, 1.0, size=N)
        else:
            uvs = uv[:N]
            C[:, 0:2] = _tilts(uvs, R)
            vals, _ = _patch_coeffs(rng, uvs / 0.45, D - 2, 50, 0.5)
            C[:, 2:D] = vals
            target = np.ones(N)
        amp = gaussian_amplitude(nx, ny) if D != 11 else flat_amplitude(nx, ny)
        phase0 = random_phase(rng, nx, ny)
        out.append(Problem(f"c5_h{h:02d}_{nx}x{ny}_N{N}_D{D}", nx, ny, amp, phase0, noll,
                           C.astype(np.float32), target.astype(np.float32), 50))
    return out


C5_SMALL_SIZES = [(256, 256), (384, 384), (512, 512)]


def config_c5_small(seed: int = 1, count: int = 64) -> list:
    """Many small holograms: the c5 recipe with grids of 256^2 to 512^2 and
    N log-uniform in [10, 300], where no single member fills the GPU (one
    launch per phase for the whole batch against one graph per hologram)."""
    return config_c5(seed, count=count, sizes=C5_SMALL_SIZES, max_spots=300)


CONFIG_NAMES = ("c1", "c2", "c3", "c4")


def make_config(name: str, seed: int = 1) -> Problem:
    return {"c1": config_c1, "c2": config_c2, "c3": config_c3, "c4": config_c4}[name](seed)


def random_problem(seed: int, nx: int, ny: int, N: int, noll, tilt_span: float = 0.45,
                   aberr_sigma: float = 0.5, defocus_max: float = 0.0, flat: bool = False,
                   target_range=(1.0, 1.0)) -> Problem:
    """Small random problem for parity sweeps: random spot positions within
    +-tilt_span Nyquist, other modes N(0, aberr_sigma), optional defocus
    uniform in [-defocus_max, defocus_max] (Noll 4 column, if present)."""
    rng = np.random.default_rng(seed)
    R = _radius(nx, ny)
    noll = list(noll)
    D = len(noll)
    C = rng.normal(0.0, aberr_sigma, size=(N, D))
    uv = rng.uniform(-tilt_span, tilt_span, size=(N, 2))
    for k, j in enumerate(noll):
        if j == 2:
            C[:, k] = uv[:, 0] * math.pi * R
        elif j == 3:
            C[:, k] = uv[:, 1] * math.pi * R
        elif j == 4 and defocus_max > 0:
            C[:, k] = rng.uniform(-defocus_max, defocus_max, size=N)
    amp = flat_amplitude(nx, ny) if flat else gaussian_amplitude(nx, ny)
    target = rng.uniform(target_range[0], target_range[1], size=N)
    return Problem(f"rand_{nx}x{ny}_N{N}_D{D}_s{seed}", nx, ny, amp, random_phase(rng, nx, ny),
                   noll, C.astype(np.float32), target.astype(np.float32), 10)


def pixel_sample(nx: int, ny: int, frac: float, seed: int) -> np.ndarray:
    """Seeded random subset of the flat pixel indices (each pixel kept with
    probability `frac`), sorted. A problem restricted to these pixels is the
    same problem with the illumination amplitude set to 0 everywhere else."""
    rng = np.random.default_rng(seed)
    keep = rng.random(nx * ny) < frac
    return np.flatnonzero(keep)


def masked_amplitude(p: Problem, idx: np.ndarray) -> Problem:
    """Copy of `p` whose amplitude is kept on the flat pixels `idx` and is 0
    elsewhere (no renormalisation: the weighted-GS loop is scale-invariant)."""
    amp = np.zeros(p.M, np.float32)
    amp[idx] = p.amp.ravel()[idx]
    return dataclasses.replace(p, amp=amp.reshape(p.ny, p.nx), name=p.name + f"_sampled{idx.size}")
