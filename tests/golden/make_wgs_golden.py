"""Writes wgs_full_loops.json: the oracle's final spot uniformity and
efficiency after the full weighted-GS loops of the two benchmark workloads.

Calls only `oracle/` (the complex128 loop of Sec. II / Sec. III, readings
of its update rule and metrics in oracle/wgs.py) and `workloads/` (seeded
inputs). Nothing here comes from the CUDA path.

  * anisoplanatic 2D array: 1024 x 1024, N = 400, D = 10, 50 iterations,
    every pixel (the exact workload the benchmark times);
  * 3D volume: 1920 x 1152, N = 2000, D = 11, 100 iterations, on a seeded
    random 1/16 of the pixels: the illumination amplitude is 0 elsewhere,
    so the GPU runs the same loop on the full grid with that amplitude,
    and the oracle sums over the kept pixels only (a zero-amplitude pixel
    adds nothing to any forward, and its phase reaches no later step).

The loop amplifies differences in its inputs: the final uniformity moves by
about 1e-3 when the starting phase moves by a fraction of its fp32 spacing.
So, besides the run on the given phase, `--ensemble K` runs the oracle on K
starting phases that each round to the same float32 values (the given
phase plus a seeded uniform offset within half a float32 spacing per
pixel): the spread of their final uniformity is how far the float32 inputs
themselves leave the result open.

  python tests/golden/make_wgs_golden.py [--only c2|c3] [--ensemble K] [--skip-base]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import wgs, zernike  # noqa: E402
from workloads import config_c2, config_c3, masked_amplitude, pixel_sample  # noqa: E402

OUT = os.path.join(HERE, "wgs_full_loops.json")
C3_FRAC, C3_SEED = 1.0 / 16.0, 7


def sub_ulp_offset(phase32: np.ndarray, seed: int) -> np.ndarray:
    """A float64 offset, uniform within half the float32 spacing of each
    phase value, so that phase32 + offset rounds back to phase32. The
    spacing is the smaller of the two sides' (at a power of two the one
    below is half the one above)."""
    rng = np.random.default_rng(seed)
    a = np.abs(phase32.astype(np.float32))
    up = np.spacing(a).astype(np.float64)
    down = np.where(a > 0, a.astype(np.float64) - np.nextafter(a, np.float32(0)).astype(np.float64), up)
    return rng.uniform(-0.499, 0.499, size=phase32.shape) * np.minimum(up, down)


def _run(p, idx, workers, seed=None):
    Z = zernike.basis(p.nx, p.ny, p.noll)
    amp = p.amp.astype(np.float64).ravel()
    ph0 = p.phase0.astype(np.float64).ravel()
    if seed is not None:
        ph0 = ph0 + sub_ulp_offset(p.phase0.ravel(), seed)
    if idx is not None:
        Z, amp, ph0 = Z[:, idx], amp[idx], ph0[idx]
    t0 = time.time()
    r = wgs.run(amp, ph0, p.coeff.astype(np.float64), Z, p.target.astype(np.float64), p.iters, workers=workers)
    return {
        "nx": p.nx, "ny": p.ny, "N": p.N, "D": p.D, "iters": p.iters, "seed": 1,
        "pixels_summed": int(amp.size),
        "uniformity": r.uniformity,
        # efficiency over the pixels summed (the GPU's M is nx * ny: scale by pixels_summed / (nx ny))
        "efficiency": r.efficiency,
        "history": [float(u) for u in r.history],
        "oracle_seconds": time.time() - t0,
    }


ENSEMBLE_SEED0 = 1000


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--only", choices=["c2", "c3"], default=None)
    ap.add_argument("--ensemble", type=int, default=0)
    ap.add_argument("--skip-base", action="store_true")
    args = ap.parse_args()
    workers = os.cpu_count() or 1
    out = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            out = json.load(f)
    out["_source"] = ("oracle.wgs.run (complex128) on workloads.config_c2(1) / config_c3(1); "
                      "written by tests/golden/make_wgs_golden.py")

    def save():
        with open(OUT, "w") as f:
            json.dump(out, f, indent=1)

    jobs = []
    if args.only in (None, "c2"):
        jobs.append(("c2", config_c2(1), None, {}))
    if args.only in (None, "c3"):
        p = config_c3(1)
        idx = pixel_sample(p.nx, p.ny, C3_FRAC, C3_SEED)
        jobs.append(("c3_sampled", masked_amplitude(p, idx), idx, {"sample_frac": C3_FRAC, "sample_seed": C3_SEED}))
    for key, p, idx, extra in jobs:
        if not args.skip_base or key not in out:
            out[key] = _run(p, idx, workers) | extra
            print(key, out[key]["uniformity"], out[key]["efficiency"], flush=True)
            save()
        ens = out[key].setdefault("ensemble", [])
        for k in range(len(ens), len(ens) + args.ensemble):
            r = _run(p, idx, workers, seed=ENSEMBLE_SEED0 + k)
            ens.append({"seed": ENSEMBLE_SEED0 + k, "uniformity": r["uniformity"], "efficiency": r["efficiency"]})
            print(key, "ensemble", k, r["uniformity"], flush=True)
            save()
    save()


if __name__ == "__main__":
    main()
