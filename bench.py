"""Benchmark of the aberration-space holography hot path on GB300.

One step = one complete weighted-GS solve of the anisoplanatic 2D workload
(1024 x 1024 SLM, N = 400 spots in a 20 x 20 grid over +-0.45 Nyquist,
50 isoplanatic patches, D = 10 Zernike modes, 50 iterations + the final
forward and metrics), inputs resident in HBM. The metric counts spot-kernel
terms (one (spot, pixel) phase + sincos + complex MAC) of the forward and
adjoint passes: terms/step = (2 * iters + 1) * N * M.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun each rank solves its own independent hologram (weak scaling,
no collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "spot-kernel Gterm/s (N*M phase+sincos+cMAC) fwd+adj; WGS iter/s at 1024^2 x 400"
UNIT = "Gterm/s"
L2_FLUSH_BYTES = 256 << 20
# Nominal pipe rates per SM per clock; the bench lines use the rates the
# library's probe (ash_probe_rates) measures on the GPU at hand instead.
MUFU_PER_CLK_PER_SM = 16          # sin.approx / cos.approx results
MUFU_PER_TERM = 2                 # one sin and one cos per term
FP32_PER_CLK_PER_SM = 128         # FP32 lane results (an FFMA2 gives two)
# FP32 lane-operations per term of this design: on the MUFU path the
# argument scaling (1) and the complex multiply-accumulate (4); on the FP32
# path the sin / cos polynomial with its reduction (16) and the same
# multiply-accumulate (4)
FP32_PER_TERM_MUFU_PATH = 5
FP32_PER_TERM_POLY_PATH = 20
MAX_SM_MHZ = 2070.0               # nominal maximum SM clock (MEASURED_PEAKS.json's sm_max_mhz when present)
# ncu DRAM traffic of the transforms: a summary under profiles/ whose rows
# name the kernel, its dram bytes per launch and the hash of the kernel
# sources the counters were taken on (reported only while they match)
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic_k_tc_transforms_c2_1024x1024_N400_D10.md")
TRAFFIC_SOURCES = ["common.cuh", "tc_common.cuh", "tc_kernels.cuh", "tc_launch.h", "tc.cu"]


def alu_terms_per_clk_per_sm(mufu=MUFU_PER_CLK_PER_SM, fp32=FP32_PER_CLK_PER_SM):
    """Two-pipe ceiling of a term (sin, cos, complex MAC): a share a of the
    terms takes its sin / cos on the FP32 pipe, the rest on the MUFU pipe;
    the best a equalises the two pipes' times,
    MUFU_PER_TERM (1 - a) / MUFU rate = (f_m (1 - a) + f_p a) / FP32 rate."""
    m, F = MUFU_PER_TERM / mufu, 1.0 / fp32
    fm, fp = FP32_PER_TERM_MUFU_PATH, FP32_PER_TERM_POLY_PATH
    a = (m - F * fm) / (m + F * (fp - fm))
    return 1.0 / (m * (1.0 - a))


def planned_terms_per_clk_per_sm(D, mufu=MUFU_PER_CLK_PER_SM, fp32=FP32_PER_CLK_PER_SM):
    """The FP32/SFU roofline of a term with the phase on the FP32 pipe: D
    FMAs of the phase, about 3 FP32 operations of range reduction and 4 of
    the complex multiply-accumulate (D + 7 lane operations), and one sin and
    one cos on the MUFU: min(FP32 rate / (D + 7), MUFU rate / 2)."""
    return min(fp32 / (D + 7.0), mufu / 2.0)


def max_sm_mhz():
    """The GPU's maximum SM clock: MEASURED_PEAKS.json (driver-written) when
    present, else the nominal figure."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            v = float(json.load(f).get("sm_max_mhz") or 0.0)
        if v > 0:
            return v, "MEASURED_PEAKS.json sm_max_mhz"
    except (OSError, ValueError):
        pass
    return MAX_SM_MHZ, "nominal maximum SM clock"


def probe_rates(lib, stream_ptr):
    """Per-SM unit rates measured by the library's probe on this GPU."""
    import ctypes
    from paper_2505_08777_gb300 import _lib
    out = (ctypes.c_double * 6)()
    _lib.check(lib.ash_probe_rates(out, stream_ptr), "ash_probe_rates")
    v = list(out)
    return {"mufu_sincos_per_clk_sm": v[0], "ffma_lanes_per_clk_sm": v[1], "ffma2_lanes_per_clk_sm": v[2],
            "ex2_per_clk_sm": v[3], "probe_sm_mhz": v[4], "sms": int(v[5]),
            "how": "ash_probe_rates: one 1024-thread CTA per SM, independent chains, SM cycle counter"}


def source_hash(names=TRAFFIC_SOURCES):
    import hashlib
    h = hashlib.sha256()
    for n in names:
        with open(os.path.join(ROOT, "paper_2505_08777_gb300", "csrc", n), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:12]


def ncu_traffic(kernel):
    """dram bytes per launch of `kernel` from the committed ncu summary, if
    it was taken on the current kernel sources; else None."""
    try:
        rows = open(TRAFFIC_FILE).read().splitlines()
    except OSError:
        return None
    want = source_hash()
    for r in rows:
        cells = [c.strip() for c in r.strip().strip("|").split("|")]
        if len(cells) >= 3 and cells[0] == kernel and cells[2] == want:
            try:
                return float(cells[1])
            except ValueError:
                return None
    return None


def roofline_alu(achieved, D, rates, kernel, algorithmic):
    """roofline object of an ALU-bound transform: peak = the FP32/SFU
    roofline R_terms = SMs x f_clk x min(FP32 / (D + 7), MUFU / 2) from the
    probe's measured rates at the maximum SM clock; the design's two-pipe
    ceiling (tensor-core phases, sin/cos shared by the MUFU and an FP32
    polynomial) and the MUFU-only bound beside it."""
    mhz, mhz_src = max_sm_mhz()
    sms = rates["sms"]
    mufu = rates["mufu_sincos_per_clk_sm"]
    fp32 = max(rates["ffma_lanes_per_clk_sm"], rates["ffma2_lanes_per_clk_sm"])
    per_sm = planned_terms_per_clk_per_sm(D, mufu, fp32)
    peak = sms * per_sm * mhz * 1e6 / 1e9
    two = sms * alu_terms_per_clk_per_sm(mufu, fp32) * mhz * 1e6 / 1e9
    mufu_only = sms * (mufu / MUFU_PER_TERM) * mhz * 1e6 / 1e9
    return {
        "bound": "alu", "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "Gterm/s",
        "frac": achieved / peak, "traffic": ncu_traffic(kernel.split(" ")[0]),
        "peak_basis": f"R_terms = SMs x f_clk x min(FP32/(D+7), MUFU/2) = {sms} x {mhz:.0f} MHz ({mhz_src}) x "
                      f"min({fp32:.1f}/{D + 7}, {mufu:.2f}/2) = {per_sm:.2f} terms/clk/SM; rates measured by "
                      f"ash_probe_rates on this GPU",
        "two_pipe_peak": two, "frac_two_pipe": achieved / two,
        "two_pipe_basis": f"tensor-core phases; a term costs 2 MUFU + {FP32_PER_TERM_MUFU_PATH} FP32 or "
                          f"{FP32_PER_TERM_POLY_PATH} FP32 (polynomial sin/cos), best split "
                          f"{alu_terms_per_clk_per_sm(mufu, fp32):.2f} terms/clk/SM",
        "mufu_only_peak": mufu_only, "frac_mufu_only": achieved / mufu_only,
        "algorithmic_per_launch": algorithmic, "rates": rates,
    }


WORKLOAD_TEXT = {
    "c2": "anisoplanatic 2D tweezer array: SLM {nx}x{ny}, N={N} spots (20x20 grid, +-0.45 Nyquist, "
          "50 isoplanatic patches x 8 modes), D={D} (Noll 2-11), {iters} WGS iterations per step",
    "c3": "3D volumetric spots: SLM {nx}x{ny} flat-top, N={N} spots (20x20x5 lattice, defocus in [-20, 20] rad), "
          "D={D} (Noll 2-12), {iters} WGS iterations per step",
}


def _workload_config(p, iters, cfg="c2"):
    return {
        "workload": WORKLOAD_TEXT[cfg].format(nx=p.nx, ny=p.ny, N=p.N, D=p.D, iters=iters),
        "nx": p.nx, "ny": p.ny, "N": p.N, "D": p.D, "iters_per_step": iters,
        "terms_per_step": (2 * iters + 1) * p.N * p.M,
        "l2": "flushed between steps (256 MiB write)",
        "parallelism": "one independent hologram per GPU",
    }


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--shard", action="store_true",
                    help="c2 as ONE hologram sharded by pixel rows over the ranks: band handles, one NCCL "
                         "all-reduce of the N spot fields per forward, replicated spot update, local adjoint "
                         "(strong scaling); default: one independent hologram per rank (weak scaling)")
    ap.add_argument("--batch-solo-terms", type=int, default=None,
                    help="c5: N*M threshold above which a batch member runs standalone in the batch's graph "
                         "(default: the library's)")
    ap.add_argument("--config", default="c2", choices=["c2", "c3", "c4", "c5", "c5s", "zsub", "cg", "peaks"],
                    help="c2 (default, the headline): anisoplanatic 2D WGS; c3: 3D volume WGS; "
                         "c4: autograd + Adam on 8 holograms; c5: 64 uneven holograms, batched vs looped; "
                         "c5s: 64 small uneven holograms (256^2-512^2, N 10-300), batched vs looped; "
                         "zsub: simulated Zernike-subtraction calibration round on the c2 system; "
                         "cg: conjugate-gradient top-hat refinement after WGS on c2; "
                         "peaks: the per-SM pipe rates the roofline is built from (ash_probe_rates)")
    return ap.parse_args()


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _scratch_dir() -> str:
    """Where the clock samples and the batch autotuner cache go
    (ASH_BENCH_DIR, else the system temporary directory)."""
    import tempfile
    d = os.environ.get("ASH_BENCH_DIR") or tempfile.gettempdir()
    os.makedirs(d, exist_ok=True)
    return d


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(_scratch_dir(), f"clocks_rank{gpu_index}.csv")

    def __enter__(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        top = max(sm)
        loaded = [s for s in sm if s >= 0.5 * top] or sm
        return {"sm_mhz": float(np.median(loaded)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


def _cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_sample(p, Z, workers):
    """One WGS iteration of the workload on the CPU oracle (forward + spot
    update + adjoint over the full grid and all spots). Returns (terms, s)."""
    from oracle import transform, wgs
    A = p.amp.astype(np.float64).ravel()
    C = p.coeff.astype(np.float64)
    t0 = time.perf_counter()
    E = transform.forward(transform.field(A, p.phase0), C, Z, workers=workers)
    w, y = wgs.weight_update(E, p.target.astype(np.float64), p.target)
    g = transform.adjoint(y, C, Z, workers=workers)
    transform.phase_of(g)
    dt = time.perf_counter() - t0
    return 2 * p.N * p.M, dt


# Pixel-sampled oracle timings: the transforms' sums run over pixels, so the
# oracle on every stride-th pixel does the same work per term; the stride
# bounds the sample (the forward and the WGS adjoint use a thread pool, the
# gradient's adjoint and moments run single-threaded).
ORACLE_SAMPLE_TERMS = {"wgs": 1.5e9, "grad": 2e8}


def oracle_sampled(kind, ps, workers):
    """kind "wgs": one WGS iteration (forward, spot update, adjoint, arg) per
    problem; "grad": the forward, then dL/dphi and dL/dC (adjoint and
    moments). Returns (terms, seconds, stride)."""
    from oracle import grad, transform, wgs, zernike
    per_term = 2 if kind == "wgs" else 3
    total = sum(per_term * p.N * p.M for p in ps)
    stride = max(1, int(math.ceil(total / ORACLE_SAMPLE_TERMS[kind])))
    terms, secs = 0, 0.0
    for p in ps:
        idx = np.arange(0, p.M, stride)
        Z = zernike.basis(p.nx, p.ny, p.noll)[:, idx]
        A = p.amp.astype(np.float64).ravel()[idx]
        ph = p.phase0.astype(np.float64).ravel()[idx]
        C = p.coeff.astype(np.float64)
        T = p.target.astype(np.float64)
        t0 = time.perf_counter()
        E = transform.forward(transform.field(A, ph), C, Z, workers=workers)
        if kind == "wgs":
            _, y = wgs.weight_update(E, T, T)
            transform.phase_of(transform.adjoint(y, C, Z, workers=workers))
        else:
            grad.backward(A, ph, C, Z, grad.grad_E(E, T))
        secs += time.perf_counter() - t0
        terms += per_term * p.N * idx.size
    return terms, secs, stride


def _sampled_baseline(kind, ps, what):
    cores = _cpu_cores()
    terms, secs, stride = oracle_sampled(kind, ps, cores)
    return {"value": terms / secs / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{what} over every {stride}-th pixel ({terms:.3g} terms), numpy complex128",
            "seconds": secs}


def run_reference(args):
    rank, world, _ = _dist()
    if rank != 0:
        return 0
    from oracle import zernike
    from workloads import config_c2
    p = config_c2(1)
    Z = zernike.basis(p.nx, p.ny, p.noll)
    cores = _cpu_cores()
    for _ in range(args.warmup):
        oracle_sample(p, Z, cores)
    terms, secs = 0, 0.0
    for _ in range(args.steps):
        t, dt = oracle_sample(p, Z, cores)
        terms += t
        secs += dt
    val = terms / secs / 1e9
    sample = "one WGS iteration (forward + update + adjoint, full 1024x1024 grid, all 400 spots) per step"
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c128", "data": "synthetic",
        "config": _workload_config(p, 1) | {"oracle": "numpy complex128, pixel chunks x all spots, thread pool"},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def main():
    args = _args()
    if args.impl == "reference":
        return run_reference(args)
    if args.config == "c4":
        return bench_autograd(args)
    if args.config in ("c5", "c5s"):
        return bench_batch(args)
    if args.config == "zsub":
        return bench_zsub(args)
    if args.config == "cg":
        return bench_cg(args)
    if args.config == "peaks":
        return bench_peaks(args)
    if args.shard:
        return bench_shard(args)
    import torch

    from paper_2505_08777_gb300 import Hologram
    from workloads import config_c2, config_c3

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    p = (config_c2 if args.config == "c2" else config_c3)(1 + rank)
    iters = p.iters
    terms_per_step = (2 * iters + 1) * p.N * p.M
    stream = torch.cuda.current_stream()

    t0 = time.perf_counter()
    h = Hologram(torch.from_numpy(p.amp).to(dev), torch.from_numpy(p.coeff).to(dev), noll=p.noll)
    create_s = time.perf_counter() - t0
    phase0 = torch.from_numpy(p.phase0).to(dev)
    target = torch.from_numpy(p.target).to(dev)
    phase = torch.empty_like(phase0)
    w = torch.empty_like(target)
    E = torch.empty(p.N, dtype=torch.complex64, device=dev)
    met = torch.empty(4, dtype=torch.float32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def step():
        phase.copy_(phase0)
        w.copy_(target)
        h.wgs(phase, w, target, iters, E_out=E, metrics_out=met)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()

    # ---- timed region: K steps, per-step CUDA events, L2 flushed in between
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        for k in range(args.steps):
            flush.zero_()
            phase.copy_(phase0)
            w.copy_(target)
            ev[k][0].record(stream)
            h.wgs(phase, w, target, iters, E_out=E, metrics_out=met)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = float(sum(step_ms))
    uniformity = float(met[0].item())
    t = torch.tensor([total_ms], device=dev)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    total_ms_max = float(t.item())
    value = world * terms_per_step * args.steps / (total_ms_max * 1e-3) / 1e9

    # ---- end to end through the public API with host buffers
    ph_host = torch.from_numpy(p.phase0).pin_memory()
    T_host = torch.from_numpy(p.target).pin_memory()
    ph_out = torch.empty_like(ph_host).pin_memory()
    E_out = torch.empty(p.N, dtype=torch.complex64).pin_memory()
    met_out = torch.empty(4, dtype=torch.float32).pin_memory()
    e2e_ms = 0.0
    for k in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        phase.copy_(ph_host, non_blocking=True)
        target.copy_(T_host, non_blocking=True)
        w.copy_(target)
        h.wgs(phase, w, target, iters, E_out=E, metrics_out=met)
        ph_out.copy_(phase, non_blocking=True)
        E_out.copy_(E, non_blocking=True)
        met_out.copy_(met, non_blocking=True)
        b.record(stream)
        b.synchronize()
        e2e_ms += a.elapsed_time(b)
    h2d = ph_host.numel() * 4 + T_host.numel() * 4
    d2h = ph_out.numel() * 4 + E_out.numel() * 8 + 16
    t = torch.tensor([e2e_ms], device=dev)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    e2e_value = world * terms_per_step * args.steps / (float(t.item()) * 1e-3) / 1e9

    # ---- per-kernel timing: ash_profile records CUDA events around each kernel
    # on this stream, back to back as in the WGS loop (no L2 flush between the
    # kernels: a WGS step does none either)
    import ctypes

    from paper_2505_08777_gb300 import _lib
    L = _lib.load()
    rng = np.random.default_rng(5)
    y = torch.from_numpy((rng.normal(size=p.N) + 1j * rng.normal(size=p.N)).astype(np.complex64)).to(dev)
    names = ["forward", "forward_reduce", "adjoint", "adjoint_fixup", "wgs_update", "grad_coeff"]
    acc = np.zeros(6)
    reps = 20
    ms = (ctypes.c_float * 6)()
    for r in range(reps + 1):
        _lib.check(L.ash_profile(h.handle, ctypes.c_void_p(phase0.data_ptr()), ctypes.c_void_p(y.data_ptr()), ms,
                                 ctypes.c_void_p(stream.cuda_stream)), "ash_profile")
        if r > 0:
            acc += np.array(list(ms))
    kms = dict(zip(names, (acc / reps).tolist()))
    NM = p.N * p.M
    gterm = {k: NM / (kms[k] * 1e-3) / 1e9 for k in ("forward", "adjoint", "grad_coeff") if kms[k] > 0}

    clk = clocks.summary()
    rates = probe_rates(L, ctypes.c_void_p(stream.cuda_stream))
    dom = "forward" if kms["forward"] >= kms["adjoint"] else "adjoint"
    P = 8 if p.D <= 12 else 4
    linfo = h.launch_info()
    fwd_tc = bool(linfo["kernels"] & 4)
    adj_tc = bool(linfo["kernels"] & 2)
    # K-atoms per tensor-core operand row: one for D <= 10, and for D = 11
    # when the basis holds both tilts (their two-slot exact form)
    NA = 1 if 3 * p.D <= 32 or (3 * (p.D - 2) + 4 <= 32 and 2 in p.noll and 3 in p.noll) else 2
    kernel_names = {"forward": (f"k_tc_forward<{NA}> (spot-stationary: tcgen05 split-tf32 MMA of 128 spots x 64 "
                                f"pixels into TMEM, sincos + packed complex MAC)") if fwd_tc else
                               f"k_forward<D={p.D},P={P}> (pixel-stationary forward, warp transpose reduction)",
                    "adjoint": (f"k_tc_adjoint<{NA},true> (pixel-stationary: tcgen05 split-tf32 MMA of 128 pixels x 64 "
                                f"spots into TMEM, sincos + packed complex MAC, arg epilogue)") if adj_tc else
                               f"k_adjoint<D={p.D},P={P}> (pixel-stationary adjoint, arg epilogue)"}
    achieved = gterm[dom]
    roofline = roofline_alu(achieved, p.D, rates, kernel_names[dom], f"N*M = {NM} terms")
    roofline["per_kernel_frac"] = {k: v / roofline["peak"] for k, v in gterm.items()}
    if clk.get("sm_mhz"):
        roofline["frac_at_sampled_clock"] = achieved / (roofline["peak"] * clk["sm_mhz"] / max_sm_mhz()[0])
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic", "config": _workload_config(p, iters, args.config),
        "wgs_iter_per_s": world * iters * args.steps / (total_ms_max * 1e-3),
        "final_uniformity": uniformity,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(L.ash_wgs_launches(h.handle, iters)) * args.steps,
        "roofline": roofline,
        "kernels": {"ms": kms, "gterm_s": gterm, "create_s": create_s, "launch_info": linfo},
        "clocks": clk,
    }
    if args.config != "c2":
        line["metric"] = f"spot-kernel Gterm/s (N*M phase+sincos+cMAC) fwd+adj; WGS iter/s, workload {args.config}"
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.config == "c2":
        from oracle import zernike
        Z = zernike.basis(p.nx, p.ny, p.noll)
        cores = _cpu_cores()
        terms, secs = oracle_sample(p, Z, cores)
        line["cpu_baseline"] = {"value": terms / secs / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": "one WGS iteration (forward + update + adjoint) over the full 1024x1024 "
                                          "grid and all 400 spots, numpy complex128 thread pool",
                                "seconds": secs}
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.config == "c3":
        line["cpu_baseline"] = _sampled_baseline("wgs", [p], "one WGS iteration (forward + update + adjoint)")
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def _peak_gterm(torch, dev, D=10):
    """R_terms (the FP32/SFU roofline, see roofline_alu) for D modes from
    the probe's measured rates on this GPU, at the maximum SM clock."""
    from paper_2505_08777_gb300 import _lib
    rates = probe_rates(_lib.load(), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    mufu = rates["mufu_sincos_per_clk_sm"]
    fp32 = max(rates["ffma_lanes_per_clk_sm"], rates["ffma2_lanes_per_clk_sm"])
    return rates["sms"] * planned_terms_per_clk_per_sm(D, mufu, fp32) * max_sm_mhz()[0] * 1e6 / 1e9


def bench_autograd(args):
    """c4: gradient descent (Adam) on the spot-intensity loss for a batch of 8
    holograms (1024^2, N=1024, D=10), gradients w.r.t. phase and C through the
    hand-written adjoint. One step = forward + backward for all 8 + Adam."""
    import torch

    from paper_2505_08777_gb300 import Hologram
    from paper_2505_08777_gb300.autograd import spot_field, spot_intensity_loss
    from workloads import config_c4

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    ps = [config_c4(s) for s in range(1, 9)]
    hs = [Hologram(torch.from_numpy(p.amp).to(dev), torch.from_numpy(p.coeff).to(dev), noll=p.noll) for p in ps]
    phases = [torch.from_numpy(p.phase0).to(dev).requires_grad_(True) for p in ps]
    coeffs = [torch.from_numpy(p.coeff).to(dev).requires_grad_(True) for p in ps]
    targets = [torch.from_numpy(p.target).to(dev) for p in ps]
    opt = torch.optim.Adam(phases + coeffs, lr=0.01)
    stream = torch.cuda.current_stream()

    def step():
        opt.zero_grad(set_to_none=False)
        total = 0.0
        for h, ph, c, t in zip(hs, phases, coeffs, targets):
            loss = spot_intensity_loss(spot_field(h, ph, c), t)
            loss.backward()
            total = total + loss.detach()
        opt.step()
        return total

    first = step()
    for _ in range(max(args.warmup, 3) - 1):
        step()
    torch.cuda.synchronize()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    ms = 0.0
    with ClockSampler(0) as clocks:
        for _ in range(args.steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            last = step()
            b.record(stream)
            b.synchronize()
            ms += a.elapsed_time(b)
    terms = sum(3 * p.N * p.M for p in ps)     # forward + adjoint (dphase) + moment pass (dC)
    value = terms * args.steps / (ms * 1e-3) / 1e9
    graphed = _graphed_autograd_step(args, hs, phases, coeffs, targets, spot_field, spot_intensity_loss, flush,
                                     terms)
    step_kernels = _autograd_step_kernels(hs, phases, coeffs)
    line = {"metric": "autograd spot-kernel Gterm/s (fwd + dphase adjoint + dC moments), Adam steps/s, workload c4",
            "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "8 holograms 1024x1024, N=1024 (32x32 grid), D=10; loss sum (I/mean I - t)^2, "
                                   "t ~ U[0.5, 1.5]; Adam lr 0.01 on phase and C; one step = 8 x (fwd + bwd) + Adam",
                       "l2": "flushed between steps (256 MiB write)"},
            "adam_steps_per_s": args.steps / (ms * 1e-3),
            "loss_first_step": float(first.item()), "loss_last_step": float(last.item()),
            "graph_captured_step": graphed,
            "gpu_launches": None if step_kernels is None else step_kernels * args.steps,
            "clocks": clocks.summary()}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = _sampled_baseline("grad", ps[:1], "one hologram's forward + dL/dphi + dL/dC")
    print(json.dumps(line))
    return 0


def _graph_kernel_nodes(cu, g):
    """Kernel nodes of a CUDA graph (driver API), child graphs included."""
    import ctypes
    n = ctypes.c_size_t(0)
    if cu.cuGraphGetNodes(g, None, ctypes.byref(n)) != 0:
        return None
    nodes = (ctypes.c_void_p * n.value)()
    if n.value and cu.cuGraphGetNodes(g, nodes, ctypes.byref(n)) != 0:
        return None
    k = 0
    for nd in nodes:
        t = ctypes.c_int(-1)
        if cu.cuGraphNodeGetType(ctypes.c_void_p(nd), ctypes.byref(t)) != 0:
            return None
        if t.value == 0:       # CU_GRAPH_NODE_TYPE_KERNEL
            k += 1
        elif t.value == 4:     # CU_GRAPH_NODE_TYPE_GRAPH
            child = ctypes.c_void_p()
            if cu.cuGraphChildGraphNodeGetGraph(ctypes.c_void_p(nd), ctypes.byref(child)) != 0:
                return None
            m = _graph_kernel_nodes(cu, child)
            if m is None:
                return None
            k += m
    return k


def _kernels_enqueued(fn, stream):
    """Kernels fn() enqueues on `stream` (a torch side stream): counted from a
    stream capture through the CUDA driver API, a graph that is inspected and
    destroyed, never launched. None if the capture or the inspection fails."""
    import ctypes
    try:
        cu = ctypes.CDLL("libcuda.so.1")
    except OSError:
        return None
    s = ctypes.c_void_p(stream.cuda_stream)
    if cu.cuStreamBeginCapture_v2(s, 2) != 0:   # CU_STREAM_CAPTURE_MODE_RELAXED
        return None
    g = ctypes.c_void_p()
    try:
        fn()
    finally:
        rc = cu.cuStreamEndCapture(s, ctypes.byref(g))
    if rc != 0 or not g.value:
        return None
    try:
        return _graph_kernel_nodes(cu, g)
    finally:
        cu.cuGraphDestroy(g)


def _autograd_step_kernels(hs, phases, coeffs):
    """The library kernels of one c4 step: per hologram the calls SpotField
    makes (coefficients and forward; then ash_grad for both gradients, the
    handle still holding those coefficients), with preallocated outputs so
    that nothing else is enqueued."""
    import ctypes

    import torch
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    cplx = dict(dtype=torch.complex64, device=phases[0].device)
    outs = [(torch.empty(c.shape[0], **cplx), torch.zeros(c.shape[0], **cplx), torch.empty_like(ph), torch.empty_like(c))
            for ph, c in zip(phases, coeffs)]
    torch.cuda.synchronize()

    def calls():
        for h, ph, c, (E, gE, dph, dC) in zip(hs, phases, coeffs, outs):
            h.set_coefficients(c.detach(), stream=side)
            h.forward(ph.detach(), out=E, stream=side)
            rc = h._lib.ash_grad(h.handle, ctypes.c_void_p(ph.data_ptr()), ctypes.c_void_p(gE.data_ptr()),
                                 ctypes.c_void_p(dph.data_ptr()), ctypes.c_void_p(dC.data_ptr()),
                                 ctypes.c_void_p(side.cuda_stream))
            if rc != 0:
                raise RuntimeError(f"ash_grad status {rc} under capture")

    try:
        return _kernels_enqueued(calls, side)
    except Exception:   # noqa: BLE001 -- reported as null, the measurement stands
        return None


def _zsub_round_kernels(model, system, T, modes, deltas):
    """The library kernels of one calibration round: per order the C-ABI
    calls zernike_subtraction makes (baseline adjoint, sweep, estimate with
    subtraction, model coefficients), on preallocated buffers."""
    import ctypes

    import torch
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    K, N, D = len(deltas), model.N, model.D
    y = T.to(torch.complex64)
    phi = torch.empty((model.ny, model.nx), dtype=torch.float32, device=T.device)
    I = torch.empty((K, N), dtype=torch.float32, device=T.device)
    ds = torch.empty(N, dtype=torch.float32, device=T.device)
    C = model.coefficients().clone()
    dk = (ctypes.c_float * K)(*[float(v) for v in deltas])
    vp = ctypes.c_void_p
    sp = vp(side.cuda_stream)
    torch.cuda.synchronize()

    def calls():
        for d in modes:
            for rc in (model._lib.ash_adjoint(model.handle, vp(y.data_ptr()), None, vp(phi.data_ptr()), sp),
                       system._lib.ash_zsub_sweep(system.handle, vp(phi.data_ptr()), int(d), dk, K, vp(I.data_ptr()), sp),
                       model._lib.ash_zsub_estimate(vp(I.data_ptr()), dk, K, N, vp(ds.data_ptr()), vp(C.data_ptr()), D,
                                                    int(d), sp),
                       model._lib.ash_set_coefficients(model.handle, vp(C.data_ptr()), sp)):
                if rc != 0:
                    raise RuntimeError(f"status {rc} under capture")

    try:
        return _kernels_enqueued(calls, side)
    except Exception:   # noqa: BLE001 -- reported as null, the measurement stands
        return None


def _graphed_autograd_step(args, hs, phases, coeffs, targets, spot_field, spot_intensity_loss, flush, terms):
    """The same c4 step captured once as a CUDA graph (every library call is
    stream-ordered and allocation-free, Adam with capturable=True) and
    replayed: what the step costs without Python and launch overhead."""
    import torch
    try:
        opt = torch.optim.Adam(phases + coeffs, lr=0.01, capturable=True)

        def step():
            opt.zero_grad(set_to_none=False)
            total = None
            for h, ph, c, t in zip(hs, phases, coeffs, targets):
                loss = spot_intensity_loss(spot_field(h, ph, c), t)
                loss.backward()
                total = loss.detach() if total is None else total + loss.detach()
            opt.step()
            return total

        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            for _ in range(3):
                step()
        torch.cuda.current_stream().wait_stream(side)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            step()
        stream = torch.cuda.current_stream()
        for _ in range(max(args.warmup, 3)):
            graph.replay()
        torch.cuda.synchronize()
        ms = 0.0
        for _ in range(args.steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            graph.replay()
            b.record(stream)
            b.synchronize()
            ms += a.elapsed_time(b)
        return {"value": terms * args.steps / (ms * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": ms / args.steps,
                "adam_steps_per_s": args.steps / (ms * 1e-3)}
    except Exception as e:   # noqa: BLE001 -- reported, not fatal: the eager step is the measurement
        return {"unavailable": f"{type(e).__name__}: {e}"[:300]}


def bench_cg(args):
    """Conjugate-gradient top-hat refinement (paper Methods) on the c2
    workload (1024^2, N = 400, D = 10): from the phase of 50 WGS iterations,
    one step = 20 CG iterations on the spot-intensity loss with flat targets
    (two forwards and one gradient adjoint each, one CUDA graph)."""
    import torch

    from paper_2505_08777_gb300 import Hologram
    from workloads import config_c2

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    p = config_c2(1)
    h = Hologram(torch.from_numpy(p.amp).to(dev), torch.from_numpy(p.coeff).to(dev), noll=p.noll)
    T = torch.from_numpy(p.target).to(dev)
    ph0 = torch.from_numpy(p.phase0).to(dev)
    w = T.clone()
    _, met = h.wgs(ph0, w, T, p.iters)
    t = (T * T / torch.mean(T * T)).contiguous()
    iters = 20
    stream = torch.cuda.current_stream()
    ph = ph0.clone()
    L = h.cg_refine(ph, t, iters)
    E = h.forward(ph)
    I = (E.abs() ** 2) / (T * T)
    unif_after = float(1.0 - (I.max() - I.min()) / (I.max() + I.min()))
    for _ in range(max(args.warmup, 3) - 1):
        ph.copy_(ph0)
        h.cg_refine(ph, t, iters)
    torch.cuda.synchronize()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    ms = 0.0
    with ClockSampler(0) as clocks:
        for _ in range(args.steps):
            ph.copy_(ph0)
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            h.cg_refine(ph, t, iters)
            b.record(stream)
            b.synchronize()
            ms += a.elapsed_time(b)
    # end to end: the start phase and targets from pinned host memory, the
    # refined phase and the losses back
    ph_host = ph0.cpu().pin_memory()
    t_host = t.cpu().pin_memory()
    out_host = torch.empty_like(ph_host).pin_memory()
    L_host = torch.empty(iters + 1, dtype=torch.float32).pin_memory()
    e2e_ms = 0.0
    for _ in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        phd = ph_host.to(dev, non_blocking=True)
        td = t_host.to(dev, non_blocking=True)
        Ld = h.cg_refine(phd, td, iters)
        out_host.copy_(phd, non_blocking=True)
        L_host.copy_(Ld, non_blocking=True)
        b.record(stream)
        b.synchronize()
        e2e_ms += a.elapsed_time(b)
    terms = iters * 3 * p.N * p.nx * p.ny + 2 * p.N * p.nx * p.ny    # 3 transforms per iteration + the start
    value = terms * args.steps / (ms * 1e-3) / 1e9
    peak = _peak_gterm(torch, dev, p.D)
    line = {"metric": "conjugate-gradient refinement Gterm/s (2 forwards + 1 gradient adjoint per iteration), "
                      "CG iterations/s, workload cg",
            "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "c2 (SLM 1024x1024, N=400, D=10) after 50 WGS iterations; 20 CG iterations on "
                                   "L = sum (I/mean I - t)^2, t = T^2/mean T^2 (flat), theta 0.05 rad",
                       "l2": "flushed between steps (256 MiB write)"},
            "cg_iterations_per_s": iters * args.steps / (ms * 1e-3),
            "loss": {"after_wgs": float(L[0].item()), "after_cg": float(L[-1].item())},
            "uniformity": {"after_wgs": float(met[0].item()), "after_cg": unif_after},
            "e2e": {"value": terms * args.steps / (e2e_ms * 1e-3) / 1e9, "unit": UNIT,
                    "h2d_bytes_per_step": ph_host.numel() * 4 + t_host.numel() * 4,
                    "d2h_bytes_per_step": out_host.numel() * 4 + L_host.numel() * 4},
            "roofline": {"bound": "alu", "kernel": "whole CG step (transforms with the vector and scalar kernels)",
                         "achieved": value, "peak": peak, "unit": UNIT, "frac": value / peak, "traffic": None},
            "gpu_launches": h.graph_kernels(-iters) * args.steps, "clocks": clocks.summary()}
    print(json.dumps(line))
    return 0


def bench_zsub(args):
    """Simulated Zernike-subtraction calibration (paper Sec. III) on the c2
    system (1024^2, N = 400, D = 10): one step = one round over Noll 4-11,
    per order a superposition baseline (one adjoint), a 7-offset sweep (seven
    forwards through the column-shifted system) and the per-spot estimate and
    subtraction. Each step starts from the uncalibrated model."""
    import torch

    from paper_2505_08777_gb300 import Hologram, zernike_subtraction
    from workloads import ZSUB_DELTAS, config_zsub, zsub_model0

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    p = config_zsub(1)
    modes = [k for k, j in enumerate(p.noll) if j >= 4]
    system = Hologram(torch.from_numpy(p.amp).to(dev), torch.from_numpy(p.coeff).to(dev), noll=p.noll)
    C0 = torch.from_numpy(zsub_model0(p)).to(dev)
    model = Hologram(torch.from_numpy(p.amp).to(dev), C0.clone(), noll=p.noll)
    T = torch.from_numpy(p.target).to(dev)
    stream = torch.cuda.current_stream()
    mid = len(ZSUB_DELTAS) // 2      # the zero offset

    def step():
        model.set_coefficients(C0)
        return zernike_subtraction(model, system, T, modes, ZSUB_DELTAS, rounds=1)

    def brightness(C):
        model.set_coefficients(C)
        _, phi = model.adjoint(T.to(torch.complex64), want_field=False, want_phase=True)
        return float(system.zsub_sweep(phi, modes[0], [0.0]).mean().item())

    b0 = brightness(C0)
    for _ in range(max(args.warmup, 3)):
        C1, _ = step()
    b1 = brightness(C1.clone())
    torch.cuda.synchronize()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    ms = 0.0
    with ClockSampler(0) as clocks:
        for _ in range(args.steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step()
            b.record(stream)
            b.synchronize()
            ms += a.elapsed_time(b)
    # end to end through the public API: coefficients and targets from host
    # memory, the calibrated coefficients back to the host, every step
    C0_host = torch.from_numpy(zsub_model0(p)).pin_memory()
    T_host = torch.from_numpy(p.target).pin_memory()
    C_out = torch.empty_like(C0_host).pin_memory()
    torch.cuda.synchronize()
    e2e_ms = 0.0
    for _ in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        Cd = C0_host.to(dev, non_blocking=True)
        Td = T_host.to(dev, non_blocking=True)
        model.set_coefficients(Cd)
        Cr, _ = zernike_subtraction(model, system, Td, modes, ZSUB_DELTAS, rounds=1)
        C_out.copy_(Cr, non_blocking=True)
        b.record(stream)
        b.synchronize()
        e2e_ms += a.elapsed_time(b)
    round_kernels = _zsub_round_kernels(model, system, T, modes, ZSUB_DELTAS)
    per_order = 1 + len(ZSUB_DELTAS)               # one adjoint + K forwards
    terms = len(modes) * per_order * p.N * p.nx * p.ny
    value = terms * args.steps / (ms * 1e-3) / 1e9
    peak = _peak_gterm(torch, dev, p.D)
    line = {"metric": "Zernike-subtraction calibration Gterm/s (baseline adjoint + 7-offset sweep per order), "
                      "rounds/s, workload zsub",
            "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "c2 system as the optical system: SLM 1024x1024, N=400, D=10 (Noll 2-11); model "
                                   "starts with the spot tilts only; one round over Noll 4-11, offsets "
                                   "linspace(-1.5, 1.5, 7) rad, superposition baseline",
                       "l2": "flushed between steps (256 MiB write)"},
            "rounds_per_s": args.steps / (ms * 1e-3),
            "mean_spot_intensity_at_zero_offset": {"before": b0, "after_one_round": b1},
            "e2e": {"value": terms * args.steps / (e2e_ms * 1e-3) / 1e9, "unit": UNIT,
                    "h2d_bytes_per_step": C0_host.numel() * 4 + T_host.numel() * 4,
                    "d2h_bytes_per_step": C_out.numel() * 4},
            "roofline": {"bound": "alu", "kernel": "whole round (forwards and adjoints, with the small kernels)",
                         "achieved": value, "peak": peak, "unit": UNIT, "frac": value / peak, "traffic": None},
            "gpu_launches": None if round_kernels is None else round_kernels * args.steps,
            "clocks": clocks.summary()}
    print(json.dumps(line))
    return 0


def bench_batch(args):
    """c5: 64 uneven holograms (512^2 / 1024^2 / 1920x1152, N log-uniform in
    [10, 5000], D in {5, 10, 11}), 50 WGS iterations each: the batched form
    (one launch per phase for all holograms, one CUDA graph) against looping
    the per-hologram path. One step = the whole batch solved once."""
    import torch

    from paper_2505_08777_gb300 import Batch, Hologram
    from workloads import config_c5, config_c5_small

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    small = args.config == "c5s"
    ps = config_c5_small(1, count=64) if small else config_c5(1, count=64)
    iters = ps[0].iters
    amps = [torch.from_numpy(p.amp).to(dev) for p in ps]
    coeffs = [torch.from_numpy(p.coeff).to(dev) for p in ps]
    b = Batch([(a, c, p.noll) for a, c, p in zip(amps, coeffs, ps)], solo_terms=args.batch_solo_terms)
    hs = [Hologram(a, c, noll=p.noll) for a, c, p in zip(amps, coeffs, ps)]
    ph0 = [torch.from_numpy(p.phase0).to(dev) for p in ps]
    T = [torch.from_numpy(p.target).to(dev) for p in ps]
    ph = [x.clone() for x in ph0]
    w = [t.clone() for t in T]
    tuned = b.tune(ph0, os.path.join(_scratch_dir(), "ash_tune.txt"))
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def reset():
        for x, y in zip(ph, ph0):
            x.copy_(y)
        for x, y in zip(w, T):
            x.copy_(y)

    def batched():
        b.wgs(ph, w, T, iters)

    def looped():
        for h, x, y, t in zip(hs, ph, w, T):
            h.wgs(x, y, t, iters)

    def timed(fn, reps):
        for _ in range(max(args.warmup, 3)):
            reset()
            fn()
        tot = 0.0
        for _ in range(reps):
            reset()
            flush.zero_()
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            e.record(stream)
            e.synchronize()
            tot += a.elapsed_time(e)
        return tot / reps

    with ClockSampler(0) as clocks:
        ms_b = timed(batched, args.steps)
        ms_l = timed(looped, args.steps)
    met = b.wgs([x.clone() for x in ph0], [t.clone() for t in T], T, iters).cpu().numpy()
    terms = sum((2 * iters + 1) * p.N * p.M for p in ps)
    info = b.info()
    wl = ("64 holograms, sizes {256^2, 384^2, 512^2}, N log-uniform [10, 300]" if small else
          "64 holograms, sizes {512^2, 1024^2, 1920x1152}, N log-uniform [10, 5000]")
    line = {"metric": "spot-kernel Gterm/s fwd+adj, batched uneven WGS (64 holograms x 50 iterations), "
                      f"workload {args.config}",
            "value": terms / (ms_b * 1e-3) / 1e9, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_b, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl + ", D in {5, 10, 11}, 50 WGS iterations each; one step = the whole batch",
                       "terms_per_step": terms, "l2": "flushed between steps (256 MiB write)",
                       "tuned_grid": tuned, "resident_ctas": info["resident_ctas"],
                       "standalone_members": info["standalone"]},
            "looped_gterm_s": terms / (ms_l * 1e-3) / 1e9, "looped_ms_per_step": ms_l,
            "batched_speedup_vs_loop": ms_l / ms_b,
            "gpu_launches": b.launches(iters) * args.steps,
            "looped_gpu_launches": sum(int(h._lib.ash_wgs_launches(h.handle, iters)) for h in hs) * args.steps,
            "uniformity_min": float(met[:, 0].min()), "uniformity_median": float(np.median(met[:, 0])),
            "frac_of_peak": terms / (ms_b * 1e-3) / 1e9 / _peak_gterm(torch, dev),
            "clocks": clocks.summary()}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = _sampled_baseline("wgs", ps[:8], "one WGS iteration of the first 8 holograms")
    print(json.dumps(line))
    return 0


def bench_peaks(args):
    """The per-SM unit rates behind the roofline, measured by the library's
    probe (`--steps` repetitions, median), with the SM clocks sampled while
    it runs; prints one JSON line."""
    import torch

    from paper_2505_08777_gb300 import _lib
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    L = _lib.load()
    sp = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(max(args.warmup, 1)):
        probe_rates(L, sp)
    runs = []
    with ClockSampler(0) as clocks:
        for _ in range(max(args.steps, 1)):
            runs.append(probe_rates(L, sp))
    keys = ["mufu_sincos_per_clk_sm", "ffma_lanes_per_clk_sm", "ffma2_lanes_per_clk_sm", "ex2_per_clk_sm",
            "probe_sm_mhz"]
    med = {k: float(np.median([r[k] for r in runs])) for k in keys}
    mhz, mhz_src = max_sm_mhz()
    sms = runs[0]["sms"]
    fp32 = max(med["ffma_lanes_per_clk_sm"], med["ffma2_lanes_per_clk_sm"])
    line = {"metric": "per-SM pipe rates (results per clock per SM)", "value": med["mufu_sincos_per_clk_sm"],
            "unit": "sin/cos per clk per SM", "n_gpus": 1, "steps": len(runs), "warmup": args.warmup,
            "rates": med | {"sms": sms}, "runs": runs,
            "r_terms_gterm_s": {str(D): sms * planned_terms_per_clk_per_sm(D, med["mufu_sincos_per_clk_sm"], fp32)
                                * mhz * 1e6 / 1e9 for D in (5, 10, 11)},
            "two_pipe_gterm_s": sms * alu_terms_per_clk_per_sm(med["mufu_sincos_per_clk_sm"], fp32) * mhz * 1e6 / 1e9,
            "clock_for_peaks_mhz": mhz, "clock_source": mhz_src, "clocks": clocks.summary(),
            "higher_is_better": True, "data": "synthetic", "dtype": "f32"}
    print(json.dumps(line))
    return 0


def bench_shard(args):
    """c2 as one hologram sharded over the ranks by whole 32-row tile bands
    (Methods, per-pixel independence): each rank holds a band handle; per
    WGS iteration its forward partial fields, one all-reduce of N complex64
    (NCCL), the replicated spot update and the band's adjoint. One step =
    one full solve (50 iterations + the final forward) of the one hologram;
    value = its terms / the max over ranks of the step time."""
    import torch

    from paper_2505_08777_gb300.shard import band_holograms, row_block, sharded_wgs
    from workloads import config_c2

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    p = config_c2(1)
    iters = p.iters
    r0, r1 = row_block(p.ny, rank, world)
    amp = torch.from_numpy(p.amp).to(dev)
    coeff = torch.from_numpy(p.coeff).to(dev)
    bands = band_holograms(amp, coeff, p.noll, p.ny, [(r0, r1)])
    sa = torch.tensor([bands[0].band_info()[2]], dtype=torch.float64, device=dev)
    allreduce = None
    if world > 1:
        torch.distributed.all_reduce(sa)
        allreduce = lambda E: torch.distributed.all_reduce(E)   # noqa: E731
    sum_a2 = float(sa.item())
    ph0 = torch.from_numpy(p.phase0[r0:r1]).to(dev)
    T = torch.from_numpy(p.target).to(dev)
    ph = ph0.clone()
    w = T.clone()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        ph.copy_(ph0)
        w.copy_(T)
        return sharded_wgs(bands, [ph], w, T, iters, allreduce=allreduce, sum_a2=sum_a2)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    total = 0.0
    with ClockSampler(local) as clocks:
        for _ in range(args.steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            _, met = step()
            b.record(stream)
            b.synchronize()
            total += a.elapsed_time(b)
    if world > 1:
        torch.distributed.barrier()
    t = torch.tensor([total], device=dev)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    total_max = float(t.item())
    terms = (2 * iters + 1) * p.N * p.M
    value = terms * args.steps / (total_max * 1e-3) / 1e9
    line = {"metric": METRIC + " (one hologram sharded by pixel rows)", "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_max / args.steps,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": _workload_config(p, iters) | {"parallelism": f"pixel rows over {world} rank(s), "
                                                                   "one all-reduce of N complex64 per forward",
                                                    "band_rows": [r0, r1]},
            "wgs_iter_per_s": iters * args.steps / (total_max * 1e-3),
            "final_uniformity": float(met[0].item()), "clocks": clocks.summary()}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
