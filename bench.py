#!/usr/bin/env python
"""Benchmark: pressure solves per second of the ISM projection step.

Workload (one "step"): one Goda projection time step of the 2048 x 2048
lid-driven cavity on the staggered grid (Re = 1000, lid speed 1, unit box,
explicit central advection/diffusion, dt at 0.9 of the stability limit),
whose pressure increment is solved by two-level ISM with 32h coarsening
(64 x 64 coarse grid): single-precision cycles inside FP64 iterative
refinement to relative residual 1e-8.  The FP64 ISM runs the same steps for
the mixed-vs-FP64 comparison.  Synthetic state: the cavity starts from rest.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  With N > 1 (torchrun, one process per GPU)
every rank runs its own independent cavity (replicas; the solve does not
shard), timings are reduced with a max over ranks and ``value`` counts the
solves of all ranks.  ``--impl reference`` times the CPU oracle instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "pressure solves/s to rel. residual 1e-8: mixed vs FP64 ISM; % HBM peak"
UNIT = "solves/s"
N_GRID = 2048
COARSEN = 32
RE_NU = 1e-3          # Re = 1000 with lid speed 1 and unit box
LID = 1.0
TOL = 1e-8
L2_FLUSH_BYTES = 512 << 20
PROFILE_MD = os.path.join(ROOT, "profiles", "k_sweep32_cavity2048.md")
SWEEP_SRC = os.path.join(ROOT, "paper_1309_7128_gb300", "csrc", "ism_sweep32.cuh")
GOLDEN = os.path.join(ROOT, "tests", "golden", "cavity2048_step1.json")


def cavity_dt(n=N_GRID, nu=RE_NU, lid=LID):
    h = 1.0 / n
    return h, 0.9 * min(0.4 * h / lid, 0.25 * h * h / nu, 2.0 * nu / lid ** 2)


def workload_config(tuned=None):
    cfg = {"workload": "lid-driven cavity 2048x2048 MAC, Re=1000, ISM 32h (64x64 coarse), "
                       "FP32 cycles in FP64 refinement to rel. residual 1e-8",
           "nx": N_GRID, "ny": N_GRID, "coarsen": COARSEN, "tol": TOL,
           "l2": "flushed between timed steps (512 MB write)"}
    if tuned:
        cfg.update(tuned)
    return cfg


# ------------------------------------------------------------------ distributed

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_max(value: float, world: int, device=None) -> float:
    """Max of a float over all ranks (identity when world == 1)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def whole_job_rate(world: int, steps: int, max_total_ms: float) -> float:
    """Solves/s of the whole job: every rank solves `steps` problems; the job
    takes as long as its slowest rank (max over ranks of the summed step times)."""
    return world * steps / (max_total_ms / 1000.0)


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu_id}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, flag in zip(self.NAMES, parts[3:7]):
                if flag.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------------ roofline bookkeeping

def large_grid_passes(peak, peak_kind, dev):
    """Pass rates on a grid whose single-precision fields (128 MB) exceed L2:
    the streaming one-sweep pass, the streaming residual + restriction pass and
    the fused 8-sweep tiled pass, each timed alone with CUDA events on the
    library's stream."""
    import torch

    from paper_1309_7128_gb300 import ism
    nx, ny, m = 8192, 4096, 32
    n = nx * ny
    s, c = ism.ism_setup(nx, ny, 1.0 / nx, (0, 0, 0, 0), m, ism.ISM_MIXED)
    ism.check(s, "ism_setup (large grid)")
    p = torch.zeros((ny, nx), dtype=torch.float32, device=dev)
    b = torch.randn((ny, nx), dtype=torch.float32, device=dev) * 1e-6
    rc = torch.zeros((ny // m, nx // m), dtype=torch.float32, device=dev)
    o = ism.ism_get_options(c)
    o.stream = 1
    ism.check(ism.ism_set_options(c, o), "ism_set_options")
    s, us_s = ism.ism_time_pass(c, p, b, 1, 20)
    ism.check(s, "ism_time_pass")
    s, us_r = ism.ism_time_restrict(c, p, b, rc, 20)
    ism.check(s, "ism_time_restrict")
    o.stream = 0
    ism.check(ism.ism_set_options(c, o), "ism_set_options")
    s, us_t = ism.ism_time_pass(c, p, b, 8, 10)
    ism.check(s, "ism_time_pass")
    del c

    def entry(kernel, us, bytes_cell, sweeps=None):
        a = bytes_cell * n / (us * 1e-6) / 1e9
        d = {"kernel": kernel, "bound": "hbm", "us_per_launch": round(us, 2),
             "algorithmic_bytes_per_launch": bytes_cell * n, "achieved": round(a, 1), "peak": peak,
             "unit": "GB/s", "frac": round(a / peak, 4), "peak_source": peak_kind}
        if sweeps:
            d["us_per_sweep"] = round(us / sweeps, 2)
        return d

    return {"grid": f"{nx}x{ny}, 32h (fields of 128 MB, larger than L2)",
            "stream_sweep": entry("k_stream32<1>: one red-black sweep, streaming", us_s, 12.0, 1),
            "restriction": entry("k_restrict_stream<float>: residual + block sums + norm partials", us_r, 8.0),
            "tiled_8_sweeps": entry("k_sweep32: fused 8-sweep tiled pass (the solver's default)", us_t, 12.0, 8)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, burst copy)"
    return 6800.0, "fallback 6.8 TB/s (no MEASURED_PEAKS.json)"


def profiled_traffic():
    """DRAM bytes per launch of the fused pass from the committed ncu summary,
    or None when the kernel source changed since the capture."""
    if not os.path.exists(PROFILE_MD):
        return None
    sha = hashlib.sha256(open(SWEEP_SRC, "rb").read()).hexdigest()
    vals = {}
    for line in open(PROFILE_MD):
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("source_sha256") != sha:
        return None
    try:
        return float(vals["dram_bytes_per_pass"])
    except (KeyError, ValueError):
        return None


# ------------------------------------------------------------------ CPU oracle legs

def cpu_sample(cycles: int):
    """Bounded CPU sample of one benchmark step with the oracle (FP64, one
    thread): predictor + divergence of the first step from rest, `cycles`
    ISM cycles of its pressure solve, and the correction.  Returns seconds
    for the parts; the caller scales the cycles to a whole solve."""
    import numpy as np

    import oracle as O
    n = N_GRID
    h, dt = cavity_dt()
    cav = (O.VEL_NOSLIP,) * 4
    s = O.OracleISM(n, n, COARSEN, nu=8)              # setup (LU of the coarse operator): untimed
    u = np.zeros((n, n + 1)); v = np.zeros((n + 1, n)); p = np.zeros((n, n))
    t0 = time.perf_counter()
    us, vs = O.predictor(u, v, p, h, dt, RE_NU, cav, wall_u=(0, 0, 0, LID))
    b = s.prepare_rhs(O.divergence(us, vs, h, dt))
    t1 = time.perf_counter()
    dp = np.zeros_like(b)
    for _ in range(cycles):
        s.cycle(dp, b)
    t2 = time.perf_counter()
    O.correct(us, vs, p, dp, h, dt, cav)
    t3 = time.perf_counter()
    return {"setup_free_step_s": (t1 - t0) + (t3 - t2), "cycle_s": (t2 - t1) / cycles, "cycles": cycles}


def run_cpu_sample_subprocess(cycles: int):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    out = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-sample", str(cycles)],
                         env=env, capture_output=True, text=True, timeout=1800)
    if out.returncode != 0:
        raise RuntimeError("CPU oracle sample failed:\n" + out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def golden_cycles():
    with open(GOLDEN) as f:
        return int(json.load(f)["cycles"])


def cpu_rate(sample):
    """Solves/s of the oracle scaled from a sample: one step = predictor,
    divergence, correction + (oracle cycle count of this solve) cycles."""
    cyc = golden_cycles()
    return 1.0 / (sample["setup_free_step_s"] + sample["cycle_s"] * cyc), cyc


# ------------------------------------------------------------------ our implementation

def run_ours(args):
    import torch

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")

    import __graft_entry__
    __graft_entry__.build()
    from paper_1309_7128_gb300 import ism

    n = N_GRID
    h, dt = cavity_dt()
    cav = (ism.ISM_VEL_NOSLIP,) * 4

    def make_ctx(prec):
        s, ctx = ism.ism_setup(n, n, h, (0, 0, 0, 0), COARSEN, prec)
        ism.check(s, "ism_setup")
        o = ism.ism_get_options(ctx)
        o.use_graphs = args.use_graphs
        ism.check(ism.ism_set_options(ctx, o), "ism_set_options")
        ism.check(ism.ism_set_flow(ctx, cav, (0, 0, 0, LID), None, 1.0), "ism_set_flow")
        ism.check(ism.ism_proj_tol(ctx, TOL, 1_000_000, False), "ism_proj_tol")
        return ctx

    # autotune sweeps per cycle / per fused pass on a smooth right-hand side (untimed)
    from synth.inputs import smooth_rhs
    rhs_tune = torch.tensor(smooth_rhs(n, n, 0), dtype=torch.float64, device=dev)

    def tuned_ctx(prec):
        c = make_ctx(prec)
        if args.no_autotune:
            o = ism.ism_get_options(c)
            o.nu = args.nu if prec == ism.ISM_MIXED else args.nu_fp64
            o.sweeps_per_pass = args.sweeps_per_pass if prec == ism.ISM_MIXED else 4
            ism.check(ism.ism_set_options(c, o), "ism_set_options")
        else:
            s, o = ism.ism_autotune(c, rhs_tune, TOL, 1_000_000)
            ism.check(s, "ism_autotune")
        o = ism.ism_get_options(c)
        return c, {"nu_sweeps": o.nu, "sweeps_per_pass": o.sweeps_per_pass, "stream": o.stream,
                   "inner_tol": o.inner_tol, "autotuned": not args.no_autotune}

    ctx, opt_mixed = tuned_ctx(ism.ISM_MIXED)
    u = torch.zeros((n, n + 1), dtype=torch.float32, device=dev)
    v = torch.zeros((n + 1, n), dtype=torch.float32, device=dev)
    p = torch.zeros((n, n), dtype=torch.float32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def step(c, uu, vv, pp):
        s = ism.proj_step(c, uu, vv, pp, dt, RE_NU)
        if s != ism.ISM_OK:
            raise ism.IsmError(s, "proj_step")

    for _ in range(args.warmup):
        step(ctx, u, v, p)
    torch.cuda.synchronize()

    # ---- timed region: K projection steps, L2 flushed before each
    gpu_id = getattr(torch.cuda.get_device_properties(dev), "uuid", None)
    sampler = ClockSampler(f"GPU-{gpu_id}" if gpu_id else str(local))
    launches0 = ism.ism_last_counts(ctx)[2]          # cumulative launch counter of the context
    per_step, cycles, outers, relres = [], [], [], []
    sampler.start()
    barrier(world)
    torch.cuda.synchronize()
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        step(ctx, u, v, p)
        e1.record()
        e1.synchronize()
        per_step.append(e0.elapsed_time(e1))
        o, c, _ = ism.ism_last_counts(ctx)
        cycles.append(c)
        outers.append(o)
        relres.append(ism.ism_last_history(ctx, 64)[-1])
    torch.cuda.synchronize()
    barrier(world)
    clocks = sampler.stop()
    launches = ism.ism_last_counts(ctx)[2] - launches0
    total_ms = reduce_max(sum(per_step), world, dev)
    value = whole_job_rate(world, args.steps, total_ms)

    # ---- FP64 ISM on the same steps (state copied from the mixed run)
    ctx64, opt_fp64 = tuned_ctx(ism.ISM_FP64)
    u64, v64, p64 = u.clone(), v.clone(), p.clone()
    fp64_ms, fp64_cycles = [], []
    for _ in range(args.fp64_steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        step(ctx64, u64, v64, p64)
        e1.record()
        e1.synchronize()
        fp64_ms.append(e0.elapsed_time(e1))
        fp64_cycles.append(ism.ism_last_counts(ctx64)[1])
    fp64_total = reduce_max(sum(fp64_ms), world, dev)
    fp64_value = whole_job_rate(world, args.fp64_steps, fp64_total)
    del ctx64

    # ---- dominant kernel: the fused 4-sweep single-precision pass, timed alone
    b32 = torch.randn((n, n), dtype=torch.float32, device=dev) * 1e-6
    e32 = torch.zeros((n, n), dtype=torch.float32, device=dev)
    kpass = opt_mixed["sweeps_per_pass"]
    s, us_pass = ism.ism_time_pass(ctx, e32, b32, kpass, 50)
    ism.check(s, "ism_time_pass")
    bytes_pass = 12.0 * n * n                    # read p and b, write p (4 B each)
    achieved = bytes_pass / (us_pass * 1e-6) / 1e9
    peak, peak_kind = measured_peaks()
    traffic = profiled_traffic()
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic,
                "kernel": f"k_sweep32: fused {kpass}-sweep red-black pass (interior + edge launches)",
                "us_per_launch": round(us_pass, 2), "algorithmic_bytes_per_launch": bytes_pass,
                "peak_source": peak_kind,
                "cell_sweeps_per_s": round(kpass * n * n / (us_pass * 1e-6), 1),
                "note": "2048^2 single-precision fields are L2-resident between passes; the pass "
                        "moves 12 B per cell whatever the number of fused sweeps, so the fraction is "
                        "of an L2-resident, latency-bound kernel (cell_sweeps_per_s is its rate)"}

    # ---- grids larger than L2: the streaming passes at 8192 x 4096 (128 MB fields)
    large = None
    if rank == 0 and not args.no_large:
        large = large_grid_passes(peak, peak_kind, dev)

    # ---- end to end through the public API with host buffers
    hu = torch.zeros((n, n + 1), dtype=torch.float32).pin_memory()
    hv = torch.zeros((n + 1, n), dtype=torch.float32).pin_memory()
    hp = torch.zeros((n, n), dtype=torch.float32).pin_memory()
    hu.copy_(u.cpu()); hv.copy_(v.cpu()); hp.copy_(p.cpu())
    hout = torch.empty((n, n), dtype=torch.float32).pin_memory()
    du, dv, dpp = torch.empty_like(u), torch.empty_like(v), torch.empty_like(p)
    e2e_ms = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        du.copy_(hu, non_blocking=True)
        dv.copy_(hv, non_blocking=True)
        dpp.copy_(hp, non_blocking=True)
        step(ctx, du, dv, dpp)
        hout.copy_(dpp, non_blocking=True)
        e1.record()
        e1.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
    e2e_total = reduce_max(sum(e2e_ms), world, dev)
    e2e = {"value": round(whole_job_rate(world, args.steps, e2e_total), 3), "unit": UNIT,
           "h2d_bytes_per_step": int(hu.nbytes + hv.nbytes + hp.nbytes),
           "d2h_bytes_per_step": int(hout.nbytes)}

    out = {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
           "data": "synthetic (cavity from rest)",
           "config": workload_config({"mixed_options": opt_mixed, "fp64_options": opt_fp64, "use_graphs": args.use_graphs}),
           "fp64": {"value": round(fp64_value, 3), "unit": UNIT, "steps": args.fp64_steps,
                    "ms_per_step": round(fp64_total / args.fp64_steps, 3),
                    "cycles_per_solve": fp64_cycles},
           "mixed_over_fp64": round(value / fp64_value, 2),
           "solve": {"cycles_per_solve": cycles, "refinements_per_solve": outers,
                     "final_relres_max": max(relres),
                     "mcell_cycles_per_s": round(world * N_GRID * N_GRID * sum(cycles) / (total_ms / 1000.0) / 1e6, 1)},
           "roofline": roofline, "clocks": clocks, "e2e": e2e, "gpu_launches": int(launches)}
    if large is not None:
        out["large_grid_passes"] = large

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        smp = run_cpu_sample_subprocess(args.cpu_cycles)
        rate, cyc = cpu_rate(smp)
        out["cpu_baseline"] = {"value": round(rate, 6), "unit": UNIT, "cores": 1, "kind": "oracle",
                               "sample": f"first cavity step from rest: predictor, divergence, {smp['cycles']} "
                                         f"FP64 oracle ISM cycles ({smp['cycle_s']:.3f} s/cycle), correction; "
                                         f"scaled to the oracle's {cyc} cycles per solve (tests/golden)"}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ------------------------------------------------------------------ reference arm

def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    per_step = []
    smp = None
    for k in range(args.warmup + args.steps):
        smp = run_cpu_sample_subprocess(args.ref_cycles)
        rate, cyc = cpu_rate(smp)
        if k >= args.warmup:
            per_step.append(1.0 / rate)
    total = sum(per_step)
    value = args.steps / total
    out = {"metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(1000 * total / args.steps, 1), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (cavity from rest)",
           "config": workload_config(), "impl": "reference",
           "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": f"per step: predictor, divergence, {args.ref_cycles} FP64 oracle ISM "
                                      f"cycles, correction, scaled to {golden_cycles()} cycles per solve"},
           "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--cpu-cycles", type=int, default=12)
    ap.add_argument("--ref-cycles", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-large", action="store_true", help="skip the 8192x4096 pass measurements")
    ap.add_argument("--no-autotune", action="store_true",
                    help="use --nu / --sweeps-per-pass / --nu-fp64 instead of ism_autotune")
    ap.add_argument("--nu", type=int, default=32)
    ap.add_argument("--sweeps-per-pass", type=int, default=8)
    ap.add_argument("--nu-fp64", type=int, default=32)
    ap.add_argument("--use-graphs", type=int, default=2, choices=[0, 1, 2],
                    help="2: one graph per solve with device-side loops (default); 1: graphs of "
                         "16-cycle chunks (the form whose kernels ncu lists one by one); 0: plain launches")
    ap.add_argument("--cpu-sample", type=int, default=0, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.cpu_sample:
        print(json.dumps(cpu_sample(args.cpu_sample)))
        return
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
