"""Time the other workloads of the pressure solver (measurement helper).

    python -m paper_1309_7128_gb300.workloads jet      [--steps N]
    python -m paper_1309_7128_gb300.workloads rollout  [--steps N]
    python -m paper_1309_7128_gb300.workloads batched  [--n N]

Each prints one JSON line with device times taken by CUDA events on the
caller's stream (warm-up excluded):

* jet -- the planar jet: 8192 x 4096 staggered grid, h = 1, inlet of 64
  cells (top-hat 1 with 1% seeded noise, coflow 0.05), convective outflow with
  pressure Dirichlet 0, free-slip sides, Re = 5000 on the inlet width; mixed
  ISM with 32h coarsening, warm start, solves to 1e-8.  Three developing
  steps, then `steps` timed steps; also one FP64 step for comparison.
* rollout -- the differentiable rollout: 512 x 512 cavity, Re = 400, FP32
  steps with the mixed ISM (16h); the forward step, and the checkpointed
  gradient of the final enstrophy over 200 steps (checkpoints every 20).
* batched -- the ensemble: `n` Neumann cavities of uneven sizes (multiples of
  32 in [128, 1024], aspect 1..4, smooth divergence right-hand sides),
  coarsening picked by ism_setup(coarsen = 0), sweeps per cycle and coarse
  engine by ism_autotune_batched; one batched solve to 1e-8 against the same
  problems solved one by one with the FP64 ISM.
"""
import argparse
import json
import time

import numpy as np
import torch

from . import build, ism

JET = (ism.ISM_VEL_INFLOW, ism.ISM_VEL_OUTFLOW, ism.ISM_VEL_FREESLIP, ism.ISM_VEL_FREESLIP)
CAVITY = (ism.ISM_VEL_NOSLIP,) * 4


def _timed(fn):
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    out = fn()
    e1.record()
    e1.synchronize()
    return e0.elapsed_time(e1), out


def _check(s, where):
    if s != ism.ISM_OK:
        raise ism.IsmError(s, where)


def run_jet(steps):
    from synth.inputs import jet_inflow
    nx, ny, m = 8192, 4096, 32
    h, nu = 1.0, 64.0 / 5000
    dt = 0.9 * min(0.4 * h / 1.0, 0.25 * h * h / nu, 2 * nu / 1.0)
    prof = torch.tensor(jet_inflow(ny, width=64, seed=0), dtype=torch.float32, device="cuda")
    out = {"workload": "planar jet 8192x4096 MAC, h=1, inlet 64 cells, Re=5000, ISM 32h, rel. residual 1e-8"}
    for name, prec in (("mixed", ism.ISM_MIXED), ("fp64", ism.ISM_FP64)):
        # pressure faces: Neumann except the Dirichlet-0 outflow (east)
        s, ctx = ism.ism_setup(nx, ny, h, (0, 1, 0, 0), m, prec)
        _check(s, "ism_setup")
        _check(ism.ism_set_flow(ctx, JET, (0, 0, 0, 0), prof, 1.0), "ism_set_flow")
        _check(ism.ism_proj_tol(ctx, 1e-8, 1_000_000, True), "ism_proj_tol")
        u = torch.zeros((ny, nx + 1), dtype=torch.float32, device="cuda")
        u[:, 0] = prof
        v = torch.zeros((ny + 1, nx), dtype=torch.float32, device="cuda")
        p = torch.zeros((ny, nx), dtype=torch.float32, device="cuda")
        for _ in range(3):
            _check(ism.proj_step(ctx, u, v, p, dt, nu), "proj_step")
        ms, cyc = [], []
        for _ in range(steps if prec == ism.ISM_MIXED else 1):
            t, s = _timed(lambda: ism.proj_step(ctx, u, v, p, dt, nu))
            _check(s, "proj_step")
            ms.append(t)
            cyc.append(ism.ism_last_counts(ctx)[1])
        o = ism.ism_get_options(ctx)
        out[name] = {"ms_per_step": round(float(np.mean(ms)), 2), "cycles_per_step": cyc, "nu": o.nu,
                     "sweeps_per_pass": o.sweeps_per_pass}
        del ctx
    return out


def run_rollout(steps):
    from synth.inputs import random_field, smooth_velocity
    n, m, nu = 512, 16, 1.0 / 400
    h = 1.0 / n
    dt = 0.9 * min(0.4 * h, 0.25 * h * h / nu, 2 * nu)
    us, vs = smooth_velocity(n, n, 16)
    u = torch.tensor(0.25 * us + 0.02 * random_field(n + 1, n, 17), dtype=torch.float32, device="cuda")
    v = torch.tensor(0.25 * vs + 0.02 * random_field(n, n + 1, 18), dtype=torch.float32, device="cuda")
    p = torch.zeros((n, n), dtype=torch.float32, device="cuda")
    s, ctx = ism.ism_setup(n, n, h, (0, 0, 0, 0), m, ism.ISM_MIXED)
    _check(s, "ism_setup")
    _check(ism.ism_set_flow(ctx, CAVITY, (0, 0, 0, 1.0), None, 1.0), "ism_set_flow")
    _check(ism.ism_proj_tol(ctx, 1e-8, 1_000_000, False), "ism_proj_tol")
    uu, vv, pp = u.clone(), v.clone(), p.clone()
    for _ in range(3):
        _check(ism.proj_step(ctx, uu, vv, pp, dt, nu), "proj_step")
    ms = []
    for _ in range(steps):
        t, s = _timed(lambda: ism.proj_step(ctx, uu, vv, pp, dt, nu))
        _check(s, "proj_step")
        ms.append(t)
    g = [torch.empty_like(t) for t in (u, v, p)]
    t_grad, (s, loss) = _timed(lambda: ism.proj_rollout_grad(ctx, u, v, p, dt, nu, 200, 20, *g))
    _check(s, "proj_rollout_grad")
    return {"workload": "cavity 512x512 MAC, Re=400, ISM 16h mixed, 200 steps, checkpoints every 20",
            "forward_ms_per_step": round(float(np.mean(ms)), 3),
            "rollout_forward_and_gradient_s": round(t_grad / 1000.0, 3), "final_enstrophy": loss}


def run_batched(n):
    from synth.inputs import batch_shapes, smooth_rhs
    shapes = batch_shapes(n, seed=0)
    t0 = time.perf_counter()
    ctxs, rhs, ps = [], [], []
    for k, (nx, ny) in enumerate(shapes):
        s, c = ism.ism_setup(nx, ny, 1.0 / nx, (0, 0, 0, 0), 0, ism.ISM_MIXED)
        _check(s, "ism_setup")
        ctxs.append(c)
        rhs.append(torch.tensor(smooth_rhs(nx, ny, 1000 + k), dtype=torch.float64, device="cuda"))
        ps.append(torch.zeros((ny, nx), dtype=torch.float64, device="cuda"))
    t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    s, _ = ism.ism_autotune_batched(ctxs, rhs, ps, 1e-8)
    _check(s, "ism_autotune_batched")
    o = ism.ism_get_options(ctxs[0])
    t_tune = time.perf_counter() - t0
    for q in ps:
        q.zero_()
    ism.ism_solve_batched(ctxs, rhs, ps, 1e-8, 200000)            # warm-up (graph build)
    for q in ps:
        q.zero_()
    t_b, (s, cyc, rr) = _timed(lambda: ism.ism_solve_batched(ctxs, rhs, ps, 1e-8, 200000))
    _check(s, "ism_solve_batched")
    # the same problems with the FP64 ISM, one by one
    ctx64 = []
    for (nx, ny), c in zip(shapes, ctxs):
        s, c64 = ism.ism_setup(nx, ny, 1.0 / nx, (0, 0, 0, 0), ism.ism_coarsening(c), ism.ISM_FP64)
        _check(s, "ism_setup")
        ctx64.append(c64)
    for c64, b, q in zip(ctx64, rhs, ps):                         # warm-up
        q.zero_()
        ism.ism_solve(c64, b, q, 1e-8, 200000)

    def all64():
        for c64, b, q in zip(ctx64, rhs, ps):
            q.zero_()
            st, _, _ = ism.ism_solve(c64, b, q, 1e-8, 200000)
            _check(st, "ism_solve")
    t_64, _ = _timed(all64)
    ms = [ism.ism_coarsening(c) for c in ctxs]
    return {"workload": f"{n} Neumann cavities, sides multiples of 32 in [128, 1024], aspect 1..4, rel. residual 1e-8",
            "setup_s": round(t_setup, 2), "autotune_s": round(t_tune, 2),
            "coarsening": {"16": ms.count(16), "32": ms.count(32)},
            "nu": o.nu, "coarse_tc": o.coarse_tc,
            "batched_solves_per_s": round(n / (t_b / 1000.0), 1),
            "fp64_one_by_one_solves_per_s": round(n / (t_64 / 1000.0), 1),
            "max_relres": max(rr), "max_cycles": max(cyc)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("which", choices=["jet", "rollout", "batched"])
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--n", type=int, default=256)
    a = ap.parse_args()
    build.build()
    if a.which == "jet":
        out = run_jet(a.steps)
    elif a.which == "rollout":
        out = run_rollout(a.steps)
    else:
        out = run_batched(a.n)
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
