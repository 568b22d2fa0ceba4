"""Benchmark I of the paper with its accommodative strategy: iteration and
synchronisation counts against the coarse criterion and the coarsening
(Sec. 4.3.1, the shape of Tables 3 and Fig. 4).

    python -m paper_1309_7128_gb300.tolc_study [--n 500] [--steps 1000]
        [--m 8 16 32] [--tolc 1e-6 1e-5 2e-5 3e-5 4e-5 5e-5 1e-4]

Workload: a cavity whose walls move against each other (the north wall at
-v0 along x, the west wall at +v0 along y), kinematic viscosity 0.1, v0 = 0.1,
h = 1, dt = 1, from rest, n x n cells; every projection step solves its
pressure increment (FP64) with the accommodative strategy (option cycle = 1):
coarse Gauss-Seidel on the nine-point ISM equations until max |r_c| <= tol_c,
bilinear correction, red-black sweeps until max |r| <= 1e-6, warm-started
from the previous increment.

Counters per step (ism_last_counts): I_c coarse iterations, I_f fine sweeps.
Reported as averages over the steps, in the paper's measures (readings of
its text, checked against its Table 3, e.g. 4h, tol_c 1e-6: 2.5 + 72.8/16 =
7.0): NCC_f = 2 I_f (a red-black sweep synchronises twice), NCC_c = I_c (one
synchronisation per coarse iteration), NCC_t = NCC_f + NCC_c, and
N_Lap = I_f + I_c / m^2 (Laplacians per fine cell and step).  Prints one JSON
line per (m, tol_c) and a markdown table at the end.
"""
import argparse
import json

import torch

from . import build, ism

SHEAR = (ism.ISM_VEL_NOSLIP,) * 4


def run(n, m, tol_c, steps, nu=0.1, v0=0.1, dt=1.0, tol_f=1e-6):
    """Counts of `steps` Benchmark I steps on an n x n grid with coarsening m."""
    s, ctx = ism.ism_setup(n, n, 1.0, (0, 0, 0, 0), m, ism.ISM_FP64)
    ism.check(s, "ism_setup")
    o = ism.ism_get_options(ctx)
    o.cycle = 1
    o.accom_tol_c = tol_c
    ism.check(ism.ism_set_options(ctx, o), "ism_set_options")
    ism.check(ism.ism_set_flow(ctx, SHEAR, (v0, 0.0, 0.0, -v0), None, 1.0), "ism_set_flow")
    ism.check(ism.ism_proj_tol(ctx, tol_f, 10_000_000, True), "ism_proj_tol")
    u = torch.zeros((n, n + 1), dtype=torch.float32, device="cuda")
    v = torch.zeros((n + 1, n), dtype=torch.float32, device="cuda")
    p = torch.zeros((n, n), dtype=torch.float32, device="cuda")
    ic, jf = [], []
    for _ in range(steps):
        ism.check(ism.proj_step(ctx, u, v, p, dt, nu), "proj_step")
        o_, c_, _ = ism.ism_last_counts(ctx)
        ic.append(o_)
        jf.append(c_)
    i_c = sum(ic) / steps
    i_f = sum(jf) / steps
    return {"n": n, "m": m, "tol_c": tol_c, "steps": steps, "I_c": i_c, "I_f": i_f,
            "NCC_f": 2 * i_f, "NCC_c": i_c, "NCC_t": 2 * i_f + i_c, "N_Lap": i_f + i_c / (m * m),
            "first_steps": {"I_c": ic[:10], "I_f": jf[:10]}}


def table(rows, ms, tols):
    out = []
    for key in ("NCC_f", "NCC_c", "NCC_t", "N_Lap"):
        out.append(f"| {key} | " + " | ".join(f"{m}h" for m in ms) + " |")
        out.append("|---|" + "---|" * len(ms))
        for t in tols:
            vals = [next(r[key] for r in rows if r["m"] == m and r["tol_c"] == t) for m in ms]
            out.append(f"| {t:g} | " + " | ".join(f"{x:.1f}" for x in vals) + " |")
        out.append("")
    return "\n".join(out)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=500)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--m", type=int, nargs="+", default=[8, 16, 32])
    ap.add_argument("--tolc", type=float, nargs="+", default=[1e-6, 1e-5, 2e-5, 3e-5, 4e-5, 5e-5, 1e-4])
    a = ap.parse_args()
    build.build()
    rows = []
    for m in a.m:
        for t in a.tolc:
            r = run(a.n, m, t, a.steps)
            rows.append(r)
            print(json.dumps(r), flush=True)
    print(table(rows, a.m, a.tolc), flush=True)


if __name__ == "__main__":
    main()
