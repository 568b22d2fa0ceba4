"""Time one pass kind on an nx x ny grid (measurement and profiling helper).

    python -m paper_1309_7128_gb300.timepass N K [REPS]
    python -m paper_1309_7128_gb300.timepass --nx NX --ny NY --pass {tiled,stream,restrict} [--k K]
                                             [--reps R] [--prec {mixed,fp64}]

Creates a context (32h, Neumann walls), fills b with N(0,1) values and prints
the mean device time of one pass measured with CUDA events on the library's
work stream: `tiled` is the fused K-sweep register-tiled pass (the one
bench.py reports in its roofline), `stream` the streaming K-sweep pass
(option stream = 1, K in 1, 2, 4), `restrict` the residual + restriction
pass, `coarse` the exact coarse solve (ism_coarse_solve, single precision;
--tc 1 on the tensor cores, 2 the tiled tensor-core chain on every size, 0 on
the CUDA cores; host-launched calls, then the same number in one graph).  The
first form times the tiled pass on an N x N grid.
"""
import argparse
import sys

import torch

from . import build, ism


def main():
    if len(sys.argv) > 1 and not sys.argv[1].startswith("-"):
        n = int(sys.argv[1])
        args = argparse.Namespace(nx=n, ny=n, kind="tiled", k=int(sys.argv[2]) if len(sys.argv) > 2 else 8,
                                  reps=int(sys.argv[3]) if len(sys.argv) > 3 else 4, prec="mixed")
    else:
        ap = argparse.ArgumentParser()
        ap.add_argument("--nx", type=int, default=2048)
        ap.add_argument("--ny", type=int, default=2048)
        ap.add_argument("--pass", dest="kind", choices=["tiled", "stream", "restrict", "coarse"], default="tiled")
        ap.add_argument("--tc", type=int, default=1)
        ap.add_argument("--k", type=int, default=8)
        ap.add_argument("--reps", type=int, default=4)
        ap.add_argument("--prec", choices=["mixed", "fp64"], default="mixed")
        args = ap.parse_args()
    build.build()
    prec = ism.ISM_MIXED if args.prec == "mixed" else ism.ISM_FP64
    dt = torch.float32 if prec == ism.ISM_MIXED else torch.float64
    nx, ny = args.nx, args.ny
    s, ctx = ism.ism_setup(nx, ny, 1.0 / nx, (0, 0, 0, 0), 32, prec)
    ism.check(s, "ism_setup")
    g = torch.Generator(device="cuda").manual_seed(0)
    p = torch.zeros((ny, nx), dtype=dt, device="cuda")
    b = torch.randn((ny, nx), dtype=dt, device="cuda", generator=g)
    if args.kind == "coarse":
        o = ism.ism_get_options(ctx)
        o.coarse_tc = args.tc
        ism.check(ism.ism_set_options(ctx, o), "ism_set_options")
        ncx, ncy = ism_ceil(nx, 32), ism_ceil(ny, 32)
        rc = torch.randn((ncy, ncx), dtype=dt, device="cuda", generator=g)
        rc -= rc.mean()
        ec = torch.zeros_like(rc)
        ism.check(ism.ism_coarse_solve(ctx, rc, ec), "ism_coarse_solve")        # warm-up
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(args.reps):
            ism.check(ism.ism_coarse_solve(ctx, rc, ec), "ism_coarse_solve")
        e1.record()
        e1.synchronize()
        us = 1000.0 * e0.elapsed_time(e1) / args.reps
        s, usg = ism.ism_time_coarse(ctx, rc, ec, args.reps)
        ism.check(s, "ism_time_coarse")
        print(f"coarse solve {ncx}x{ncy} tc={args.tc} reps={args.reps}: {us:.2f} us per call (host-launched), "
              f"{usg:.2f} us per solve (graph of {args.reps})")
        return
    if args.kind == "restrict":
        rc = torch.zeros((ism_ceil(ny, 32), ism_ceil(nx, 32)), dtype=dt, device="cuda")
        s, us = ism.ism_time_restrict(ctx, p, b, rc, args.reps)
        ism.check(s, "ism_time_restrict")
        algo = 2.0 * p.element_size() * nx * ny
    else:
        if args.kind == "stream":
            o = ism.ism_get_options(ctx)
            o.stream = 1
            ism.check(ism.ism_set_options(ctx, o), "ism_set_options")
        s, us = ism.ism_time_pass(ctx, p, b, args.k, args.reps)
        ism.check(s, "ism_time_pass")
        algo = 3.0 * p.element_size() * nx * ny
    print(f"{nx}x{ny} {args.kind} K={args.k} reps={args.reps}: {us:.2f} us/pass, "
          f"{algo / (us * 1e-6) / 1e9:.1f} GB/s algorithmic")


def ism_ceil(n, m):
    return -(-n // m)


if __name__ == "__main__":
    main()
