"""Time the fused single-precision smoothing pass on an n x n grid.

    python -m paper_1309_7128_gb300.timepass N K [REPS]

Creates a mixed-precision context (32h, Neumann walls), fills b with N(0,1)
values and prints the mean device time of one K-sweep pass measured by
ism_time_pass (CUDA events on the library's work stream).  Used to profile
the kernel that bench.py reports in its roofline.
"""
import sys

import torch

from . import build, ism


def main():
    n = int(sys.argv[1]) if len(sys.argv) > 1 else 2048
    k = int(sys.argv[2]) if len(sys.argv) > 2 else 8
    reps = int(sys.argv[3]) if len(sys.argv) > 3 else 4
    build.build()
    s, ctx = ism.ism_setup(n, n, 1.0 / n, (0, 0, 0, 0), 32, ism.ISM_MIXED)
    ism.check(s, "ism_setup")
    g = torch.Generator(device="cuda").manual_seed(0)
    p = torch.zeros((n, n), dtype=torch.float32, device="cuda")
    b = torch.randn((n, n), dtype=torch.float32, device="cuda", generator=g)
    s, us = ism.ism_time_pass(ctx, p, b, k, reps)
    ism.check(s, "ism_time_pass")
    algo = 12.0 * n * n
    print(f"n={n} K={k} reps={reps}: {us:.2f} us/pass, {algo / (us * 1e-6) / 1e9:.1f} GB/s algorithmic")


if __name__ == "__main__":
    main()
