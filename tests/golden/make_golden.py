"""Write the oracle-generated reference values used by bench.py's CPU legs.

Calls only the CPU oracle (oracle/) and the seeded input generators.
Output: tests/golden/cavity2048_step1.json -- the FP64 oracle's cycle count
and final relative residual for the pressure solve of the first projection
step of the 2048 x 2048 lid-driven cavity (Re = 1000, lid speed 1, from
rest, 32h coarsening, nu = 8 sweeps, tol 1e-8).  The count scales the
bounded CPU samples of the benchmark to whole solves.

    python tests/golden/make_golden.py
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle as O  # noqa: E402

CAVITY = (O.VEL_NOSLIP,) * 4


def cavity_step1_problem(n=2048, nu=1e-3, lid=1.0):
    h = 1.0 / n
    dt = 0.9 * min(0.4 * h / lid, 0.25 * h * h / nu, 2 * nu / lid ** 2)
    u = np.zeros((n, n + 1))
    v = np.zeros((n + 1, n))
    p = np.zeros((n, n))
    us, vs = O.predictor(u, v, p, h, dt, nu, CAVITY, wall_u=(0, 0, 0, lid))
    return O.divergence(us, vs, h, dt), h, dt


def main():
    n, m = 2048, 32
    b, h, dt = cavity_step1_problem(n)
    s = O.OracleISM(n, n, m, nu=8)
    t = time.perf_counter()
    p, cycles, hist = s.solve(b, tol=1e-8)
    el = time.perf_counter() - t
    out = {"problem": "2048x2048 lid-driven cavity, first projection step from rest, Re=1000, lid 1",
           "coarsen": m, "nu": 8, "tol": 1e-8, "cycles": cycles, "relres": hist[-1],
           "dt": dt, "h": h, "oracle_seconds": round(el, 1)}
    with open(os.path.join(HERE, "cavity2048_step1.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(out)


if __name__ == "__main__":
    main()
