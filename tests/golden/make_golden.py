"""Write the oracle-generated reference values used by bench.py's CPU legs.

Calls only the CPU oracle (oracle/) and the seeded input generators.
Outputs:
* tests/golden/cavity2048_step1.json -- the FP64 oracle's cycle count and
  final relative residual for the pressure solve of the first projection
  step of the 2048 x 2048 lid-driven cavity (Re = 1000, lid speed 1, from
  rest, 32h coarsening, nu = 8 sweeps, tol 1e-8);
* tests/golden/jet8192_step1.json -- the same for the first projection step
  of the 8192 x 4096 planar jet from rest (h = 1, inlet of 64 cells, top-hat
  1 with 1% seeded noise, coflow 0.05, Re = 5000 on the inlet width,
  convective outflow with pressure Dirichlet 0, free-slip sides; 32h,
  nu = 8, tol 1e-8).
The counts scale the bounded CPU samples of the benchmark's reference arm to
whole solves.

    python tests/golden/make_golden.py [cavity|jet]
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
JET = (O.VEL_INFLOW, O.VEL_OUTFLOW, O.VEL_FREESLIP, O.VEL_FREESLIP)


def cavity_step1_problem(n=2048, nu=1e-3, lid=1.0):
    h = 1.0 / n
    dt = 0.9 * min(0.4 * h / lid, 0.25 * h * h / nu, 2 * nu / lid ** 2)
    u = np.zeros((n, n + 1))
    v = np.zeros((n + 1, n))
    p = np.zeros((n, n))
    us, vs = O.predictor(u, v, p, h, dt, nu, CAVITY, wall_u=(0, 0, 0, lid))
    return O.divergence(us, vs, h, dt), h, dt


def jet_dt(h=1.0, nu=64.0 / 5000, u=1.0):
    return 0.9 * min(0.4 * h / u, 0.25 * h * h / nu, 2 * nu / u ** 2)


def jet_step1_problem(nx=8192, ny=4096, width=64):
    """Predictor and divergence of the first jet step from rest: u = 0
    except the inflow face, which carries the seeded inlet profile (as
    float32, the precision in which the GPU step stores velocities)."""
    from synth.inputs import jet_inflow
    h, nu = 1.0, 64.0 / 5000
    dt = jet_dt(h, nu)
    prof = jet_inflow(ny, width=width, seed=0).astype(np.float32).astype(np.float64)
    u = np.zeros((ny, nx + 1))
    u[:, 0] = prof
    v = np.zeros((ny + 1, nx))
    p = np.zeros((ny, nx))
    us, vs = O.predictor(u, v, p, h, dt, nu, JET, u_in=prof, conv_u=1.0)
    return O.divergence(us, vs, h, dt), h, dt, nu, prof


def main_jet():
    nx, ny, m = 8192, 4096, 32
    O.set_threads(0)
    b, h, dt, nu, _ = jet_step1_problem(nx, ny)
    s = O.OracleISM(nx, ny, m, O.pressure_bc(JET), nu=8)
    t = time.perf_counter()
    p, cycles, hist = s.solve(b, tol=1e-8)
    el = time.perf_counter() - t
    out = {"problem": "8192x4096 planar jet, first projection step from rest, h=1, inlet 64 cells, Re=5000",
           "coarsen": m, "nu": 8, "tol": 1e-8, "cycles": cycles, "relres": hist[-1],
           "dt": dt, "h": h, "oracle_seconds": round(el, 1), "oracle_threads": O.get_threads()}
    with open(os.path.join(HERE, "jet8192_step1.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(out)


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
    which = sys.argv[1] if len(sys.argv) > 1 else "cavity"
    main_jet() if which == "jet" else main()
