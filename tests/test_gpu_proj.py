"""Projection time step on the GPU (single-precision velocities, FP64
pressure increment) against the oracle's FP64 step from the same state."""
import numpy as np
import pytest

import oracle as O
from oracle import VEL_FREESLIP, VEL_INFLOW, VEL_NOSLIP, VEL_OUTFLOW
from synth.inputs import jet_inflow, smooth_velocity
from tests.gpu_util import dev32, ensure_built, host, ism, rel, setup, torch

pytestmark = pytest.mark.gpu

CAVITY = (VEL_NOSLIP,) * 4
JET = (VEL_INFLOW, VEL_OUTFLOW, VEL_FREESLIP, VEL_FREESLIP)


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def run_gpu(u, v, p, nx, ny, h, dt, nu, vel_bc, m, prec, wall_u=(0, 0, 0, 0), u_in=None, conv_u=1.0,
            steps=1, tol=1e-8):
    bc = O.pressure_bc(vel_bc)
    ctx = setup(nx, ny, m, bc, prec=prec, h=h)
    uin = dev32(u_in) if u_in is not None else None
    ism.check(ism.ism_set_flow(ctx, vel_bc, wall_u, uin, conv_u), "ism_set_flow")
    ism.check(ism.ism_proj_tol(ctx, tol, 100000, False))
    ud, vd, pd = dev32(u), dev32(v), dev32(p)
    for _ in range(steps):
        s = ism.proj_step(ctx, ud, vd, pd, dt, nu)
        assert s == ism.ISM_OK, ism.status_str(s)
    return host(ud), host(vd), host(pd), ctx


@pytest.mark.parametrize("prec", [0, 1])
def test_cavity_step_matches_oracle(prec):
    nx = ny = 128
    h = 1.0 / nx
    nu = 1e-3
    dt = 0.9 * min(0.25 * h * h / nu, 0.4 * h)
    u0, v0 = smooth_velocity(nx, ny, 4)
    u0, v0 = f32(u0), f32(v0)
    p0 = np.zeros((ny, nx))
    ug, vg, pg, ctx = run_gpu(u0, v0, p0, nx, ny, h, dt, nu, CAVITY, 16, prec, wall_u=(0, 0, 0, 1.0))
    u, v, p = u0.copy(), v0.copy(), p0.copy()
    s = O.OracleISM(nx, ny, 16)
    O.proj_step(u, v, p, h, dt, nu, CAVITY, s, wall_u=(0, 0, 0, 1.0), tol=1e-10)
    # single-precision velocities: one rounding per stored value
    assert np.abs(ug - u).max() <= 2e-6 * np.abs(u).max()
    assert np.abs(vg - v).max() <= 2e-6 * np.abs(v).max()
    assert rel(pg, p) <= 1e-5
    div = O.divergence(ug, vg, h, dt)
    div_star = O.divergence(*O.predictor(u0, v0, p0, h, dt, nu, CAVITY, wall_u=(0, 0, 0, 1.0)), h, dt)
    assert np.linalg.norm(div) <= 1e-5 * np.linalg.norm(div_star)


@pytest.mark.parametrize("prec", [0, 1])
def test_jet_step_matches_oracle(prec):
    nx, ny = 256, 128
    h, nu = 1.0, 64.0 / 5000
    prof = f32(jet_inflow(ny, width=16, seed=3))
    dt = 0.9 * min(0.4 * h / 1.0, 0.25 * h * h / nu, 2 * nu / 1.0)
    u0 = np.zeros((ny, nx + 1)); v0 = np.zeros((ny + 1, nx)); p0 = np.zeros((ny, nx))
    ug, vg, pg, ctx = run_gpu(u0, v0, p0, nx, ny, h, dt, nu, JET, 32, prec, u_in=prof, conv_u=1.0, steps=3)
    u, v, p = u0.copy(), v0.copy(), p0.copy()
    s = O.OracleISM(nx, ny, 32, O.pressure_bc(JET))
    for _ in range(3):
        O.proj_step(u, v, p, h, dt, nu, JET, s, u_in=prof, conv_u=1.0, tol=1e-10)
    assert np.abs(ug - u).max() <= 1e-5 * np.abs(u).max()
    assert np.abs(vg - v).max() <= 1e-5 * max(np.abs(v).max(), 1e-3)
    assert rel(pg, p) <= 1e-4
    # mass: outflow equals inflow
    assert abs(ug[:, -1].sum() - prof.sum()) <= 1e-5 * prof.sum()


def test_proj_dp_matches_fp64_between_precisions():
    """Mixed and FP64 contexts give the same pressure increment to the
    solver tolerance from the same state (the per-step comparison of the
    cavity benchmark)."""
    nx = ny = 256
    h = 1.0 / nx
    nu = 1e-3
    dt = 0.9 * min(0.25 * h * h / nu, 0.4 * h)
    u0, v0 = smooth_velocity(nx, ny, 5)
    dps = []
    for prec in (0, 1):
        ctx = setup(nx, ny, 32, (0, 0, 0, 0), prec=prec, h=h)
        ism.check(ism.ism_set_flow(ctx, CAVITY, (0, 0, 0, 1.0), None, 1.0))
        ud, vd, pd = dev32(u0), dev32(v0), dev32(np.zeros((ny, nx)))
        assert ism.proj_step(ctx, ud, vd, pd, dt, nu) == ism.ISM_OK
        torch.cuda.synchronize()
        dps.append(host(pd))
    assert rel(dps[1], dps[0]) <= 1e-7


def test_set_flow_validation():
    ctx = setup(64, 64, 16, (0, 0, 0, 0))
    assert ism.ism_set_flow(ctx, (VEL_INFLOW, VEL_OUTFLOW, 0, 0), (0, 0, 0, 0), None, 1.0) == ism.ISM_ERR_ARG
    assert ism.ism_set_flow(ctx, (0, VEL_INFLOW, 0, 0), (0, 0, 0, 0), None, 1.0) == ism.ISM_ERR_ARG
    u = dev32(np.zeros((64, 65)))
    assert ism.proj_step(ctx, u, u, u, 0.1, 0.1) == ism.ISM_ERR_ARG     # flow not set
