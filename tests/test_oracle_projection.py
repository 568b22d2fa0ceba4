"""Pins of the oracle's projection time step (Sec. 2.2-2.3, Eq. 3-4) against
exact discrete steady states, exactness of central differences on linear
fields, the adjoint relation between gradient and divergence, and mass
conservation."""
import numpy as np
import pytest

import oracle as O
from oracle import VEL_FREESLIP, VEL_INFLOW, VEL_NOSLIP, VEL_OUTFLOW
from synth.inputs import jet_inflow, random_field, smooth_velocity

CAVITY = (VEL_NOSLIP,) * 4
JET = (VEL_INFLOW, VEL_OUTFLOW, VEL_FREESLIP, VEL_FREESLIP)


def test_couette_channel_is_a_discrete_steady_state():
    """Plane Couette flow u = U y / H between a resting south wall and a
    north wall moving at U, fed by the same profile at the inlet and leaving
    through a convective outlet, solves the discrete equations exactly."""
    nx, ny, h, U = 48, 32, 1.0 / 32, 0.7
    yc = (np.arange(ny) + 0.5) / ny
    prof = U * yc
    u = np.tile(prof[:, None], (1, nx + 1))
    v = np.zeros((ny + 1, nx))
    p = np.zeros((ny, nx))
    vel_bc = (VEL_INFLOW, VEL_OUTFLOW, VEL_NOSLIP, VEL_NOSLIP)
    s = O.OracleISM(nx, ny, 16, O.ism_oracle.pressure_bc(vel_bc))
    O.proj_step(u, v, p, h, 1e-3, 0.05, vel_bc, s, wall_u=(0, 0, 0, U), u_in=prof, conv_u=1.0)
    np.testing.assert_allclose(u, np.tile(prof[:, None], (1, nx + 1)), atol=1e-14)
    assert np.abs(v).max() <= 1e-14 and np.abs(p).max() <= 1e-12


def test_predictor_exact_on_stagnation_flow():
    """u = a x, v = -a y is divergence free and central differences are exact
    on it: advection gives (a^2 x, a^2 y), diffusion 0, so away from walls
    v* - v = -dt (a^2 x, a^2 y)."""
    nx, ny, h, a, dt = 16, 12, 0.1, 0.8, 0.01
    xf = np.arange(nx + 1) * h
    yf = np.arange(ny + 1) * h
    xc = (np.arange(nx) + 0.5) * h
    yc = (np.arange(ny) + 0.5) * h
    u = np.tile(a * xf[None, :], (ny, 1))
    v = np.tile(-a * yf[:, None], (1, nx))
    p = np.zeros((ny, nx))
    us, vs = O.predictor(u, v, p, h, dt, 0.3, CAVITY)
    np.testing.assert_allclose((us - u)[1:-1, 1:-1], (-dt * a * a * np.tile(xf[None, :], (ny, 1)))[1:-1, 1:-1],
                               rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose((vs - v)[1:-1, 1:-1], (-dt * a * a * np.tile(yf[:, None], (1, nx)))[1:-1, 1:-1],
                               rtol=1e-12, atol=1e-15)
    del xc, yc


def test_predictor_pressure_gradient_sign():
    """At rest, p = c x accelerates the fluid towards -x: u* = -dt c."""
    nx, ny, h, c, dt = 16, 8, 0.5, 2.0, 0.1
    xc = (np.arange(nx) + 0.5) * h
    p = np.tile(c * xc[None, :], (ny, 1))
    us, vs = O.predictor(np.zeros((ny, nx + 1)), np.zeros((ny + 1, nx)), p, h, dt, 0.0, CAVITY)
    np.testing.assert_allclose(us[:, 1:-1], -dt * c, rtol=1e-12)
    assert np.abs(us[:, [0, -1]]).max() == 0.0 and np.abs(vs).max() == 0.0


@pytest.mark.parametrize("vel_bc", [CAVITY, JET])
def test_gradient_is_minus_divergence_transpose(vel_bc):
    """<D w, q> = <w, -G q>_W over the faces whose velocity the projection
    corrects.  W weighs interior faces by 1 and the outflow face by 1/2: its
    gradient spans the half cell to the Dirichlet-0 face (ghost -p_c), which
    keeps D G = A_f."""
    nx, ny = 20, 12
    rng = np.random.Generator(np.random.PCG64(5))
    w_u = rng.standard_normal((ny, nx + 1))
    w_v = rng.standard_normal((ny + 1, nx))
    w_u[:, 0] = 0.0
    if vel_bc[1] != VEL_OUTFLOW:
        w_u[:, -1] = 0.0
    w_v[[0, -1], :] = 0.0
    q = random_field(nx, ny, 6)
    Dw = O.divergence(w_u, w_v, 1.0, 1.0)
    gu = np.zeros((ny, nx + 1))
    gv = np.zeros((ny + 1, nx))
    O.correct(gu, gv, np.zeros((ny, nx)), q, 1.0, 1.0, vel_bc)   # gu, gv = -G q
    wt = np.ones((ny, nx + 1))
    wt[:, -1] = 0.5
    assert abs(np.vdot(Dw, q) - (np.vdot(w_u * wt, gu) + np.vdot(w_v, gv))) <= 1e-11 * np.abs(Dw).sum()


def test_cavity_step_is_divergence_free():
    nx = ny = 64
    h = 1.0 / nx
    u, v = smooth_velocity(nx, ny, 3)
    p = np.zeros((ny, nx))
    s = O.OracleISM(nx, ny, 16)
    dt = 0.9 * min(0.25 * h * h / 1e-3, 0.4 * h)
    us, vs = O.predictor(u, v, p, h, dt, 1e-3, CAVITY, wall_u=(0, 0, 0, 1.0))
    div_star = np.linalg.norm(O.divergence(us, vs, h, dt))
    O.proj_step(u, v, p, h, dt, 1e-3, CAVITY, s, wall_u=(0, 0, 0, 1.0), tol=1e-10)
    assert np.linalg.norm(O.divergence(u, v, h, dt)) <= 1e-9 * div_star


def test_jet_step_conserves_mass_through_outflow():
    """With a Dirichlet-0 outflow face the projection routes the inflow
    through the outlet: total outflow equals total inflow after one step."""
    nx, ny = 96, 64
    h = 1.0
    u = np.zeros((ny, nx + 1))
    v = np.zeros((ny + 1, nx))
    p = np.zeros((ny, nx))
    prof = jet_inflow(ny, width=16, seed=2)
    s = O.OracleISM(nx, ny, 16, O.ism_oracle.pressure_bc(JET))
    O.proj_step(u, v, p, h, 0.02, 0.0128, JET, s, u_in=prof, conv_u=1.0, tol=1e-11)
    assert abs(u[:, -1].sum() - prof.sum()) <= 1e-8 * prof.sum()
    assert np.abs(O.divergence(u, v, h, 0.02)).max() <= 1e-8
