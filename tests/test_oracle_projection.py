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


# ------------------------------------------------------------------ periodic faces

PERIODIC = (O.VEL_PERIODIC,) * 4


def taylor_green(n, t=0.0, nu=0.0):
    """The Taylor-Green vortex on [0, 2 pi]^2 sampled on the MAC grid: an
    exact solution of the incompressible Navier-Stokes equations,
    u = sin x cos y F, v = -cos x sin y F, p = (cos 2x + cos 2y) F^2 / 4,
    F = exp(-2 nu t); the last face of each axis repeats the first."""
    h = 2 * np.pi / n
    F = np.exp(-2 * nu * t)
    xf, xc = np.arange(n + 1) * h, (np.arange(n) + 0.5) * h
    u = np.sin(xf)[None, :] * np.cos(xc)[:, None] * F
    v = -np.cos(xc)[None, :] * np.sin(xf)[:, None] * F
    p = (np.cos(2 * xc)[None, :] + np.cos(2 * xc)[:, None]) * F * F / 4
    u[:, n] = u[:, 0]
    v[n, :] = v[0, :]
    return u, v, p, h


def tg_error(n, nu=0.1, t_end=0.16):
    """Relative error of the Taylor-Green vortex at t_end, in 4 (n / 32)^2
    steps: dt exactly proportional to h^2, so the first-order time error
    falls like h^2 too."""
    u, v, p, h = taylor_green(n)
    steps = 4 * (n // 32) ** 2
    dt = t_end / steps
    s = O.OracleISM(n, n, 16, (2, 2, 2, 2))
    for _ in range(steps):
        O.proj_step(u, v, p, h, dt, nu, PERIODIC, s, tol=1e-12)
    ue, ve, _, _ = taylor_green(n, t_end, nu)
    return (np.linalg.norm(u - ue) + np.linalg.norm(v - ve)) / (np.linalg.norm(ue) + np.linalg.norm(ve))


def test_taylor_green_vortex_second_order():
    """Fully periodic box: the Taylor-Green vortex at a fixed time against the
    exact decaying solution.  The error falls as h^2 (3x to 5x when h
    halves); a wrong sign or a dropped term at a periodic face leaves an
    error that does not fall."""
    e32, e64 = tg_error(32), tg_error(64)
    assert e64 < 2e-3
    assert 3.0 <= e32 / e64 <= 5.0, (e32, e64)


def test_periodic_projection_is_divergence_free_and_keeps_the_duplicate_faces():
    nx, ny, h = 64, 48, 1.0 / 64
    u = 0.3 * random_field(nx + 1, ny, 40)
    v = 0.3 * random_field(nx, ny + 1, 41)
    u[:, nx] = u[:, 0]
    v[ny, :] = v[0, :]
    p = np.zeros((ny, nx))
    s = O.OracleISM(nx, ny, 16, (2, 2, 2, 2))
    us, vs = O.predictor(u, v, p, h, 1e-3, 0.01, PERIODIC)
    d0 = np.abs(O.divergence(us, vs, h, 1e-3)).max()
    O.proj_step(u, v, p, h, 1e-3, 0.01, PERIODIC, s, tol=1e-12)
    assert np.array_equal(u[:, nx], u[:, 0]) and np.array_equal(v[ny, :], v[0, :])
    assert np.abs(O.divergence(u, v, h, 1e-3)).max() <= 1e-9 * d0


def test_periodic_channel_step_commutes_with_a_shift_by_m():
    """Channel periodic in x with no-slip walls in y: shifting the state by m
    cells along x (the coarse cells shift with it) commutes with the step."""
    nx, ny, m, h = 96, 32, 16, 1.0 / 32
    vel = (O.VEL_PERIODIC, O.VEL_PERIODIC, O.VEL_NOSLIP, O.VEL_NOSLIP)
    u = 0.2 * random_field(nx + 1, ny, 42)
    v = 0.2 * random_field(nx, ny + 1, 43)
    u[:, nx] = u[:, 0]
    v[0, :] = 0.0
    v[ny, :] = 0.0
    p = random_field(nx, ny, 44)
    s = O.OracleISM(nx, ny, m, O.pressure_bc(vel))

    def step(u, v, p):
        u, v, p = u.copy(), v.copy(), p.copy()
        O.proj_step(u, v, p, h, 1e-3, 0.02, vel, s, wall_u=(0, 0, 0, 0.5), tol=1e-12)
        return u, v, p

    def shift(u, v, p):
        uu = np.empty_like(u)
        uu[:, :nx] = np.roll(u[:, :nx], m, axis=1)
        uu[:, nx] = uu[:, 0]
        return uu, np.roll(v, m, axis=1), np.roll(p, m, axis=1)

    a = shift(*step(u, v, p))
    b = step(*shift(u, v, p))
    for x, y in zip(a, b):
        np.testing.assert_allclose(x, y, rtol=0, atol=1e-10 * np.abs(y).max())
