"""Pins of the FP64 gradient oracle of the projection step.

The oracle's step (plain torch CPU ops, exact dense solve) is pinned to the C
oracle's step, which the projection pins fix to the physics; its gradient
(torch.autograd) is pinned by
* central differences of the C oracle's step: the step is a quadratic map of
  (u, v, p) (advection is quadratic, everything else affine), so a central
  difference equals the directional derivative exactly, whatever the step;
* closed forms of the pressure block: with an exact solve the step maps p to
  mean(p) (all faces Neumann) or to 0 (a Dirichlet-0 face), at any velocity;
* a closed form of the enstrophy (solid-body rotation);
* central differences of a short rollout (error O(eps^2)).
"""
import numpy as np
import pytest

import oracle as O
from oracle.adjoint_oracle import TorchProjection
from synth.inputs import jet_inflow, random_field, smooth_velocity

CAVITY = (O.VEL_NOSLIP,) * 4
JET = (O.VEL_INFLOW, O.VEL_OUTFLOW, O.VEL_FREESLIP, O.VEL_FREESLIP)
SLIP = (O.VEL_FREESLIP,) * 4

FLOWS = {
    "cavity": dict(vel_bc=CAVITY, wall_u=(0.0, 0.0, 0.0, 1.0)),
    "jet": dict(vel_bc=JET),
    "slip": dict(vel_bc=SLIP),
}


def state(nx, ny, seed, flow):
    u, v = smooth_velocity(nx, ny, seed)
    u = u * 2.0 + 0.05 * random_field(nx + 1, ny, seed + 1)
    v = v * 2.0 + 0.05 * random_field(nx, ny + 1, seed + 2)
    p = random_field(nx, ny, seed + 3)
    extra = {}
    if flow == "jet":
        prof = jet_inflow(ny, width=max(2, ny // 4))
        u[:, 0] = prof
        extra = dict(u_in=prof, conv_u=1.0)
    return u, v, p, extra


def make(nx, ny, flow, extra):
    h = 1.0 / nx
    kw = dict(FLOWS[flow])
    kw.update(extra)
    return TorchProjection(nx, ny, h, **kw), h, kw


def c_step(u, v, p, h, dt, nu, kw, m=4):
    u, v, p = u.copy(), v.copy(), p.copy()
    s = O.OracleISM(p.shape[1], p.shape[0], m, O.pressure_bc(kw["vel_bc"]))
    O.proj_step(u, v, p, h, dt, nu, kw["vel_bc"], s, wall_u=kw.get("wall_u", (0, 0, 0, 0)),
                u_in=kw.get("u_in"), conv_u=kw.get("conv_u", 1.0), tol=1e-14, max_cycles=5000)
    return u, v, p


@pytest.mark.parametrize("flow", ["cavity", "jet", "slip"])
def test_torch_step_matches_c_oracle(flow):
    nx, ny = 16, 12
    u, v, p, extra = state(nx, ny, 10, flow)
    T, h, kw = make(nx, ny, flow, extra)
    dt, nu = 0.2 * h, 0.01
    a = T.step_np(u, v, p, dt, nu)
    b = c_step(u, v, p, h, dt, nu, kw)
    for x, y in zip(a, b):
        assert np.abs(x - y).max() <= 1e-11 * max(1.0, np.abs(y).max())


def _dot(a, b):
    return sum(float(np.sum(x * y)) for x, y in zip(a, b))


@pytest.mark.parametrize("flow", ["cavity", "jet", "slip"])
def test_vjp_equals_exact_central_difference_of_c_step(flow):
    nx, ny = 16, 12
    u, v, p, extra = state(nx, ny, 20, flow)
    T, h, kw = make(nx, ny, flow, extra)
    dt, nu = 0.2 * h, 0.01
    rng = np.random.Generator(np.random.PCG64(5))
    bar = [rng.standard_normal(a.shape) for a in (u, v, p)]
    g = T.step_vjp(u, v, p, dt, nu, *bar)
    for k in range(3):
        d = [rng.standard_normal(a.shape) for a in (u, v, p)]
        if flow == "jet":
            d[0][:, 0] = 0.0           # the inlet face is prescribed by u_in
        eps = 0.5                      # exact for a quadratic map: any eps
        fp = c_step(*[a + eps * b for a, b in zip((u, v, p), d)], h, dt, nu, kw)
        fm = c_step(*[a - eps * b for a, b in zip((u, v, p), d)], h, dt, nu, kw)
        fd = _dot(bar, [(x - y) / (2 * eps) for x, y in zip(fp, fm)])
        ad = _dot(g, d)
        assert abs(fd - ad) <= 1e-8 * (abs(ad) + 1.0), (k, fd, ad)


@pytest.mark.parametrize("flow", ["cavity", "jet"])
def test_pressure_adjoint_closed_form(flow):
    """Exact solve: u', v' do not depend on p; p' = mean(p) (Neumann) or 0
    (Dirichlet-0 outflow).  So p-bar = mean(p'-bar) or 0 for any state."""
    nx, ny = 12, 12
    u, v, p, extra = state(nx, ny, 30, flow)
    T, h, kw = make(nx, ny, flow, extra)
    rng = np.random.Generator(np.random.PCG64(6))
    bar = [rng.standard_normal(a.shape) for a in (u, v, p)]
    gp = T.step_vjp(u, v, p, 0.2 * h, 0.01, *bar)[2]
    want = np.full_like(p, bar[2].mean()) if flow == "cavity" else np.zeros_like(p)
    assert np.abs(gp - want).max() <= 1e-10


def test_enstrophy_solid_body_rotation():
    """u = -W (y - 1/2), v = W (x - 1/2): vorticity 2W at every node."""
    nx, ny, W = 10, 8, 1.7
    h = 1.0 / nx
    T = TorchProjection(nx, ny, h, SLIP)
    yc = (np.arange(ny) + 0.5) * h
    xc = (np.arange(nx) + 0.5) * h
    u = np.tile(-W * (yc - 0.5)[:, None], (1, nx + 1))
    v = np.tile(W * (xc - 0.5)[None, :], (ny + 1, 1))
    e = float(T.enstrophy(T._t(u), T._t(v)))
    assert e == pytest.approx(0.5 * (2 * W) ** 2 * h * h * (nx - 1) * (ny - 1), rel=1e-13)


def test_rollout_gradient_central_difference():
    nx, ny = 12, 12
    u, v, p, extra = state(nx, ny, 40, "cavity")
    T, h, kw = make(nx, ny, "cavity", extra)
    dt, nu, steps = 0.3 * h, 0.02, 6
    loss, g = T.rollout_grad(u, v, p, dt, nu, steps)
    assert loss == pytest.approx(T.rollout_loss(u, v, p, dt, nu, steps), rel=1e-14)
    rng = np.random.Generator(np.random.PCG64(7))
    for k in range(3):
        d = [rng.standard_normal(a.shape) for a in (u, v, p)]
        eps = 1e-4
        lp = T.rollout_loss(*[a + eps * b for a, b in zip((u, v, p), d)], dt, nu, steps)
        lm = T.rollout_loss(*[a - eps * b for a, b in zip((u, v, p), d)], dt, nu, steps)
        fd = (lp - lm) / (2 * eps)
        assert fd == pytest.approx(_dot(g, d), rel=1e-6, abs=1e-10), k
