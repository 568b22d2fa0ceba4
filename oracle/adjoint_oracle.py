"""TEST INFRASTRUCTURE ONLY: FP64 oracle of the projection step's gradient.

The projection step (Sec. 2.2-2.3, Eq. 3-4) restated with plain PyTorch CPU
tensor operations in float64, with the pressure equation solved exactly by a
dense LU factorisation (a library primitive).  Its gradient is the plain
definition of the adjoint: the vector-Jacobian product of the step, taken by
torch.autograd through these operations (the solve's derivative is the
library's transposed LU solve).  No blocking, fusion or reordering: one
array expression per formula, in the order the step states them.

Readings (restated where used):
* predictor: forward Euler, advective form, second-order central
  differences, transverse velocity = mean of the four nearest faces,
  tangential ghosts mirrored about the wall speed (no-slip), negated (inlet)
  or copied (free slip, outflow); convective outflow face with a Dirichlet-0
  pressure ghost;
* pressure: A_f dp = h div(v*) / dt, the mean of the right-hand side removed
  and dp of zero mean when every face is Neumann (dp = A_f^+ b);
* loss of the rollout: enstrophy 1/2 sum w^2 h^2 over the interior grid
  nodes, w = dv/dx - du/dy.

Only ``tests/`` use this module; it shares no code with the CUDA library.
"""
from __future__ import annotations

import numpy as np
import torch

from .ism_oracle import VEL_FREESLIP, VEL_INFLOW, VEL_NOSLIP, VEL_OUTFLOW, apply_af, pressure_bc

__all__ = ["TorchProjection"]


def _ghost(kind, wall, inner):
    """Tangential velocity beyond a wall (see the module's readings)."""
    if kind == VEL_NOSLIP:
        return 2.0 * wall - inner
    if kind == VEL_INFLOW:
        return -inner
    return inner


class TorchProjection:
    """Projection step of an nx x ny MAC grid with cell size h (FP64)."""

    def __init__(self, nx, ny, h, vel_bc, wall_u=(0.0, 0.0, 0.0, 0.0), u_in=None, conv_u=1.0):
        self.nx, self.ny, self.h = nx, ny, float(h)
        self.vel_bc = tuple(int(k) for k in vel_bc)
        self.wall_u = tuple(float(w) for w in wall_u)
        self.u_in = torch.zeros(ny, dtype=torch.float64) if u_in is None else \
            torch.as_tensor(np.asarray(u_in, dtype=np.float64))
        self.conv_u = float(conv_u)
        self.bc = pressure_bc(self.vel_bc)
        self.singular = not any(self.bc)
        n = nx * ny
        # A_f assembled column by column from the oracle's operator
        eye = np.eye(n)
        A = np.empty((n, n))
        for k in range(n):
            A[:, k] = apply_af(eye[k].reshape(ny, nx), self.bc).ravel()
        if self.singular:
            A = A - np.full((n, n), 1.0 / n)       # invertible; same solution on mean-zero b
        self.A = A
        self.lu = torch.linalg.lu_factor(torch.from_numpy(A))

    # ------------------------------------------------------------ the step
    def predictor(self, u, v, p, dt, nu):
        nx, ny, ih = self.nx, self.ny, 1.0 / self.h
        W, E, S, N = self.vel_bc
        wW, wE, wS, wN = self.wall_u
        # x-faces 1..nx-1 (all rows)
        uc = u[:, 1:nx]
        uw, ue = u[:, 0:nx - 1], u[:, 2:nx + 1]
        usx = torch.cat([_ghost(S, wS, uc[0:1]), uc[:-1]], dim=0)
        unx = torch.cat([uc[1:], _ghost(N, wN, uc[-1:])], dim=0)
        vbar = 0.25 * (v[0:ny, 0:nx - 1] + v[0:ny, 1:nx] + v[1:ny + 1, 0:nx - 1] + v[1:ny + 1, 1:nx])
        adv = uc * (ue - uw) * (0.5 * ih) + vbar * (unx - usx) * (0.5 * ih)
        lap = (ue + uw + unx + usx - 4.0 * uc) * ih * ih
        gp = (p[:, 1:nx] - p[:, 0:nx - 1]) * ih
        us_in = uc + dt * (-adv + nu * lap - gp)
        west = self.u_in.reshape(ny, 1) if W == VEL_INFLOW else torch.zeros(ny, 1, dtype=u.dtype)
        if E == VEL_OUTFLOW:
            ub = u[:, nx:nx + 1]
            east = ub + dt * (-self.conv_u * (ub - u[:, nx - 1:nx]) * ih + 2.0 * p[:, nx - 1:nx] * ih)
        else:
            east = torch.zeros(ny, 1, dtype=u.dtype)
        us = torch.cat([west, us_in, east], dim=1)
        # y-faces 1..ny-1 (all columns); south and north faces are walls
        vc = v[1:ny]
        vsy, vny = v[0:ny - 1], v[2:ny + 1]
        vw = torch.cat([_ghost(W, wW, vc[:, 0:1]), vc[:, :-1]], dim=1)
        ve = torch.cat([vc[:, 1:], _ghost(E, wE, vc[:, -1:])], dim=1)
        ubar = 0.25 * (u[0:ny - 1, 0:nx] + u[0:ny - 1, 1:nx + 1] + u[1:ny, 0:nx] + u[1:ny, 1:nx + 1])
        adv = ubar * (ve - vw) * (0.5 * ih) + vc * (vny - vsy) * (0.5 * ih)
        lap = (ve + vw + vny + vsy - 4.0 * vc) * ih * ih
        gp = (p[1:ny] - p[0:ny - 1]) * ih
        vs_in = vc + dt * (-adv + nu * lap - gp)
        zero = torch.zeros(1, nx, dtype=v.dtype)
        vs = torch.cat([zero, vs_in, zero], dim=0)
        return us, vs

    def divergence(self, us, vs, dt):
        return self.h * ((us[:, 1:] - us[:, :-1]) + (vs[1:] - vs[:-1])) / dt

    def solve(self, b):
        """dp = A_f^+ b (mean of b removed first when every face is Neumann)."""
        if self.singular:
            b = b - b.mean()
        x = torch.linalg.lu_solve(*self.lu, b.reshape(-1, 1))
        return x.reshape(self.ny, self.nx)

    def correct(self, us, vs, p, dp, dt):
        nx, ny, s = self.nx, self.ny, dt / self.h
        inner = us[:, 1:nx] - s * (dp[:, 1:] - dp[:, :-1])
        east = us[:, nx:nx + 1]
        if self.vel_bc[1] == VEL_OUTFLOW:
            east = east + s * 2.0 * dp[:, nx - 1:nx]
        u1 = torch.cat([us[:, 0:1], inner, east], dim=1)
        v1 = torch.cat([vs[0:1], vs[1:ny] - s * (dp[1:] - dp[:-1]), vs[ny:ny + 1]], dim=0)
        return u1, v1, p + dp

    def step(self, u, v, p, dt, nu):
        us, vs = self.predictor(u, v, p, dt, nu)
        dp = self.solve(self.divergence(us, vs, dt))
        return self.correct(us, vs, p, dp, dt)

    # ------------------------------------------------------------ loss and gradients
    def enstrophy(self, u, v):
        nx, ny, ih = self.nx, self.ny, 1.0 / self.h
        w = (v[1:ny, 1:nx] - v[1:ny, 0:nx - 1]) * ih - (u[1:ny, 1:nx] - u[0:ny - 1, 1:nx]) * ih
        return 0.5 * (w * w).sum() * self.h * self.h

    @staticmethod
    def _t(a):
        return torch.as_tensor(np.asarray(a, dtype=np.float64)).clone()

    def step_np(self, u, v, p, dt, nu):
        with torch.no_grad():
            out = self.step(self._t(u), self._t(v), self._t(p), dt, nu)
        return tuple(o.numpy() for o in out)

    def step_vjp(self, u, v, p, dt, nu, gu, gv, gp):
        """Adjoints of (u, v, p) given those of the step's outputs."""
        x = [self._t(a).requires_grad_(True) for a in (u, v, p)]
        out = self.step(*x, dt, nu)
        grads = torch.autograd.grad(out, x, [self._t(g) for g in (gu, gv, gp)], allow_unused=True)
        return tuple(np.zeros(a.shape) if g is None else g.numpy() for g, a in zip(grads, x))

    def rollout_loss(self, u0, v0, p0, dt, nu, steps):
        with torch.no_grad():
            u, v, p = self._t(u0), self._t(v0), self._t(p0)
            for _ in range(steps):
                u, v, p = self.step(u, v, p, dt, nu)
            return float(self.enstrophy(u, v))

    def rollout_grad(self, u0, v0, p0, dt, nu, steps):
        """Final enstrophy and its gradient with respect to (u0, v0, p0)."""
        x = [self._t(a).requires_grad_(True) for a in (u0, v0, p0)]
        u, v, p = x
        for _ in range(steps):
            u, v, p = self.step(u, v, p, dt, nu)
        loss = self.enstrophy(u, v)
        grads = torch.autograd.grad(loss, x, allow_unused=True)
        return float(loss.detach()), tuple(np.zeros(a.shape) if g is None else g.numpy()
                                  for g, a in zip(grads, x))
