"""Hand-written adjoint of the projection step, the enstrophy loss and the
checkpointed rollout gradient on the GPU, against the FP64 gradient oracle
and central finite differences of the GPU's own forward rollout."""
import numpy as np
import pytest

import oracle as O
from oracle.adjoint_oracle import TorchProjection
from synth.inputs import jet_inflow, random_field, smooth_velocity
from tests.gpu_util import dev32, ensure_built, host, ism, setup, torch

pytestmark = pytest.mark.gpu

CAVITY = (O.VEL_NOSLIP,) * 4
JET = (O.VEL_INFLOW, O.VEL_OUTFLOW, O.VEL_FREESLIP, O.VEL_FREESLIP)
SLIP = (O.VEL_FREESLIP,) * 4
FLOWS = {"cavity": (CAVITY, (0.0, 0.0, 0.0, 1.0)), "jet": (JET, (0.0,) * 4), "slip": (SLIP, (0.0,) * 4)}


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def relv(a, b):
    num = sum(float(np.sum((x - y) ** 2)) for x, y in zip(a, b))
    den = sum(float(np.sum(y ** 2)) for y in b)
    return (num / den) ** 0.5


def flow_state(nx, ny, flow, seed, amp=1.0):
    u, v = smooth_velocity(nx, ny, seed)
    u = f32(amp * u + 0.02 * random_field(nx + 1, ny, seed + 1))
    v = f32(amp * v + 0.02 * random_field(nx, ny + 1, seed + 2))
    p = f32(random_field(nx, ny, seed + 3))
    prof = None
    if flow == "jet":
        prof = f32(jet_inflow(ny, width=max(2, ny // 4)))
        u[:, 0] = prof
    return u, v, p, prof


def gpu_ctx(nx, ny, m, flow, prec, prof=None, tol=1e-11, h=None):
    vel_bc, wall_u = FLOWS[flow]
    h = 1.0 / nx if h is None else h
    ctx = setup(nx, ny, m, O.pressure_bc(vel_bc), prec=prec, h=h)
    keep = dev32(prof) if prof is not None else None
    ism.check(ism.ism_set_flow(ctx, vel_bc, wall_u, keep, 1.0), "ism_set_flow")
    ism.check(ism.ism_proj_tol(ctx, tol, 100000, False))
    ctx._keep = keep
    return ctx


def oracle_for(nx, ny, flow, prof, h=None):
    vel_bc, wall_u = FLOWS[flow]
    return TorchProjection(nx, ny, 1.0 / nx if h is None else h, vel_bc, wall_u=wall_u, u_in=prof, conv_u=1.0)


@pytest.mark.parametrize("prec", [ism.ISM_FP64, ism.ISM_MIXED])
@pytest.mark.parametrize("flow", ["cavity", "jet", "slip"])
def test_step_adjoint_matches_oracle(flow, prec):
    nx, ny, m = 64, 48, 16
    u, v, p, prof = flow_state(nx, ny, flow, 11)
    ctx = gpu_ctx(nx, ny, m, flow, prec, prof)
    T = oracle_for(nx, ny, flow, prof)
    h = 1.0 / nx
    dt, nu = 0.2 * h, 0.01
    rng = np.random.Generator(np.random.PCG64(3))
    bar = [f32(rng.standard_normal(a.shape)) for a in (u, v, p)]
    want = T.step_vjp(u, v, p, dt, nu, *bar)
    gu, gv, gp = (dev32(b) for b in bar)
    s = ism.proj_step_adjoint(ctx, dev32(u), dev32(v), dt, nu, gu, gv, gp)
    assert s == ism.ISM_OK, ism.status_str(s)
    got = [host(g) for g in (gu, gv, gp)]
    assert relv(got, want) <= 1e-5
    # entrywise, against the largest adjoint (p-bar cancels to ~0 exactly
    # with a Dirichlet face and to its mean without one)
    scale = max(np.abs(w).max() for w in want)
    for g, w in zip(got, want):
        assert np.abs(g - w).max() <= 1e-5 * scale


def test_step_adjoint_leaves_forward_increment_and_rejects_bad_args():
    nx, ny, m = 64, 64, 16
    u, v, p, _ = flow_state(nx, ny, "cavity", 12)
    ctx = gpu_ctx(nx, ny, m, "cavity", ism.ISM_MIXED)
    ud, vd, pd = dev32(u), dev32(v), dev32(p)
    assert ism.proj_step(ctx, ud, vd, pd, 1e-3, 0.01) == ism.ISM_OK
    dp = _wrap(ism.ism_last_dp(ctx), nx * ny)
    torch.cuda.synchronize()
    dp_before = dp.clone()
    gu, gv, gp = (dev32(np.ones(a.shape)) for a in (u, v, p))
    assert ism.proj_step_adjoint(ctx, ud, vd, 1e-3, 0.01, gu, gv, gp) == ism.ISM_OK
    torch.cuda.synchronize()
    assert torch.equal(dp_before, dp)
    assert ism.proj_step_adjoint(ctx, ud, vd, -1.0, 0.01, gu, gv, gp) == ism.ISM_ERR_ARG
    assert ism.proj_step_adjoint(ctx, ud, vd, 1e-3, 0.01, None, gv, gp) == ism.ISM_ERR_ARG
    bare = setup(nx, ny, m, prec=ism.ISM_MIXED)
    assert ism.proj_step_adjoint(bare, ud, vd, 1e-3, 0.01, gu, gv, gp) == ism.ISM_ERR_ARG


def _wrap(addr, n):
    """A float64 CUDA tensor view of n doubles at a device address."""
    class _Arr:
        __cuda_array_interface__ = {"shape": (n,), "typestr": "<f8", "data": (addr, False), "version": 3}
    return torch.as_tensor(_Arr(), device="cuda:0")


def test_enstrophy_matches_oracle_and_closed_form():
    nx, ny = 96, 80
    u, v, _, _ = flow_state(nx, ny, "cavity", 13)
    ctx = gpu_ctx(nx, ny, 16, "cavity", ism.ISM_MIXED)
    T = oracle_for(nx, ny, "cavity", None)
    x = [T._t(u).requires_grad_(True), T._t(v).requires_grad_(True)]
    e = T.enstrophy(*x)
    ge = torch.autograd.grad(e, x)
    gu, gv = dev32(np.zeros(u.shape)), dev32(np.zeros(v.shape))
    s, val = ism.ism_enstrophy(ctx, dev32(u), dev32(v), gu, gv)
    assert s == ism.ISM_OK
    assert val == pytest.approx(float(e.detach()), rel=1e-12)
    assert relv([host(gu), host(gv)], [g.numpy() for g in ge]) <= 1e-6
    # solid-body rotation: vorticity 2W at every interior node
    W, h = 1.3, 1.0 / nx
    ur = np.tile(-W * ((np.arange(ny) + 0.5) * h - 0.5)[:, None], (1, nx + 1))
    vr = np.tile(W * ((np.arange(nx) + 0.5) * h - 0.5)[None, :], (ny + 1, 1))
    s, val = ism.ism_enstrophy(ctx, dev32(ur), dev32(vr))
    assert val == pytest.approx(0.5 * (2 * W) ** 2 * h * h * (nx - 1) * (ny - 1), rel=1e-6)


def cavity_dt(n, nu, lid=1.0):
    h = 1.0 / n
    return h, 0.9 * min(0.4 * h / lid, 0.25 * h * h / nu, 2 * nu / lid ** 2)


def test_rollout_checkpoint_schedules_are_bit_identical():
    nx = ny = 64
    u, v, p, _ = flow_state(nx, ny, "cavity", 14, amp=0.25)
    ctx = gpu_ctx(nx, ny, 16, "cavity", ism.ISM_MIXED, tol=1e-8)
    h, dt = cavity_dt(nx, 1 / 400)
    ud, vd, pd = dev32(u), dev32(v), dev32(p)
    res = []
    for every in (1, 7, 20, 45):
        g = [torch.empty_like(t) for t in (ud, vd, pd)]
        s, loss = ism.proj_rollout_grad(ctx, ud, vd, pd, dt, 1 / 400, 45, every, *g)
        assert s == ism.ISM_OK
        res.append((loss, [host(t) for t in g]))
    for loss, g in res[1:]:
        assert loss == res[0][0]
        for a, b in zip(g, res[0][1]):
            assert np.array_equal(a, b)
    # inputs untouched; forward-only call gives the same loss
    assert np.array_equal(host(ud), u) and np.array_equal(host(pd), p)
    s, loss = ism.proj_rollout_grad(ctx, ud, vd, pd, dt, 1 / 400, 45, 20)
    assert loss == res[0][0]


def test_rollout_gradient_matches_fp64_oracle_64():
    """64 x 64 copy of the differentiable cavity rollout (Re = 400, 200 steps,
    checkpoints every 20): gradient of the final enstrophy against the FP64
    oracle's autograd gradient."""
    nx = ny = 64
    nu = 1.0 / 400
    u, v, p, _ = flow_state(nx, ny, "cavity", 15, amp=0.25)
    h, dt = cavity_dt(nx, nu)
    ctx = gpu_ctx(nx, ny, 16, "cavity", ism.ISM_MIXED, tol=1e-10)
    ud, vd, pd = dev32(u), dev32(v), dev32(p)
    g = [torch.empty_like(t) for t in (ud, vd, pd)]
    s, loss = ism.proj_rollout_grad(ctx, ud, vd, pd, dt, nu, 200, 20, *g)
    assert s == ism.ISM_OK
    T = oracle_for(nx, ny, "cavity", None)
    loss_ref, g_ref = T.rollout_grad(u, v, p, dt, nu, 200)
    assert loss == pytest.approx(loss_ref, rel=1e-4)
    got = [host(t) for t in g]
    assert relv(got[:2], g_ref[:2]) <= 1e-3
    # the loss does not depend on p0 (exact projection): its gradient is ~0
    assert np.abs(got[2]).max() <= 1e-4 * max(np.abs(got[0]).max(), np.abs(got[1]).max())


def test_rollout_gradient_central_differences_512():
    """The differentiable rollout at full size: 512 x 512 cavity, Re = 400,
    200 FP32 steps, checkpoints every 20; directional derivatives of the final
    enstrophy along 16 seeded smooth directions against central differences
    (eps = 1e-3) of the GPU's own forward rollout."""
    n = 512
    nu = 1.0 / 400
    u, v, p, _ = flow_state(n, n, "cavity", 16, amp=0.25)
    h, dt = cavity_dt(n, nu)
    ctx = gpu_ctx(n, n, 16, "cavity", ism.ISM_MIXED, tol=1e-8)
    ud, vd, pd = dev32(u), dev32(v), dev32(p)
    g = [torch.empty_like(t) for t in (ud, vd, pd)]
    s, loss = ism.proj_rollout_grad(ctx, ud, vd, pd, dt, nu, 200, 20, *g)
    assert s == ism.ISM_OK
    gu, gv = host(g[0]), host(g[1])
    eps = 1e-3
    errs = []
    for k in range(16):
        du, dv = smooth_velocity(n, n, 1000 + k)
        scale = 1.0 / max(np.abs(du).max(), np.abs(dv).max())
        du, dv = f32(du * scale), f32(dv * scale)
        ad = float(np.sum(gu * du) + np.sum(gv * dv))
        s1, lp = ism.proj_rollout_grad(ctx, dev32(u + eps * du), dev32(v + eps * dv), pd, dt, nu, 200, 20)
        s2, lm = ism.proj_rollout_grad(ctx, dev32(u - eps * du), dev32(v - eps * dv), pd, dt, nu, 200, 20)
        assert s1 == ism.ISM_OK and s2 == ism.ISM_OK
        fd = (lp - lm) / (2 * eps)
        errs.append(abs(fd - ad) / max(abs(ad), 1e-3 * loss))
    print("central-difference relative errors:", ["%.2e" % e for e in errs])
    assert max(errs) <= 5e-4


def test_autograd_solve_matches_exact_adjoint():
    """torch.autograd through the ISM solve: the gradient of <w, S(b)> is
    S(w) = Pi A_f^+ Pi w, checked against the oracle's dense LU solve of
    A_f (independent of the GPU solver) for Neumann and Dirichlet faces."""
    from paper_1309_7128_gb300 import autograd as AG
    for flow in ("cavity", "jet"):
        nx, ny = 64, 48
        prof = None if flow == "cavity" else np.ones(ny)
        ctx = gpu_ctx(nx, ny, 16, flow, ism.ISM_MIXED, prof)
        T = oracle_for(nx, ny, flow, prof)
        rng = np.random.Generator(np.random.PCG64(21))
        b = rng.standard_normal((ny, nx))
        w = rng.standard_normal((ny, nx))
        bt = torch.tensor(b, device="cuda:0", requires_grad=True)
        p = AG.solve(ctx, bt, 1e-12)
        (g,) = torch.autograd.grad((p * torch.tensor(w, device="cuda:0")).sum(), bt)
        want = T.solve(torch.tensor(w)).numpy()
        # relative residual 1e-12 and cond(A_f) ~ 1e3 here: errors well below 1e-8
        assert float(np.linalg.norm(host(g) - want) / np.linalg.norm(want)) <= 1e-8
        pe = T.solve(torch.tensor(b)).numpy()
        assert float(np.linalg.norm(host(p) - pe) / np.linalg.norm(pe)) <= 1e-8


def test_autograd_proj_step_matches_oracle_vjp():
    """torch.autograd through ProjStep (forward proj_step, backward
    proj_step_adjoint) against the oracle's vector-Jacobian product."""
    from paper_1309_7128_gb300 import autograd as AG
    nx, ny = 64, 48
    u, v, p, _ = flow_state(nx, ny, "cavity", 22)
    ctx = gpu_ctx(nx, ny, 16, "cavity", ism.ISM_MIXED)
    T = oracle_for(nx, ny, "cavity", None)
    h = 1.0 / nx
    dt, nu = 0.2 * h, 0.01
    rng = np.random.Generator(np.random.PCG64(23))
    bar = [f32(rng.standard_normal(a.shape)) for a in (u, v, p)]
    x = [dev32(a).requires_grad_(True) for a in (u, v, p)]
    out = AG.proj_step(ctx, *x, dt, nu)
    loss = sum((o * dev32(w)).sum() for o, w in zip(out, bar))
    got = [host(g) for g in torch.autograd.grad(loss, x)]
    want = T.step_vjp(u, v, p, dt, nu, *bar)
    assert relv(got, want) <= 1e-5
    # the forward is proj_step's
    fw = T.step_np(u, v, p, dt, nu)
    assert np.abs(host(out[0]) - fw[0]).max() <= 1e-5 * np.abs(fw[0]).max()
