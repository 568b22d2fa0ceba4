"""Periodic pressure faces on the GPU against the CPU oracle: every kernel-level
step (FP64 sweeps, the fused single-precision pass whose boundary tiles load
wrapped rows and columns, residual and restriction, coarse solves on the CUDA
and tensor cores, bilinear correction across the periodic face), whole FP64
and mixed solves, the deep ACM V-cycle, the accommodative strategy and the
batched ensemble, on grids with ragged tiles and grids narrower than one
128 x 128 sweep region."""
import numpy as np
import pytest

import oracle as O
from synth.inputs import random_field, smooth_rhs
from tests.conftest import PERIODIC_BCS
from tests.gpu_util import dev32, dev64, ensure_built, host, ism, rel, setup

pytestmark = pytest.mark.gpu

SHAPES = [(256, 192, 32), (160, 128, 16), (64, 64, 16), (128, 64, 8), (320, 96, 16)]
KINDS = {"ism": ism.ISM_COARSE_ISM, "acm": ism.ISM_COARSE_ACM, "gmg": ism.ISM_COARSE_GMG}


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def rhs_for(nx, ny, bc, seed):
    return smooth_rhs(nx, ny, seed) + (0.0 if O.is_singular(bc) else 1e-6)


@pytest.mark.parametrize("nx,ny,m", SHAPES)
@pytest.mark.parametrize("bc", PERIODIC_BCS)
def test_smooth_fp64(nx, ny, m, bc):
    p, b = random_field(nx, ny, 1), random_field(nx, ny, 2)
    ctx = setup(nx, ny, m, bc)
    pd = dev64(p)
    ism.check(ism.ism_smooth(ctx, pd, dev64(b), 3))
    ref = p.copy()
    for _ in range(3):
        O.rbgs_sweep(ref, b, bc)
    np.testing.assert_allclose(host(pd), ref, rtol=0, atol=1e-13 * np.abs(ref).max())


@pytest.mark.parametrize("nx,ny,m", SHAPES)
@pytest.mark.parametrize("bc", PERIODIC_BCS)
@pytest.mark.parametrize("sweeps", [1, 4, 8])
def test_smooth_fused_fp32(nx, ny, m, bc, sweeps):
    p = random_field(nx, ny, 3).astype(np.float32)
    b = random_field(nx, ny, 4).astype(np.float32)
    ctx = setup(nx, ny, m, bc, prec=ism.ISM_MIXED)
    pd = dev32(p)
    ism.check(ism.ism_smooth(ctx, pd, dev32(b), sweeps))
    ref = np.ascontiguousarray(p.copy())
    bca = np.asarray(bc, dtype=np.int32)
    for _ in range(sweeps):
        O.lib().or_rbgs_sweep_f32(nx, ny, bca, ref, np.ascontiguousarray(b))
    np.testing.assert_allclose(host(pd), ref.astype(np.float64), rtol=0, atol=2e-6 * np.abs(ref).max())


@pytest.mark.parametrize("nx,ny,m", SHAPES)
@pytest.mark.parametrize("bc", PERIODIC_BCS)
def test_residual_restrict(nx, ny, m, bc):
    p, b = random_field(nx, ny, 5), random_field(nx, ny, 6)
    ctx = setup(nx, ny, m, bc)
    rc = dev64(np.zeros((ny // m, nx // m)))
    s, rnorm, _ = ism.ism_residual_restrict(ctx, dev64(p), dev64(b), rc)
    ism.check(s)
    r = O.residual(p, b, bc)
    ref = O.restrict(r, m)
    np.testing.assert_allclose(host(rc), ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    assert abs(rnorm - np.linalg.norm(r)) <= 1e-12 * np.linalg.norm(r)
    # the context-free form
    rc2, norms = dev64(np.zeros((ny // m, nx // m))), dev64(np.zeros(2))
    ism.check(ism.ism_residual_restrict_noalloc(nx, ny, m, bc, dev64(p), dev64(b), rc2, norms))
    np.testing.assert_allclose(host(rc2), ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    # single precision
    ctx32 = setup(nx, ny, m, bc, prec=ism.ISM_MIXED)
    rc32 = dev32(np.zeros((ny // m, nx // m)))
    p32, b32 = p.astype(np.float32), b.astype(np.float32)
    ism.check(ism.ism_residual_restrict(ctx32, dev32(p32), dev32(b32), rc32)[0])
    ref32 = O.restrict(O.residual(p32.astype(np.float64), b32.astype(np.float64), bc), m)
    np.testing.assert_allclose(host(rc32), ref32, rtol=0, atol=1e-5 * np.abs(ref32).max())


@pytest.mark.parametrize("nx,ny,m", SHAPES)
@pytest.mark.parametrize("bc", PERIODIC_BCS)
@pytest.mark.parametrize("kind", ["ism", "acm", "gmg"])
def test_coarse_solve(nx, ny, m, bc, kind):
    ncx, ncy = nx // m, ny // m
    rc = random_field(ncx, ncy, 7)
    sing = O.is_singular(bc)
    if sing:
        rc -= rc.mean()
    ref = O.OracleISM(nx, ny, m, bc, kind=kind).coarse_solve(rc)
    if sing:
        ref = ref - ref.mean()
    for prec, tcflag, tol in ((ism.ISM_FP64, 0, 1e-11), (ism.ISM_MIXED, 0, 2e-5), (ism.ISM_MIXED, 1, 1e-2)):
        ctx = setup(nx, ny, m, bc, prec=prec, kind=KINDS[kind], coarse_tc=tcflag)
        mk = dev64 if prec == ism.ISM_FP64 else dev32
        ec = mk(np.zeros_like(rc))
        ism.check(ism.ism_coarse_solve(ctx, mk(rc), ec))
        got = host(ec)
        if sing:
            got -= got.mean()
        np.testing.assert_allclose(got, ref, rtol=0, atol=tol * np.abs(ref).max())


@pytest.mark.parametrize("nx,ny,m", SHAPES)
@pytest.mark.parametrize("bc", PERIODIC_BCS)
@pytest.mark.parametrize("kind", ["ism", "acm"])
def test_prolong_add(nx, ny, m, bc, kind):
    q, p = random_field(nx // m, ny // m, 8), random_field(nx, ny, 9)
    ref = p.copy()
    if kind == "ism":
        O.prolong_add(ref, q, m, bc)
    else:
        O.prolong_const_add(ref, q, m)
    ctx = setup(nx, ny, m, bc, kind=KINDS[kind])
    pd = dev64(p)
    ism.check(ism.ism_prolong_add(ctx, dev64(q), pd))
    np.testing.assert_allclose(host(pd), ref, rtol=0, atol=1e-14 * np.abs(ref).max())


def gpu_solve(b, nx, ny, m, bc, prec, tol=1e-8, **opts):
    ctx = setup(nx, ny, m, bc, prec=prec, **opts)
    p = dev64(np.zeros((ny, nx)))
    s, cyc, relres = ism.ism_solve(ctx, dev64(b), p, tol, 100000)
    return s, host(p), cyc, relres, ctx


SOLVE_CASES = [(256, 256, 16, (2, 2, 2, 2)), (160, 128, 16, (2, 2, 1, 0)), (256, 192, 32, (0, 1, 2, 2)),
               (64, 64, 16, (2, 2, 0, 0)), (128, 64, 8, (1, 1, 2, 2))]


@pytest.mark.parametrize("nx,ny,m,bc", SOLVE_CASES)
@pytest.mark.parametrize("kind", ["ism", "gmg"])
def test_fp64_solve_matches_oracle(nx, ny, m, bc, kind):
    b = rhs_for(nx, ny, bc, 1)
    p_ref, c_ref, h_ref = O.OracleISM(nx, ny, m, bc, kind=kind).solve(b, tol=1e-8)
    s, p, c, r, _ = gpu_solve(b, nx, ny, m, bc, ism.ISM_FP64, kind=KINDS[kind])
    assert s == ism.ISM_OK and c == c_ref
    assert rel(p, p_ref) <= 1e-12
    assert abs(r - h_ref[-1]) <= 1e-13


@pytest.mark.parametrize("nx,ny,m,bc", SOLVE_CASES)
@pytest.mark.parametrize("coarse_tc", [0, 1, 2])
def test_mixed_solve_reaches_tolerance_and_matches_oracle(nx, ny, m, bc, coarse_tc):
    """The mixed path runs the fused pass with the correction and the
    residual folded in, so the wrapped loads of the boundary tiles carry the
    prolongation and the restriction as well."""
    b = rhs_for(nx, ny, bc, 2)
    ref = O.OracleISM(nx, ny, m, bc)
    p_ex, _, _ = ref.solve(b, tol=1e-11)
    s, p, c, r, _ = gpu_solve(b, nx, ny, m, bc, ism.ISM_MIXED, coarse_tc=coarse_tc)
    assert s == ism.ISM_OK and r <= 1e-8
    assert rel(p, p_ex) <= 1e-9
    bb = ref.prepare_rhs(b)
    assert np.linalg.norm(O.residual(p, bb, bc)) / np.linalg.norm(bb) <= 1.01e-8


@pytest.mark.parametrize("nx,ny,m,bc", [(256, 256, 16, (2, 2, 2, 2)), (256, 128, 8, (0, 1, 2, 2))])
def test_deep_acm_vcycle_matches_oracle(nx, ny, m, bc):
    b = rhs_for(nx, ny, bc, 6)
    p_ref, c_ref, _ = O.OracleACMV(nx, ny, m, bc, nu=8).solve(b, tol=1e-8)
    s, p, c, r, _ = gpu_solve(b, nx, ny, m, bc, ism.ISM_FP64, kind=ism.ISM_COARSE_ACMV, nu=8)
    assert s == ism.ISM_OK and c == c_ref
    assert rel(p, p_ref) <= 1e-12


@pytest.mark.parametrize("nx,ny,m,bc", [(256, 192, 16, (2, 2, 2, 2)), (128, 128, 8, (2, 2, 0, 1))])
def test_accommodative_strategy_matches_oracle(nx, ny, m, bc):
    b = rhs_for(nx, ny, bc, 12)
    tol_f, tol_c = 1e-7, 1e-6
    p_ref, nc_ref, nf_ref, _ = O.OracleAccommodative(nx, ny, m, bc).solve(b, tol_f=tol_f, tol_c=tol_c)
    ctx = setup(nx, ny, m, bc, prec=ism.ISM_FP64, cycle=1, accom_tol_c=tol_c)
    p = dev64(np.zeros((ny, nx)))
    s, nf, mx = ism.ism_solve(ctx, dev64(b), p, tol_f, 1000000)
    outer, cycles, _ = ism.ism_last_counts(ctx)
    assert s == ism.ISM_OK and mx <= tol_f
    assert outer == nc_ref and abs(cycles - nf_ref) <= 1
    assert rel(host(p), p_ref) <= 1e-10


def test_accommodative_rejects_odd_periodic_coarse_count():
    ctx = setup(80, 64, 16, (2, 2, 0, 0))                 # 5 coarse columns, periodic
    o = ism.ism_get_options(ctx)
    o.cycle = 1
    assert ism.ism_set_options(ctx, o) == ism.ISM_ERR_ARG


def test_batched_ensemble_with_periodic_members():
    shapes = [(256, 256), (160, 128), (128, 64), (320, 96), (256, 192)]
    ms = [16, 16, 8, 16, 32]
    bcs = [(2, 2, 2, 2), (2, 2, 1, 0), (1, 1, 2, 2), (0, 0, 0, 0), (0, 1, 2, 2)]
    ctxs, rhs, ps, bs = [], [], [], []
    for k, ((nx, ny), m, bc) in enumerate(zip(shapes, ms, bcs)):
        ctxs.append(setup(nx, ny, m, bc, prec=ism.ISM_MIXED))
        bs.append(rhs_for(nx, ny, bc, 40 + k))
        rhs.append(dev64(bs[-1]))
        ps.append(dev64(np.zeros((ny, nx))))
    s, cyc, rr = ism.ism_solve_batched(ctxs, rhs, ps, 1e-8, 100000)
    assert s == ism.ISM_OK, ism.status_str(s)
    for k, ((nx, ny), m, bc) in enumerate(zip(shapes, ms, bcs)):
        assert rr[k] <= 1e-8
        p_ex, _, _ = O.OracleISM(nx, ny, m, bc).solve(bs[k], tol=1e-11)
        assert rel(host(ps[k]), p_ex) <= 1e-9, k


def periodic_fft_solve(b):
    ny, nx = b.shape
    lam = (-4 * np.sin(np.pi * np.arange(nx) / nx) ** 2)[None, :] + \
          (-4 * np.sin(np.pi * np.arange(ny) / ny) ** 2)[:, None]
    lam[0, 0] = 1.0
    ph = np.fft.fft2(b) / lam
    ph[0, 0] = 0.0
    return np.fft.ifft2(ph).real


@pytest.mark.parametrize("prec", [ism.ISM_MIXED, ism.ISM_FP64])
def test_full_size_fully_periodic_solve_matches_fft(prec):
    """2048^2 with both axes periodic, 32h: the solve against the exact
    Fourier solution of the five-point equations."""
    nx = ny = 2048
    b = smooth_rhs(nx, ny, 21)
    s, p, c, r, _ = gpu_solve(b, nx, ny, 32, (2, 2, 2, 2), prec, tol=1e-10)
    assert s == ism.ISM_OK and r <= 1e-10
    ex = periodic_fft_solve(b - b.mean())
    assert rel(p, ex) <= 1e-7


def test_projection_step_pairs_periodic_velocity_and_pressure_faces():
    """Periodic velocity faces need periodic pressure faces and the other way
    round; the adjoint step rejects periodic faces."""
    ctx = setup(128, 128, 16, (2, 2, 0, 0))
    assert ism.ism_set_flow(ctx, (0, 0, 0, 0)) == ism.ISM_ERR_ARG
    assert ism.ism_set_flow(ctx, (4, 4, 0, 0)) == ism.ISM_OK
    ctx2 = setup(128, 128, 16, (0, 0, 0, 0))
    assert ism.ism_set_flow(ctx2, (4, 4, 0, 0)) == ism.ISM_ERR_ARG
    import torch
    u = torch.zeros((128, 129), dtype=torch.float32, device="cuda:0")
    v = torch.zeros((129, 128), dtype=torch.float32, device="cuda:0")
    g = [torch.zeros_like(t) for t in (u, v, torch.zeros((128, 128), dtype=torch.float32, device="cuda:0"))]
    assert ism.proj_step_adjoint(ctx, u, v, 0.01, 0.01, *g) == ism.ISM_ERR_ARG


def _tg(n):
    h = 2 * np.pi / n
    xf, xc = np.arange(n + 1) * h, (np.arange(n) + 0.5) * h
    u = np.sin(xf)[None, :] * np.cos(xc)[:, None]
    v = -np.cos(xc)[None, :] * np.sin(xf)[:, None]
    p = (np.cos(2 * xc)[None, :] + np.cos(2 * xc)[:, None]) / 4
    u[:, n] = u[:, 0]
    v[n, :] = v[0, :]
    return u, v, p, h


@pytest.mark.parametrize("prec", [ism.ISM_FP64, ism.ISM_MIXED])
@pytest.mark.parametrize("case", ["box", "channel"])
def test_periodic_projection_steps_match_oracle(prec, case):
    """Projection steps with periodic faces against the oracle's steps: the
    Taylor-Green vortex in a fully periodic box, and a channel periodic in x
    between no-slip walls (north wall moving) with a random start; single
    precision velocities, one rounding per stored value and step."""
    import torch
    from synth.inputs import random_field
    if case == "box":
        n = 128
        u0, v0, p0, h = _tg(n)
        nx = ny = n
        vel, wall = (4, 4, 4, 4), (0, 0, 0, 0)
        nu, dt, m = 0.05, 0.002, 16
    else:
        nx, ny, h = 192, 64, 1.0 / 64
        vel, wall = (4, 4, 0, 0), (0, 0, 0, 0.5)
        u0 = 0.2 * random_field(nx + 1, ny, 50)
        v0 = 0.2 * random_field(nx, ny + 1, 51)
        u0[:, nx] = u0[:, 0]
        v0[0, :] = 0.0
        v0[ny, :] = 0.0
        p0 = np.zeros((ny, nx))
        nu, dt, m = 0.02, 1e-4, 16
    f32 = lambda a: np.asarray(a, dtype=np.float32).astype(np.float64)      # noqa: E731
    u0, v0, p0 = f32(u0), f32(v0), f32(p0)
    bc = O.pressure_bc(vel)
    ctx = setup(nx, ny, m, bc, prec=prec, h=h)
    ism.check(ism.ism_set_flow(ctx, vel, wall, None, 1.0))
    ism.check(ism.ism_proj_tol(ctx, 1e-10, 100000, False))
    ud = torch.tensor(u0, dtype=torch.float32, device="cuda:0")
    vd = torch.tensor(v0, dtype=torch.float32, device="cuda:0")
    pd = torch.tensor(p0, dtype=torch.float32, device="cuda:0")
    u, v, p = u0.copy(), v0.copy(), p0.copy()
    s = O.OracleISM(nx, ny, m, bc)
    for _ in range(3):
        assert ism.proj_step(ctx, ud, vd, pd, dt, nu) == ism.ISM_OK
        O.proj_step(u, v, p, h, dt, nu, vel, s, wall_u=wall, tol=1e-12)
    ug, vg, pg = host(ud), host(vd), host(pd)
    assert np.array_equal(ug[:, nx], ug[:, 0])
    if vel[2] == 4:
        assert np.array_equal(vg[ny, :], vg[0, :])
    assert np.abs(ug - u).max() <= 1e-5 * np.abs(u).max()
    assert np.abs(vg - v).max() <= 1e-5 * np.abs(v).max()
    assert np.abs(pg - p).max() <= 1e-4 * np.abs(p).max()
