"""ism_residual_norms (the L2 norm and the maximum norm of b - A_f p) against
the oracle's residual, on grids with ragged edges, every face mix and
periodic axes; after a solve it reproduces the solver's own stopping
quantity; non-finite residuals are reported as such."""
import numpy as np
import pytest

import oracle as O
from synth.inputs import random_field, smooth_rhs
from tests.conftest import ALL_BCS, PERIODIC_BCS
from tests.gpu_util import dev64, ensure_built, ism, setup

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


@pytest.mark.parametrize("nx,ny,m", [(160, 96, 32), (200, 136, 16), (256, 192, 32)])
@pytest.mark.parametrize("bc", ALL_BCS + PERIODIC_BCS)
@pytest.mark.parametrize("prec", [ism.ISM_FP64, ism.ISM_MIXED])
def test_residual_norms_match_oracle(nx, ny, m, bc, prec):
    if (bc[0] == 2 and (nx % m or nx // m < 4)) or (bc[2] == 2 and (ny % m or ny // m < 4)):
        pytest.skip("periodic axes are multiples of m with at least 4 coarse cells")
    if prec == ism.ISM_MIXED and nx % 4:
        pytest.skip("the mixed path needs nx % 4 == 0")
    p = random_field(nx, ny, 21)
    b = random_field(nx, ny, 22)
    ctx = setup(nx, ny, m, bc, prec=prec)
    s, l2, mx = ism.ism_residual_norms(ctx, dev64(b), dev64(p))
    assert s == ism.ISM_OK
    r = O.residual(p, b, bc)
    assert abs(l2 - np.linalg.norm(r)) <= 1e-12 * np.linalg.norm(r)
    assert abs(mx - np.abs(r).max()) <= 1e-13 * np.abs(r).max()


@pytest.mark.parametrize("bc", [(0, 0, 0, 0), (0, 1, 0, 0), (2, 2, 0, 0)])
def test_residual_norms_reproduce_the_solver_stopping_quantity(bc):
    nx, ny, m = 256, 192, 32
    b = smooth_rhs(nx, ny, 7) + (0.0 if O.is_singular(bc) else 1e-6)
    if O.is_singular(bc):
        b = b - b.mean()                                  # the equations the solver solves
    ctx = setup(nx, ny, m, bc)
    bd, pd = dev64(b), dev64(np.zeros((ny, nx)))
    s, cyc, rel = ism.ism_solve(ctx, bd, pd, 1e-8, 100000)
    assert s == ism.ISM_OK and rel <= 1e-8
    s, l2, mx = ism.ism_residual_norms(ctx, bd, pd)
    assert s == ism.ISM_OK
    assert abs(l2 / np.linalg.norm(b) - rel) <= 1e-6 * rel
    assert 0.0 < mx <= l2


def test_residual_norms_report_non_finite_and_take_one_output():
    nx, ny = 128, 64
    ctx = setup(nx, ny, 16, (0, 0, 0, 0))
    p = random_field(nx, ny, 3)
    p[10, 20] = np.nan
    s, l2, mx = ism.ism_residual_norms(ctx, dev64(random_field(nx, ny, 4)), dev64(p))
    assert s == ism.ISM_OK and np.isnan(l2) and mx == np.inf
    import ctypes as C
    d = C.c_double(-1.0)
    q = dev64(np.zeros((ny, nx)))
    assert ism.lib().ism_residual_norms(ctx.handle, q.data_ptr(), q.data_ptr(), None, C.byref(d)) == ism.ISM_OK
    assert d.value == 0.0
    assert ism.lib().ism_residual_norms(ctx.handle, q.data_ptr(), q.data_ptr(), None, None) == ism.ISM_ERR_ARG


@pytest.mark.parametrize("bc,shift", [((0, 0, 0, 0), 0.5), ((0, 0, 0, 0), 0.0), ((2, 2, 0, 0), 0.25),
                                      ((0, 1, 0, 0), 0.5)])
@pytest.mark.parametrize("prec", [ism.ISM_FP64, ism.ISM_MIXED])
def test_last_rhs_reports_the_removed_mean_and_compatibility(bc, shift, prec):
    nx, ny, m = 256, 192, 32
    b = smooth_rhs(nx, ny, 9)
    b = b - b.mean() + shift
    ctx = setup(nx, ny, m, bc, prec=prec)
    s, cyc, rel = ism.ism_solve(ctx, dev64(b), dev64(np.zeros((ny, nx))), 1e-8, 100000)
    assert s == ism.ISM_OK and rel <= 1e-8
    s, mean, flag = ism.ism_last_rhs(ctx)
    assert s == ism.ISM_OK
    if O.is_singular(bc):
        assert abs(mean - b.mean()) <= 1e-12 * max(abs(b).mean(), 1e-300)
        assert flag == (abs(b.sum()) > 1e-12 * abs(b).sum())
        assert flag == (shift != 0.0)
    else:
        assert mean == 0.0 and not flag


def test_last_rhs_after_a_projection_step():
    """The divergence of a cavity predictor sums to zero up to rounding."""
    from synth.inputs import smooth_velocity
    nx = ny = 128
    u, v = smooth_velocity(nx, ny, 4)
    import torch
    ud = torch.tensor(0.1 * u, dtype=torch.float32, device="cuda:0")
    vd = torch.tensor(0.1 * v, dtype=torch.float32, device="cuda:0")
    pd = torch.zeros((ny, nx), dtype=torch.float32, device="cuda:0")
    ctx = setup(nx, ny, 16, (0, 0, 0, 0), prec=ism.ISM_MIXED)
    cav = (ism.ISM_VEL_NOSLIP,) * 4
    ism.check(ism.ism_set_flow(ctx, cav, (0, 0, 0, 1.0), None, 1.0))
    ism.check(ism.ism_proj_tol(ctx, 1e-8, 100000, False))
    ism.check(ism.proj_step(ctx, ud, vd, pd, 1e-4, 1e-2))
    s, mean, flag = ism.ism_last_rhs(ctx)
    assert s == ism.ISM_OK and not flag


def test_last_rhs_is_not_replaced_by_the_adjoint_solve():
    """ism_last_rhs describes the caller's last ism_solve / proj_step: the
    adjoint's own pressure solve (proj_step_adjoint) leaves it unchanged."""
    from synth.inputs import random_field, smooth_velocity
    nx = ny = 128
    u, v = smooth_velocity(nx, ny, 4)
    import torch
    ud = torch.tensor(0.1 * u, dtype=torch.float32, device="cuda:0")
    vd = torch.tensor(0.1 * v, dtype=torch.float32, device="cuda:0")
    pd = torch.zeros((ny, nx), dtype=torch.float32, device="cuda:0")
    u0, v0 = ud.clone(), vd.clone()
    ctx = setup(nx, ny, 16, (0, 0, 0, 0), prec=ism.ISM_MIXED)
    ism.check(ism.ism_set_flow(ctx, (ism.ISM_VEL_NOSLIP,) * 4, (0, 0, 0, 1.0), None, 1.0))
    ism.check(ism.ism_proj_tol(ctx, 1e-8, 100000, False))
    ism.check(ism.proj_step(ctx, ud, vd, pd, 1e-4, 1e-2))
    s, mean_fwd, flag_fwd = ism.ism_last_rhs(ctx)
    assert s == ism.ISM_OK
    # adjoint seeds with a large nonzero mean in the divergence of the adjoint solve
    gu = torch.tensor(random_field(nx + 1, ny, 5) + 3.0, dtype=torch.float32, device="cuda:0")
    gv = torch.tensor(random_field(nx, ny + 1, 6) - 2.0, dtype=torch.float32, device="cuda:0")
    gp = torch.tensor(random_field(nx, ny, 7), dtype=torch.float32, device="cuda:0")
    ism.check(ism.proj_step_adjoint(ctx, u0, v0, 1e-4, 1e-2, gu, gv, gp))
    s, mean_after, flag_after = ism.ism_last_rhs(ctx)
    assert s == ism.ISM_OK
    assert mean_after == mean_fwd and flag_after == flag_fwd
