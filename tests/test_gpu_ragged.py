"""Grids that are not a multiple of the coarsening factor on the GPU (the last
coarse cell along an axis is narrower; coarse operator solved through the
1-D pencils T V = W V diag(lam)) against the CPU oracle: kernel-level steps,
FP64 solves with the oracle's cycle counts, mixed solves, tensor-core and
CUDA-core coarse solves, the batched ensemble and a full-size case."""
import numpy as np
import pytest

import oracle as O
from synth.inputs import random_field, smooth_rhs
from tests.gpu_util import dev32, dev64, ensure_built, host, ism, rel, setup

pytestmark = pytest.mark.gpu

# nx, ny, m: last-cell widths (x, y) = (8, 6), (4, 20), (4, 6), (4, 16), (32, 24), (16, 6)
SHAPES = [(200, 150, 16), (100, 84, 32), (132, 70, 8), (260, 96, 16), (96, 120, 32), (128, 150, 16)]
BCS = [(0, 0, 0, 0), (0, 1, 0, 0), (1, 1, 1, 1), (1, 0, 0, 1)]
KINDS = {"ism": ism.ISM_COARSE_ISM, "acm": ism.ISM_COARSE_ACM}


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def nc(nx, ny, m):
    return O.ncoarse(ny, m), O.ncoarse(nx, m)


def rhs_for(nx, ny, bc, seed):
    return smooth_rhs(nx, ny, seed) + (0.0 if O.is_singular(bc) else 1e-6)


@pytest.mark.parametrize("nx,ny,m", SHAPES)
@pytest.mark.parametrize("bc", BCS)
def test_residual_restrict(nx, ny, m, bc):
    p, b = random_field(nx, ny, 5), random_field(nx, ny, 6)
    ref = O.restrict(O.residual(p, b, bc), m)
    ctx = setup(nx, ny, m, bc)
    rc = dev64(np.zeros(nc(nx, ny, m)))
    ism.check(ism.ism_residual_restrict(ctx, dev64(p), dev64(b), rc)[0])
    np.testing.assert_allclose(host(rc), ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    rc2, norms = dev64(np.zeros(nc(nx, ny, m))), dev64(np.zeros(2))
    ism.check(ism.ism_residual_restrict_noalloc(nx, ny, m, bc, dev64(p), dev64(b), rc2, norms))
    np.testing.assert_allclose(host(rc2), ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    ctx32 = setup(nx, ny, m, bc, prec=ism.ISM_MIXED)
    rc32 = dev32(np.zeros(nc(nx, ny, m)))
    p32, b32 = p.astype(np.float32), b.astype(np.float32)
    ism.check(ism.ism_residual_restrict(ctx32, dev32(p32), dev32(b32), rc32)[0])
    ref32 = O.restrict(O.residual(p32.astype(np.float64), b32.astype(np.float64), bc), m)
    np.testing.assert_allclose(host(rc32), ref32, rtol=0, atol=1e-5 * np.abs(ref32).max())


@pytest.mark.parametrize("nx,ny,m", SHAPES)
@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("kind", ["ism", "acm"])
def test_prolong_add(nx, ny, m, bc, kind):
    q, p = random_field(O.ncoarse(nx, m), O.ncoarse(ny, m), 8), random_field(nx, ny, 9)
    ref = p.copy()
    if kind == "ism":
        O.prolong_add(ref, q, m, bc)
    else:
        O.prolong_const_add(ref, q, m)
    ctx = setup(nx, ny, m, bc, kind=KINDS[kind])
    pd = dev64(p)
    ism.check(ism.ism_prolong_add(ctx, dev64(q), pd))
    np.testing.assert_allclose(host(pd), ref, rtol=0, atol=1e-14 * np.abs(ref).max())


@pytest.mark.parametrize("nx,ny,m", SHAPES)
@pytest.mark.parametrize("bc", BCS + [(2, 2, 0, 0)])
@pytest.mark.parametrize("kind", ["ism", "acm"])
def test_coarse_solve(nx, ny, m, bc, kind):
    if bc[0] == 2 and (nx % m or nx // m < 4):
        pytest.skip("a periodic axis is a multiple of m with at least 4 coarse cells")
    rc = random_field(O.ncoarse(nx, m), O.ncoarse(ny, m), 7)
    sing = O.is_singular(bc)
    if sing:
        rc -= rc.mean()
    ref = O.OracleISM(nx, ny, m, bc, kind=kind).coarse_solve(rc)
    if sing:
        ref = ref - ref.mean()
    for prec, tcflag, tol in ((ism.ISM_FP64, 0, 1e-10), (ism.ISM_MIXED, 0, 1e-4), (ism.ISM_MIXED, 1, 2e-2)):
        ctx = setup(nx, ny, m, bc, prec=prec, kind=KINDS[kind], coarse_tc=tcflag)
        mk = dev64 if prec == ism.ISM_FP64 else dev32
        ec = mk(np.zeros_like(rc))
        ism.check(ism.ism_coarse_solve(ctx, mk(rc), ec))
        got = host(ec)
        if sing:
            got -= got.mean()
        np.testing.assert_allclose(got, ref, rtol=0, atol=tol * np.abs(ref).max())


def gpu_solve(b, nx, ny, m, bc, prec, tol=1e-8, **opts):
    ctx = setup(nx, ny, m, bc, prec=prec, **opts)
    p = dev64(np.zeros((ny, nx)))
    s, cyc, relres = ism.ism_solve(ctx, dev64(b), p, tol, 100000)
    return s, host(p), cyc, relres, ctx


SOLVE_CASES = [(200, 150, 16, (0, 0, 0, 0)), (100, 84, 32, (0, 1, 0, 0)), (132, 70, 8, (1, 1, 1, 1)),
               (260, 96, 16, (1, 0, 0, 1)), (128, 150, 16, (2, 2, 0, 0))]


@pytest.mark.parametrize("nx,ny,m,bc", SOLVE_CASES)
@pytest.mark.parametrize("kind", ["ism", "acm"])
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
    b = rhs_for(nx, ny, bc, 2)
    ref = O.OracleISM(nx, ny, m, bc)
    p_ex, _, _ = ref.solve(b, tol=1e-11)
    s, p, c, r, _ = gpu_solve(b, nx, ny, m, bc, ism.ISM_MIXED, coarse_tc=coarse_tc)
    assert s == ism.ISM_OK and r <= 1e-8
    assert rel(p, p_ex) <= 1e-9
    bb = ref.prepare_rhs(b)
    assert np.linalg.norm(O.residual(p, bb, bc)) / np.linalg.norm(bb) <= 1.01e-8


def test_options_that_need_uniform_coarse_cells_are_rejected():
    """GMG and the deep ACM V-cycle need uniform coarse cells; the
    accommodative cycle takes a narrower last coarse cell with walls only."""
    ctx = setup(200, 150, 16)
    for field, value in (("kind", ism.ISM_COARSE_GMG), ("kind", ism.ISM_COARSE_ACMV)):
        o = ism.ism_get_options(ctx)
        setattr(o, field, value)
        assert ism.ism_set_options(ctx, o) == ism.ISM_ERR_ARG
    o = ism.ism_get_options(ctx)
    o.cycle = 1
    assert ism.ism_set_options(ctx, o) == ism.ISM_OK
    ctx = setup(200, 128, 16, (0, 0, 2, 2))          # periodic y, x not a multiple of m
    o = ism.ism_get_options(ctx)
    o.cycle = 1
    assert ism.ism_set_options(ctx, o) == ism.ISM_ERR_ARG


def test_batched_ensemble_with_ragged_members():
    shapes = [(200, 150), (100, 84), (132, 70), (256, 256), (260, 96)]
    ms = [16, 32, 8, 16, 16]
    bcs = [(0, 0, 0, 0), (0, 1, 0, 0), (1, 1, 1, 1), (0, 0, 0, 0), (1, 0, 0, 1)]
    ctxs, rhs, ps, bs = [], [], [], []
    for k, ((nx, ny), m, bc) in enumerate(zip(shapes, ms, bcs)):
        ctxs.append(setup(nx, ny, m, bc, prec=ism.ISM_MIXED))
        bs.append(rhs_for(nx, ny, bc, 60 + k))
        rhs.append(dev64(bs[-1]))
        ps.append(dev64(np.zeros((ny, nx))))
    s, cyc, rr = ism.ism_solve_batched(ctxs, rhs, ps, 1e-8, 100000)
    assert s == ism.ISM_OK, ism.status_str(s)
    for k, ((nx, ny), m, bc) in enumerate(zip(shapes, ms, bcs)):
        assert rr[k] <= 1e-8
        p_ex, _, _ = O.OracleISM(nx, ny, m, bc).solve(bs[k], tol=1e-11)
        assert rel(host(ps[k]), p_ex) <= 1e-9, k


def test_full_size_ragged_mixed_solve():
    """2000 x 1990 with 32h: 63 x 63 coarse cells, the last 16 and 6 cells
    wide; the FP64 residual of the returned field measured by the oracle."""
    nx, ny, m = 2000, 1990, 32
    b = smooth_rhs(nx, ny, 23)
    s, p, c, r, _ = gpu_solve(b, nx, ny, m, (0, 0, 0, 0), ism.ISM_MIXED)
    assert s == ism.ISM_OK and r <= 1e-8
    bb = b - b.mean()
    assert np.linalg.norm(O.residual(p, bb, (0, 0, 0, 0))) / np.linalg.norm(bb) <= 1.01e-8
