"""Each step of the cycle on the GPU (kernel-level C-ABI entry points) against
the CPU oracle, element by element, on grids that span several 64 x 64
tiles with ragged edges and every face-type mix."""
import numpy as np
import pytest

import oracle as O
from synth.inputs import random_field, smooth_rhs
from tests.conftest import ALL_BCS
from tests.gpu_util import dev32, dev64, ensure_built, host, ism, setup

pytestmark = pytest.mark.gpu

SHAPES = [(160, 96, 32), (96, 160, 16), (128, 64, 8), (256, 192, 32)]
KINDS = {"ism": ism.ISM_COARSE_ISM, "acm": ism.ISM_COARSE_ACM, "gmg": ism.ISM_COARSE_GMG}


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


@pytest.mark.parametrize("nx,ny,m", SHAPES)
@pytest.mark.parametrize("bc", ALL_BCS)
def test_smooth_fp64(nx, ny, m, bc):
    p = random_field(nx, ny, 1)
    b = random_field(nx, ny, 2)
    ctx = setup(nx, ny, m, bc)
    pd, bd = dev64(p), dev64(b)
    ism.check(ism.ism_smooth(ctx, pd, bd, 3))
    ref = p.copy()
    for _ in range(3):
        O.rbgs_sweep(ref, b, bc)
    np.testing.assert_allclose(host(pd), ref, rtol=0, atol=1e-13 * np.abs(ref).max())


@pytest.mark.parametrize("nx,ny,m", SHAPES)
@pytest.mark.parametrize("bc", ALL_BCS)
@pytest.mark.parametrize("sweeps", [1, 4, 6, 7])
def test_smooth_fused_fp32(nx, ny, m, bc, sweeps):
    """Fused multi-sweep pass (temporal blocking) against the oracle's float
    sweeps: the same operations in the same order, so agreement is at the
    level of one rounding per update."""
    p = random_field(nx, ny, 3).astype(np.float32)
    b = random_field(nx, ny, 4).astype(np.float32)
    ctx = setup(nx, ny, m, bc, prec=ism.ISM_MIXED)
    pd, bd = dev32(p), dev32(b)
    ism.check(ism.ism_smooth(ctx, pd, bd, sweeps))
    ref = np.ascontiguousarray(p.copy())
    L = O.lib()
    bca = np.asarray(bc, dtype=np.int32)
    for _ in range(sweeps):
        L.or_rbgs_sweep_f32(nx, ny, bca, ref, np.ascontiguousarray(b))
    np.testing.assert_allclose(host(pd), ref.astype(np.float64), rtol=0, atol=2e-6 * np.abs(ref).max())


@pytest.mark.parametrize("nx,ny,m", SHAPES)
@pytest.mark.parametrize("bc", ALL_BCS)
def test_residual_restrict(nx, ny, m, bc):
    p = random_field(nx, ny, 5)
    b = random_field(nx, ny, 6)
    ctx = setup(nx, ny, m, bc)
    rc = dev64(np.zeros((ny // m, nx // m)))
    s, rnorm, psum = ism.ism_residual_restrict(ctx, dev64(p), dev64(b), rc)
    ism.check(s)
    r = O.residual(p, b, bc)
    ref = O.restrict(r, m)
    np.testing.assert_allclose(host(rc), ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    assert abs(rnorm - np.linalg.norm(r)) <= 1e-12 * np.linalg.norm(r)
    assert abs(psum - p.sum()) <= 1e-12 * np.abs(p).sum()
    # single precision
    ctx32 = setup(nx, ny, m, bc, prec=ism.ISM_MIXED)
    rc32 = dev32(np.zeros((ny // m, nx // m)))
    p32, b32 = p.astype(np.float32), b.astype(np.float32)
    ism.check(ism.ism_residual_restrict(ctx32, dev32(p32), dev32(b32), rc32)[0])
    ref32 = O.restrict(O.residual(p32.astype(np.float64), b32.astype(np.float64), bc), m)
    np.testing.assert_allclose(host(rc32), ref32, rtol=0, atol=1e-5 * np.abs(ref32).max())


@pytest.mark.parametrize("nx,ny,m", SHAPES)
@pytest.mark.parametrize("bc", ALL_BCS)
@pytest.mark.parametrize("kind", ["ism", "acm", "gmg"])
def test_coarse_solve(nx, ny, m, bc, kind):
    ncx, ncy = nx // m, ny // m
    rc = random_field(ncx, ncy, 7)
    if not any(bc):
        rc -= rc.mean()
    ref = O.OracleISM(nx, ny, m, bc, kind=kind).coarse_solve(rc)
    # FP64; FP32 on the CUDA cores; on the tensor cores (tcgen05): coarse_tc 1
    # runs the single-CTA kernel on these coarse grids, four chained products
    # of operands rounded to TF32 (2^-11 relative); coarse_tc 2 the tiled
    # chain of four launches in split TF32 (about FP32 rounding)
    for prec, tcflag, tol in ((ism.ISM_FP64, 0, 1e-11), (ism.ISM_MIXED, 0, 2e-5), (ism.ISM_MIXED, 1, 1e-2),
                              (ism.ISM_MIXED, 2, 5e-5)):
        ctx = setup(nx, ny, m, bc, prec=prec, kind=KINDS[kind], coarse_tc=tcflag)
        mk = dev64 if prec == ism.ISM_FP64 else dev32
        ec = mk(np.zeros_like(rc))
        ism.check(ism.ism_coarse_solve(ctx, mk(rc), ec))
        got = host(ec)
        if not any(bc):
            got -= got.mean()       # solutions are defined up to a constant
        np.testing.assert_allclose(got, ref - (ref.mean() if not any(bc) else 0.0),
                                   rtol=0, atol=tol * np.abs(ref).max())


@pytest.mark.parametrize("nx,ny,m", SHAPES)
@pytest.mark.parametrize("bc", ALL_BCS)
@pytest.mark.parametrize("kind", ["ism", "acm", "gmg"])
def test_prolong_add(nx, ny, m, bc, kind):
    q = random_field(nx // m, ny // m, 8)
    p = random_field(nx, ny, 9)
    ref = p.copy()
    if kind != "acm":                     # ISM and GMG share the bilinear correction
        O.prolong_add(ref, q, m, bc)
    else:
        O.prolong_const_add(ref, q, m)
    ctx = setup(nx, ny, m, bc, kind=KINDS[kind])
    pd = dev64(p)
    ism.check(ism.ism_prolong_add(ctx, dev64(q), pd))
    np.testing.assert_allclose(host(pd), ref, rtol=0, atol=1e-14 * np.abs(ref).max())


def test_full_size_single_cycle_fp32():
    """2048^2, 32h (the benchmark grid): one cycle of GPU steps against the
    oracle's steps from the same single-precision state."""
    nx = ny = 2048
    m = 32
    b = smooth_rhs(nx, ny, 0).astype(np.float32)
    rng = np.random.Generator(np.random.PCG64(11))
    p = (rng.standard_normal((ny, nx)) * 1e-6).astype(np.float32)
    ctx = setup(nx, ny, m, prec=ism.ISM_MIXED)
    pd, bd = dev32(p), dev32(b)
    rc = dev32(np.zeros((ny // m, nx // m)))
    ism.check(ism.ism_residual_restrict(ctx, pd, bd, rc)[0])
    rc_ref = O.restrict(O.residual(p.astype(np.float64), b.astype(np.float64), (0, 0, 0, 0)), m)
    np.testing.assert_allclose(host(rc), rc_ref, rtol=0, atol=1e-4 * np.abs(rc_ref).max())
    ism.check(ism.ism_smooth(ctx, pd, bd, 8))
    ref = np.ascontiguousarray(p.copy())
    bca = np.zeros(4, dtype=np.int32)
    for _ in range(8):
        O.lib().or_rbgs_sweep_f32(nx, ny, bca, ref, np.ascontiguousarray(b))
    np.testing.assert_allclose(host(pd), ref.astype(np.float64), rtol=0, atol=2e-6 * np.abs(ref).max())


def _launches(ctx):
    return ism.ism_last_counts(ctx)[2]


@pytest.mark.parametrize("nx,ny,m,tcflag", [
    (2048, 2048, 32, 1),    # 64 x 64: one CTA
    (2048, 2048, 32, 2),    # the same grid through the tiled chain
    (160, 96, 32, 1),
    (160, 96, 32, 2),       # 5 x 3: one partly filled block
    (512, 256, 8, 1),
    (2048, 2048, 16, 1),    # 128 x 128: tiled chain
    (1024, 512, 8, 1),      # 128 x 64
    (8192, 4096, 32, 1),    # 256 x 128: the jet's coarse grid
    (2304, 2560, 16, 1),    # 144 x 160: two 128-row blocks
    (3000, 2200, 32, 1),    # 94 x 69, ragged last coarse cells (1-D pencils)
    (8192, 8192, 32, 2),    # 256 x 256: the largest grid of the tiled chain
])
def test_coarse_solve_tensor_cores_against_oracle(nx, ny, m, tcflag):
    """The tcgen05 coarse solves against the FP64 oracle.  The single-CTA
    kernel (coarse grids up to 64 x 64 under coarse_tc 1) carries the error of
    TF32 operands: well below 1e-2 of the solution's scale and far above FP32
    rounding.  The tiled chain (above 64 x 64, or coarse_tc 2) computes in
    split TF32 and stays within a few FP32 roundings, like the CUDA-core
    kernels, but differs from them bit for bit.  The launch counts show which
    engine ran: 2 launches on the CUDA cores, 1 for the single CTA, 4 for the
    chain."""
    ncx, ncy = -(-nx // m), -(-ny // m)
    rc = random_field(ncx, ncy, 9)
    rc -= rc.mean()
    ref = O.OracleISM(nx, ny, m, (0, 0, 0, 0)).coarse_solve(rc)
    ref -= ref.mean()
    errs, outs, nl = {}, {}, {}
    for flag in (0, tcflag):
        ctx = setup(nx, ny, m, prec=ism.ISM_MIXED, coarse_tc=flag)
        ec = dev32(np.zeros_like(rc))
        l0 = _launches(ctx)
        ism.check(ism.ism_coarse_solve(ctx, dev32(rc), ec))
        nl[flag] = _launches(ctx) - l0
        got = host(ec)
        outs[flag] = got.copy()
        got -= got.mean()
        errs[flag] = np.abs(got - ref).max() / np.abs(ref).max()
    print(f"{nx}x{ny}/{m} ({ncx}x{ncy}) tc={tcflag}: max error FP32 {errs[0]:.2e}, tensor cores {errs[tcflag]:.2e}")
    assert errs[0] <= 2e-5 and nl[0] == 2
    if tcflag == 1 and ncx <= 64 and ncy <= 64:
        assert nl[tcflag] == 1
        assert 2e-5 < errs[tcflag] <= 1e-2
    else:
        assert nl[tcflag] == 4
        assert errs[tcflag] <= 5e-5
        assert not np.array_equal(outs[tcflag], outs[0])


def test_coarse_solve_above_the_tensor_core_limit_takes_the_cuda_cores():
    """512 x 128 coarse cells (beyond 256 along x): coarse_tc 1 and 2 fall back
    to the FP32 CUDA-core kernels (2 launches) and give their result bit for
    bit."""
    nx, ny, m = 16384, 4096, 32
    rc = random_field(nx // m, ny // m, 9)
    rc -= rc.mean()
    outs = []
    for flag in (0, 1, 2):
        ctx = setup(nx, ny, m, prec=ism.ISM_MIXED, coarse_tc=flag)
        ec = dev32(np.zeros_like(rc))
        l0 = _launches(ctx)
        ism.check(ism.ism_coarse_solve(ctx, dev32(rc), ec))
        assert _launches(ctx) - l0 == 2
        outs.append(host(ec))
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
