"""The streaming single-precision pass (option stream = 1) against the
oracle's float red-black sweeps and inside whole mixed solves: strips of 128
columns with side halos, row chunks with their wavefront warm-up, every face
mix, periodic axes and grids whose width is not a multiple of the strip."""
import numpy as np
import pytest

import oracle as O
from synth.inputs import random_field, smooth_rhs
from tests.conftest import ALL_BCS, PERIODIC_BCS
from tests.gpu_util import dev32, dev64, ensure_built, host, ism, rel, setup

pytestmark = pytest.mark.gpu

SHAPES = [(256, 192, 32), (520, 136, 8), (64, 64, 16), (1000, 700, 32), (128, 2048, 16)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def float_sweeps(p, b, bc, n):
    ny, nx = p.shape
    ref = np.ascontiguousarray(p.copy())
    bca = np.asarray(bc, dtype=np.int32)
    for _ in range(n):
        O.lib().or_rbgs_sweep_f32(nx, ny, bca, ref, np.ascontiguousarray(b))
    return ref.astype(np.float64)


@pytest.mark.parametrize("nx,ny,m", SHAPES)
@pytest.mark.parametrize("bc", ALL_BCS + PERIODIC_BCS)
@pytest.mark.parametrize("sweeps", [1, 2, 4, 12])
def test_streaming_pass_matches_float_sweeps(nx, ny, m, bc, sweeps):
    if (bc[0] == 2 and (nx % m or nx // m < 4)) or (bc[2] == 2 and (ny % m or ny // m < 4)):
        pytest.skip("periodic axes are multiples of m with at least 4 coarse cells")
    p = random_field(nx, ny, 3).astype(np.float32)
    b = random_field(nx, ny, 4).astype(np.float32)
    ctx = setup(nx, ny, m, bc, prec=ism.ISM_MIXED, stream=1)
    pd = dev32(p)
    # 12 sweeps = passes of 8 + 4: the tiled and the streaming pass in turn
    ism.check(ism.ism_smooth(ctx, pd, dev32(b), sweeps))
    ref = float_sweeps(p, b, bc, sweeps)
    np.testing.assert_allclose(host(pd), ref, rtol=0, atol=2e-6 * np.abs(ref).max())


@pytest.mark.parametrize("sweeps", [1, 2, 4])
def test_full_size_streaming_pass(sweeps):
    """4096^2 (fields larger than L2), the pass the option is made for."""
    nx = ny = 4096
    rng = np.random.Generator(np.random.PCG64(31))
    p = rng.standard_normal((ny, nx)).astype(np.float32)
    b = rng.standard_normal((ny, nx)).astype(np.float32)
    ctx = setup(nx, ny, 32, (0, 0, 0, 0), prec=ism.ISM_MIXED, stream=1)
    pd = dev32(p)
    ism.check(ism.ism_smooth(ctx, pd, dev32(b), sweeps))
    ref = float_sweeps(p, b, (0, 0, 0, 0), sweeps)
    np.testing.assert_allclose(host(pd), ref, rtol=0, atol=2e-6 * np.abs(ref).max())


@pytest.mark.parametrize("nx,ny,m,bc", [(512, 512, 16, (0, 0, 0, 0)), (520, 260, 16, (0, 1, 0, 0)),
                                         (256, 256, 16, (2, 2, 2, 2)), (1024, 512, 32, (1, 1, 1, 1))])
@pytest.mark.parametrize("nu,k", [(16, 4), (8, 2), (4, 1)])
def test_mixed_solve_with_streaming_middle_passes(nx, ny, m, bc, nu, k):
    b = smooth_rhs(nx, ny, 5) + (0.0 if O.is_singular(bc) else 1e-6)
    ref = O.OracleISM(nx, ny, m, bc)
    p_ex, _, _ = ref.solve(b, tol=1e-11)
    ctx = setup(nx, ny, m, bc, prec=ism.ISM_MIXED, stream=1, nu=nu, sweeps_per_pass=k)
    p = dev64(np.zeros((ny, nx)))
    s, cyc, r = ism.ism_solve(ctx, dev64(b), p, 1e-8, 100000)
    assert s == ism.ISM_OK and r <= 1e-8
    assert rel(host(p), p_ex) <= 1e-9
    # the same cycle count as the tiled passes (up to rounding)
    ctx2 = setup(nx, ny, m, bc, prec=ism.ISM_MIXED, nu=nu, sweeps_per_pass=k)
    q = dev64(np.zeros((ny, nx)))
    s2, cyc2, _ = ism.ism_solve(ctx2, dev64(b), q, 1e-8, 100000)
    assert s2 == ism.ISM_OK and abs(cyc - cyc2) <= max(2, cyc2 // 20)


def test_stream_option_is_validated():
    ctx = setup(256, 256, 16, prec=ism.ISM_MIXED)
    o = ism.ism_get_options(ctx)
    o.stream = 2
    assert ism.ism_set_options(ctx, o) == ism.ISM_ERR_ARG
