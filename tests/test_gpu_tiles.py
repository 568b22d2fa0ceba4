"""The fused single-precision pass with its taller region (option
tile_rows = 256: 16 warps, one CTA per SM) against the oracle: K sweeps
element by element against the oracle's float sweeps for every face mix,
including periodic axes and grids that are not a multiple of the tile, and
whole mixed solves (the passes that also carry the prolongation and the
residual) within 1e-9 of the converged oracle solution."""
import numpy as np
import pytest

import oracle as O
from synth.inputs import random_field, smooth_rhs
from tests.conftest import ALL_BCS, PERIODIC_BCS
from tests.gpu_util import dev32, dev64, ensure_built, host, ism, rel, setup

pytestmark = pytest.mark.gpu

SHAPES = [(160, 96, 32), (96, 160, 16), (160, 520, 16), (256, 640, 32)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def usable(nx, ny, m, bc):
    if bc[0] == O.BC_PERIODIC and (nx % m or nx // m < 4):
        return False
    if bc[2] == O.BC_PERIODIC and (ny % m or ny // m < 4):
        return False
    return True


@pytest.mark.parametrize("nx,ny,m", SHAPES)
@pytest.mark.parametrize("bc", ALL_BCS + PERIODIC_BCS)
@pytest.mark.parametrize("sweeps", [1, 4, 8])
def test_tall_region_fused_sweeps_match_oracle(nx, ny, m, bc, sweeps):
    if not usable(nx, ny, m, bc):
        pytest.skip("periodic axis needs a multiple of m with >= 4 coarse cells")
    p = random_field(nx, ny, 3).astype(np.float32)
    b = random_field(nx, ny, 4).astype(np.float32)
    ctx = setup(nx, ny, m, bc, prec=ism.ISM_MIXED, tile_rows=256)
    pd, bd = dev32(p), dev32(b)
    ism.check(ism.ism_smooth(ctx, pd, bd, sweeps))
    ref = np.ascontiguousarray(p.copy())
    bca = np.asarray(bc, dtype=np.int32)
    for _ in range(sweeps):
        O.lib().or_rbgs_sweep_f32(nx, ny, bca, ref, np.ascontiguousarray(b))
    np.testing.assert_allclose(host(pd), ref.astype(np.float64), rtol=0, atol=2e-6 * np.abs(ref).max())


@pytest.mark.parametrize("nx,ny,m,bc", [(256, 640, 16, (0, 0, 0, 0)), (512, 256, 32, (0, 1, 0, 0)),
                                         (160, 500, 16, (1, 1, 1, 1)), (256, 512, 32, (2, 2, 0, 0))])
@pytest.mark.parametrize("k", [8, 6, 4])
def test_tall_region_mixed_solve_matches_oracle(nx, ny, m, bc, k):
    b = smooth_rhs(nx, ny, 5) + (1e-6 if any(x == 1 for x in bc) else 0.0)
    nu = 24 if k == 6 else 32                     # a multiple of the sweeps per pass
    ctx = setup(nx, ny, m, bc, prec=ism.ISM_MIXED, tile_rows=256, nu=nu, sweeps_per_pass=k)
    p = dev64(np.zeros((ny, nx)))
    s, cyc, rr = ism.ism_solve(ctx, dev64(b), p, 1e-8, 100000)
    assert s == ism.ISM_OK and rr <= 1e-8
    p_ex, _, _ = O.OracleISM(nx, ny, m, bc, nu=nu).solve(b, tol=1e-11)
    assert rel(host(p), p_ex) <= 1e-9


def test_region_heights_agree_at_full_size():
    """2048^2, 32h: the solve with 256-row regions reaches the tolerance in the
    cycle count of the 128-row solve (up to one) and to the same solution."""
    n = 2048
    b = smooth_rhs(n, n, 0)
    res = {}
    for rows in (128, 256):
        ctx = setup(n, n, 32, prec=ism.ISM_MIXED, tile_rows=rows)
        p = dev64(np.zeros((n, n)))
        s, cyc, rr = ism.ism_solve(ctx, dev64(b), p, 1e-8, 100000)
        assert s == ism.ISM_OK and rr <= 1e-8
        res[rows] = (cyc, host(p))
    assert abs(res[128][0] - res[256][0]) <= 1
    assert rel(res[256][1], res[128][1]) <= 1e-8


def test_tile_rows_option_is_validated_and_tuned():
    ctx = setup(256, 256, 32, prec=ism.ISM_MIXED)
    o = ism.ism_get_options(ctx)
    assert o.tile_rows == 128
    o.tile_rows = 192
    assert ism.ism_set_options(ctx, o) == ism.ISM_ERR_ARG
    s, best = ism.ism_autotune(ctx, dev64(smooth_rhs(256, 256, 9)), 1e-8, 100000)
    assert s == ism.ISM_OK and best.tile_rows in (128, 256)
    assert ism.ism_get_options(ctx).tile_rows == best.tile_rows


@pytest.mark.parametrize("nx,ny,m,bc", [(160, 96, 32, (0, 0, 0, 0)), (1000, 744, 16, (1, 0, 0, 1)),
                                         (512, 256, 16, (2, 2, 0, 1)), (4096, 4096, 32, (0, 0, 0, 0))])
@pytest.mark.parametrize("tile_rows", [128, 256])
def test_packed_pair_updates_are_bit_identical(nx, ny, m, bc, tile_rows):
    """Option packed: the interior tiles' packed FP32 pair updates round each
    lane like the scalar updates, so K sweeps and whole mixed solves give the
    same bits with packed 0, 1 and 2 (automatic: packed on the 4096^2 grid,
    which runs more than four waves of tiles); the sweeps also match the
    oracle's float sweeps."""
    p = random_field(nx, ny, 3).astype(np.float32)
    b = random_field(nx, ny, 4).astype(np.float32)
    rhs = smooth_rhs(nx, ny, 6) + (1e-6 if any(x == 1 for x in bc) else 0.0)
    outs, sols = [], []
    for pk in (0, 1, 2):
        ctx = setup(nx, ny, m, bc, prec=ism.ISM_MIXED, tile_rows=tile_rows, packed=pk)
        pd = dev32(p)
        ism.check(ism.ism_smooth(ctx, pd, dev32(b), 8))
        outs.append(host(pd))
        q = dev64(np.zeros((ny, nx)))
        s, cyc, rr = ism.ism_solve(ctx, dev64(rhs), q, 1e-8, 100000)
        assert s == ism.ISM_OK and rr <= 1e-8
        sols.append((cyc, host(q)))
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
    assert all(c == sols[0][0] and np.array_equal(x, sols[0][1]) for c, x in sols[1:])
    if nx * ny <= 1000 * 744:
        ref = np.ascontiguousarray(p.copy())
        bca = np.asarray(bc, dtype=np.int32)
        for _ in range(8):
            O.lib().or_rbgs_sweep_f32(nx, ny, bca, ref, np.ascontiguousarray(b))
        np.testing.assert_allclose(outs[0], ref.astype(np.float64), rtol=0, atol=2e-6 * np.abs(ref).max())


def test_packed_option_is_validated():
    ctx = setup(64, 64, 16, prec=ism.ISM_MIXED)
    o = ism.ism_get_options(ctx)
    assert o.packed == 2
    o.packed = 3
    assert ism.ism_set_options(ctx, o) == ism.ISM_ERR_ARG
