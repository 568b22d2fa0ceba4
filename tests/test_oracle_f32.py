"""Pins of the oracle's single-precision emulation (the inner solver of the
mixed path) and of its threaded loops.

The float routines (or_rbgs_sweep_f32, or_residual_f32, or_restrict_f32,
or_prolong_add_f32, OracleISM.inner_cycle_f32) are what the GPU's
single-precision kernels are compared against, so each is pinned here to
its FP64 counterpart -- itself pinned by test_oracle_pins.py against closed
forms, spectral solves and brute force -- on data that both precisions
represent exactly: the two must agree to float rounding, a bound derived
from the number of roundings per cell.  A dropped or doubled neighbour, a
wrong divisor, a sign error or a swapped colour order moves a result by
O(1) of the field scale and fails these bounds by five orders of magnitude.
"""
import numpy as np
import pytest

import oracle as O
from synth.inputs import random_field
from tests.conftest import ALL_BCS, PERIODIC_BCS

U = 2.0 ** -24                      # unit roundoff of IEEE single precision
F32_BCS = ALL_BCS + PERIODIC_BCS
SHAPES = [(64, 48, 16), (70, 45, 16), (96, 64, 32)]     # uniform and not a multiple of m


def f32_pair(nx, ny, seed):
    """Random N(0,1) field rounded to float: exactly representable in both
    precisions."""
    a32 = np.ascontiguousarray(random_field(nx, ny, seed), dtype=np.float32)
    return a32, a32.astype(np.float64)


def usable(bc, nx, ny, m):
    """Periodic axes need a multiple of m (and an even cell count)."""
    if bc[0] == O.BC_PERIODIC and nx % m:
        return False
    if bc[2] == O.BC_PERIODIC and ny % m:
        return False
    return True


def sweep_f32(p, b, bc):
    ny, nx = p.shape
    O.lib().or_rbgs_sweep_f32(nx, ny, O.ism_oracle._bc(bc), p, b)


def residual_f32(p, b, bc):
    ny, nx = p.shape
    r = np.empty_like(p)
    O.lib().or_residual_f32(nx, ny, O.ism_oracle._bc(bc), p, b, r)
    return r


@pytest.mark.parametrize("nx,ny,m", SHAPES)
@pytest.mark.parametrize("bc", F32_BCS)
def test_f32_sweep_equals_fp64_sweep_to_rounding(nx, ny, m, bc):
    """One red-black sweep in float against the FP64 sweep (Sec. 3.1).  Per
    red update: 3 additions, 1 subtraction, 1 division, each with relative
    error <= u, on operands bounded by M = max(|p|, |b|): error <= 5 (4M + M)
    u / 3 (d >= 1 at every cell; d = 3 or more in the interior).  A black
    update adds the red errors it reads (at most 4 of them, divided by d >= 2
    where any red neighbour exists): total well inside 64 M u."""
    if not usable(bc, nx, ny, m):
        pytest.skip("periodic axis not a multiple of m")
    p32, p64 = f32_pair(nx, ny, 1)
    b32, b64 = f32_pair(nx, ny, 2)
    M = max(np.abs(p64).max(), np.abs(b64).max())
    sweep_f32(p32, b32, bc)
    O.rbgs_sweep(p64, b64, bc)
    err = np.abs(p32.astype(np.float64) - p64).max()
    assert err <= 64 * M * U, err
    # and the difference is rounding, not nothing: a float sweep is inexact
    assert err > 0.0


@pytest.mark.parametrize("bc", F32_BCS)
def test_f32_sweep_updates_red_before_black(bc):
    """After one float sweep the black cells ((i + j) odd, updated last)
    satisfy their equations to rounding, the red ones do not (red first,
    Sec. 3.1); the residual is measured in FP64 of the float field."""
    nx, ny = 64, 48
    p32, _ = f32_pair(nx, ny, 3)
    b32, b64 = f32_pair(nx, ny, 4)
    sweep_f32(p32, b32, bc)
    r = O.residual(p32.astype(np.float64), b64, bc)
    ii, jj = np.meshgrid(np.arange(nx), np.arange(ny))
    black = (ii + jj) % 2 == 1
    scale = np.abs(b64).max() + 8 * np.abs(p32).max()
    assert np.abs(r[black]).max() <= 16 * scale * U
    assert np.abs(r[~black]).max() > 1e-2 * scale


@pytest.mark.parametrize("nx,ny,m", SHAPES)
@pytest.mark.parametrize("bc", F32_BCS)
def test_f32_residual_equals_fp64_residual_to_rounding(nx, ny, m, bc):
    """r = b - A_f p in float: at most 9 roundings per cell on operands
    bounded by |b| + 8 max|p| (Dirichlet faces contribute -2 p_c)."""
    if not usable(bc, nx, ny, m):
        pytest.skip("periodic axis not a multiple of m")
    p32, p64 = f32_pair(nx, ny, 5)
    b32, b64 = f32_pair(nx, ny, 6)
    r32 = residual_f32(p32, b32, bc).astype(np.float64)
    r64 = O.residual(p64, b64, bc)
    bound = 9 * (np.abs(b64).max() + 8 * np.abs(p64).max()) * U
    assert np.abs(r32 - r64).max() <= bound
    assert np.abs(r32 - r64).max() > 0.0


@pytest.mark.parametrize("nx,ny,m", SHAPES)
def test_f32_restriction_is_the_block_sum_in_double(nx, ny, m):
    """The restriction of a float residual sums the float values in double
    (Sec. 3.2-3.3): equal to numpy block sums (np.add.reduceat) of the same
    values to double rounding, and bit-identical to the FP64 restriction of
    the values converted to double."""
    r32, r64 = f32_pair(nx, ny, 7)
    rc = np.empty((O.ncoarse(ny, m), O.ncoarse(nx, m)))
    O.lib().or_restrict_f32(nx, ny, m, r32, rc)
    ref = np.add.reduceat(np.add.reduceat(r64, np.arange(0, ny, m), axis=0), np.arange(0, nx, m), axis=1)
    np.testing.assert_allclose(rc, ref, rtol=0, atol=1e-12 * m * m)
    assert np.array_equal(rc, O.restrict(r64, m))


@pytest.mark.parametrize("nx,ny,m", SHAPES)
@pytest.mark.parametrize("bc", F32_BCS)
def test_f32_prolongation_rounds_the_fp64_prolongation_once(nx, ny, m, bc):
    """p += P q in float: the bilinear value (Eq. 5) is formed in double,
    rounded to float, added in float: two roundings of |p| + |P q|."""
    if not usable(bc, nx, ny, m):
        pytest.skip("periodic axis not a multiple of m")
    p32, p64 = f32_pair(nx, ny, 8)
    q = random_field(O.ncoarse(nx, m), O.ncoarse(ny, m), 9)
    pq = np.zeros((ny, nx))
    O.prolong_add(pq, q, m, bc)
    O.lib().or_prolong_add_f32(nx, ny, m, O.ism_oracle._bc(bc), np.ascontiguousarray(q), p32)
    O.prolong_add(p64, q, m, bc)
    bound = 2 * U * (np.abs(p64 - pq) + np.abs(pq)) + 1e-300
    assert np.all(np.abs(p32.astype(np.float64) - p64) <= bound)


@pytest.mark.parametrize("nx,ny,m", SHAPES)
@pytest.mark.parametrize("bc", [(0, 0, 0, 0), (0, 1, 0, 0), (1, 1, 1, 1), (2, 2, 0, 0)])
def test_f32_inner_cycle_equals_fp64_cycle_to_rounding(nx, ny, m, bc):
    """One single-precision inner cycle on A_f e = r against one FP64 cycle of
    the same equation from the same (float-representable) start: residual,
    block sums, exact coarse solve, bilinear correction, nu sweeps, mean
    removal.  Relative difference of the fields below 1e-5 (nu = 4 sweeps of
    float rounding on a field of unit scale); an error in any step of the
    emulated cycle moves it by more than 1e-2."""
    if not usable(bc, nx, ny, m):
        pytest.skip("periodic axis not a multiple of m")
    s = O.OracleISM(nx, ny, m, bc, nu=4)
    e32, e64 = f32_pair(nx, ny, 10)
    r32, r64 = f32_pair(nx, ny, 11)
    if s.singular:
        r32 = np.ascontiguousarray(r32 - np.float32(r64.mean()))
        r64 = r32.astype(np.float64)
    s.inner_cycle_f32(e32, r32)
    s.cycle(e64, r64)
    d = np.linalg.norm(e32.astype(np.float64) - e64) / np.linalg.norm(e64)
    assert d <= 1e-5, d


def test_f32_inner_cycles_follow_the_fp64_convergence():
    """Ten inner cycles reduce the residual like ten FP64 cycles (same cycle,
    same order of steps): histories agree to 1e-4 relative until the float
    rounding floor (~1e-6 of the start) is approached."""
    nx, ny, m = 128, 96, 16
    s = O.OracleISM(nx, ny, m, (0, 0, 0, 0), nu=8)
    r32, _ = f32_pair(nx, ny, 12)
    r32 = np.ascontiguousarray(r32 - np.float32(r32.astype(np.float64).mean()))
    r64 = r32.astype(np.float64)
    e32 = np.zeros_like(r32)
    e64 = np.zeros_like(r64)
    n0 = np.linalg.norm(r64)
    for _ in range(10):
        s.inner_cycle_f32(e32, r32)
        s.cycle(e64, r64)
        h32 = np.linalg.norm(O.residual(e32.astype(np.float64), r64, s.bc)) / n0
        h64 = np.linalg.norm(O.residual(e64, r64, s.bc)) / n0
        if h64 < 1e-4:
            break
        assert abs(h32 - h64) <= 1e-4 * h64 + 1e-6, (h32, h64)


@pytest.mark.parametrize("bc", [(0, 0, 0, 0), (0, 1, 2, 2)])
def test_threaded_loops_are_bit_identical_to_one_thread(bc):
    """The row loops may run on several threads (OpenMP): every cell is
    computed by one thread in the same order, so sweeps, residuals, block
    sums, prolongations (FP64 and float) and whole solves give bit-identical
    results for 1 and for all host threads."""
    nx, ny, m = 160, 128, 16
    p, b = random_field(nx, ny, 20), random_field(nx, ny, 21)
    p32, b32 = p.astype(np.float32), b.astype(np.float32)
    q = random_field(nx // m, ny // m, 22)
    out = {}
    prev = O.get_threads()
    try:
        for t in (1, 0):
            O.set_threads(t)
            a = p.copy()
            for _ in range(3):
                O.rbgs_sweep(a, b, bc)
            a32 = p32.copy()
            for _ in range(3):
                sweep_f32(a32, b32, bc)
            pp = p.copy()
            O.prolong_add(pp, q, m, bc)
            sol, cyc, _ = O.OracleISM(nx, ny, m, bc, nu=4).solve(b, tol=1e-4)
            out[t] = (a, a32, O.residual(a, b, bc), residual_f32(a32, b32, bc), O.restrict(a, m), pp, sol, cyc)
    finally:
        O.set_threads(prev)
    for x, y in zip(out[1], out[0]):
        assert np.array_equal(np.asarray(x), np.asarray(y))


def test_threaded_projection_step_is_bit_identical_to_one_thread():
    """Predictor, divergence and correction (Eq. 3-4) on their threaded row
    loops give the one-thread results bit for bit (jet boundaries)."""
    from synth.inputs import jet_inflow
    nx, ny = 96, 64
    jet = (O.VEL_INFLOW, O.VEL_OUTFLOW, O.VEL_FREESLIP, O.VEL_FREESLIP)
    u0 = random_field(nx + 1, ny, 30) * 0.1
    v0 = random_field(nx, ny + 1, 31) * 0.1
    p0 = random_field(nx, ny, 32)
    dp = random_field(nx, ny, 33) * 1e-3
    prof = jet_inflow(ny, width=16, seed=1)
    out = {}
    prev = O.get_threads()
    try:
        for t in (1, 0):
            O.set_threads(t)
            us, vs = O.predictor(u0, v0, p0, 1.0, 0.1, 0.01, jet, u_in=prof, conv_u=1.0)
            b = O.divergence(us, vs, 1.0, 0.1)
            u, v, p = us.copy(), vs.copy(), p0.copy()
            O.correct(u, v, p, dp, 1.0, 0.1, jet)
            out[t] = (us, vs, b, u, v, p)
    finally:
        O.set_threads(prev)
    for x, y in zip(out[1], out[0]):
        assert np.array_equal(x, y)
