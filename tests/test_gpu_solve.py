"""Whole pressure solves on the GPU against the CPU oracle.

FP64 path: same pressure field to 1e-12 relative and the same cycle count.
Mixed path (single-precision cycles inside FP64 refinement): relative
residual <= tol, and the field within 1e-9 relative of the converged oracle
solution.  Edge cases: zero and non-finite right-hand sides, exact initial
guess, exhausted cycle cap, all face-type mixes, ragged tiles."""
import numpy as np
import pytest

import oracle as O
from synth.inputs import random_field, smooth_rhs
from tests.gpu_util import dev64, ensure_built, host, ism, rel, setup

pytestmark = pytest.mark.gpu

CASES = [  # nx, ny, m, bc
    (256, 256, 16, (0, 0, 0, 0)),     # 256^2 cavity, 16h
    (160, 96, 32, (0, 0, 0, 0)),
    (96, 160, 16, (0, 1, 0, 0)),
    (128, 64, 8, (1, 1, 1, 1)),
    (192, 128, 32, (1, 0, 0, 1)),
    (224, 96, 16, (0, 0, 1, 0)),
]


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def gpu_solve(b, nx, ny, m, bc, prec, tol=1e-8, p0=None, max_cycles=100000, **opts):
    ctx = setup(nx, ny, m, bc, prec=prec, **opts)
    rhs = dev64(b)
    p = dev64(np.zeros((ny, nx)) if p0 is None else p0)
    s, cyc, relres = ism.ism_solve(ctx, rhs, p, tol, max_cycles)
    return s, host(p), cyc, relres, ism.ism_last_history(ctx), ctx


@pytest.mark.parametrize("nx,ny,m,bc", CASES)
def test_fp64_matches_oracle(nx, ny, m, bc):
    b = smooth_rhs(nx, ny, 1) + (1e-6 if any(bc) else 0.0)
    ref = O.OracleISM(nx, ny, m, bc)
    p_ref, c_ref, h_ref = ref.solve(b, tol=1e-8)
    s, p, c, r, h, _ = gpu_solve(b, nx, ny, m, bc, ism.ISM_FP64)
    assert s == ism.ISM_OK
    assert c == c_ref
    assert rel(p, p_ref) <= 1e-12
    np.testing.assert_allclose(h, h_ref, rtol=1e-6, atol=1e-13)   # rounding-level differences
    assert abs(r - h_ref[-1]) <= 1e-13


def test_fp64_acm_matches_oracle():
    nx = ny = 256
    b = smooth_rhs(nx, ny, 0)
    p_ref, c_ref, _ = O.OracleISM(nx, ny, 16, kind="acm").solve(b, tol=1e-8)
    s, p, c, r, h, _ = gpu_solve(b, nx, ny, 16, (0, 0, 0, 0), ism.ISM_FP64, kind=1)
    assert s == ism.ISM_OK and c == c_ref
    assert rel(p, p_ref) <= 1e-12


@pytest.mark.parametrize("bc", [(0, 0, 0, 0), (0, 1, 0, 0)])
def test_gmg_matches_oracle(bc):
    """The GMG comparator (re-discretised five-point coarse operator,
    bilinear correction): FP64 with the oracle's cycle count, mixed to the
    refinement tolerance."""
    nx, ny = 256, 192
    b = smooth_rhs(nx, ny, 2) + (1e-6 if any(bc) else 0.0)
    p_ref, c_ref, _ = O.OracleISM(nx, ny, 16, bc, kind="gmg").solve(b, tol=1e-8)
    s, p, c, r, h, _ = gpu_solve(b, nx, ny, 16, bc, ism.ISM_FP64, kind=ism.ISM_COARSE_GMG)
    assert s == ism.ISM_OK and c == c_ref
    assert rel(p, p_ref) <= 1e-12
    p_ex, _, _ = O.OracleISM(nx, ny, 16, bc, kind="gmg").solve(b, tol=1e-11)
    s, p, c, r, h, _ = gpu_solve(b, nx, ny, 16, bc, ism.ISM_MIXED, kind=ism.ISM_COARSE_GMG)
    assert s == ism.ISM_OK and r <= 1e-8 and rel(p, p_ex) <= 1e-9


@pytest.mark.parametrize("nx,ny,m,bc", [(256, 256, 16, (0, 0, 0, 0)), (256, 128, 8, (0, 1, 0, 0)),
                                         (512, 256, 32, (1, 1, 1, 1))])
def test_deep_acm_vcycle_matches_oracle(nx, ny, m, bc):
    """The deep additive-correction V-cycle (FP64) with the oracle's cycle
    count and field to 1e-12; mixed contexts reject it."""
    b = smooth_rhs(nx, ny, 6) + (1e-6 if any(bc) else 0.0)
    p_ref, c_ref, h_ref = O.OracleACMV(nx, ny, m, bc, nu=8).solve(b, tol=1e-8)
    s, p, c, r, h, _ = gpu_solve(b, nx, ny, m, bc, ism.ISM_FP64, kind=ism.ISM_COARSE_ACMV, nu=8)
    assert s == ism.ISM_OK and c == c_ref
    assert rel(p, p_ref) <= 1e-12
    ctx = setup(nx, ny, m, bc, prec=ism.ISM_MIXED)
    o = ism.ism_get_options(ctx)
    o.kind = ism.ISM_COARSE_ACMV
    assert ism.ism_set_options(ctx, o) == ism.ISM_ERR_ARG


@pytest.mark.parametrize("nx,ny,m,bc", [(256, 192, 16, (0, 0, 0, 0)), (128, 128, 8, (0, 1, 0, 0)),
                                         (160, 96, 32, (1, 1, 1, 1)),
                                         # not multiples of m (narrower last coarse cell): Bench I's 500^2
                                         (500, 500, 8, (0, 0, 0, 0)), (500, 500, 16, (0, 0, 0, 0)),
                                         (500, 500, 32, (0, 0, 0, 0)), (150, 90, 16, (0, 1, 0, 0)),
                                         (200, 120, 32, (1, 1, 1, 1))])
def test_accommodative_strategy_matches_oracle(nx, ny, m, bc):
    """The paper's accommodative strategy (cycle = 1, FP64): the same number
    of coarse Gauss-Seidel iterations as the oracle (the coarse arithmetic is
    rounded step by step in the oracle's order), the same number of fine
    sweeps, the criterion met, the field to 1e-10."""
    b = smooth_rhs(nx, ny, 12) + (1e-6 if any(bc) else 0.0)
    tol_f, tol_c = 1e-7, 1e-6
    p_ref, nc_ref, nf_ref, mx_ref = O.OracleAccommodative(nx, ny, m, bc).solve(b, tol_f=tol_f, tol_c=tol_c)
    ctx = setup(nx, ny, m, bc, prec=ism.ISM_FP64, cycle=1, accom_tol_c=tol_c)
    p = dev64(np.zeros((ny, nx)))
    s, nf, mx = ism.ism_solve(ctx, dev64(b), p, tol_f, 1000000)
    outer, cycles, _ = ism.ism_last_counts(ctx)
    print(f"{nx}x{ny}/{m}: coarse {outer} vs {nc_ref}, fine {cycles} vs {nf_ref}")
    assert s == ism.ISM_OK and mx <= tol_f
    assert outer == nc_ref and cycles == nf_ref
    assert rel(host(p), p_ref) <= 1e-10
    # options: FP64 with the ISM coarse operator only (mixed contexts need nx % 4 == 0)
    for prec, kind in ((ism.ISM_MIXED, 0), (ism.ISM_FP64, ism.ISM_COARSE_ACM)):
        if prec == ism.ISM_MIXED and nx % 4:
            continue
        c2 = setup(nx, ny, m, bc, prec=prec)
        o = ism.ism_get_options(c2)
        o.cycle, o.kind = 1, kind
        assert ism.ism_set_options(c2, o) == ism.ISM_ERR_ARG


def test_config0_ism_beats_acm_on_gpu():
    b = smooth_rhs(256, 256, 0)
    c_ism = gpu_solve(b, 256, 256, 16, (0, 0, 0, 0), ism.ISM_FP64)[2]
    c_acm = gpu_solve(b, 256, 256, 16, (0, 0, 0, 0), ism.ISM_FP64, kind=1)[2]
    assert c_ism < c_acm / 2


@pytest.mark.parametrize("nx,ny,m,bc", CASES)
def test_mixed_reaches_tolerance_and_matches_oracle(nx, ny, m, bc):
    b = smooth_rhs(nx, ny, 2) + (1e-6 if any(bc) else 0.0)
    ref = O.OracleISM(nx, ny, m, bc)
    p_ex, _, h_ex = ref.solve(b, tol=1e-11)
    s, p, c, r, h, ctx = gpu_solve(b, nx, ny, m, bc, ism.ISM_MIXED)
    assert s == ism.ISM_OK
    assert r <= 1e-8 and h[-1] == r
    assert rel(p, p_ex) <= 1e-9
    # the FP64 residual of the returned field, measured by the oracle
    bb = ref.prepare_rhs(b)
    assert np.linalg.norm(O.residual(p, bb, bc)) / np.linalg.norm(bb) <= 1.01e-8
    outer, cycles, _ = ism.ism_last_counts(ctx)
    assert outer >= 2 and cycles == c


def test_zero_rhs_gives_zero_solution():
    s, p, c, r, h, _ = gpu_solve(np.zeros((64, 64)), 64, 64, 16, (0, 0, 0, 0), ism.ISM_FP64,
                                 p0=random_field(64, 64, 1))
    assert s == ism.ISM_OK and c == 0 and np.all(p == 0.0)


def test_exact_initial_guess_needs_no_cycle():
    nx = ny = 128
    b = smooth_rhs(nx, ny, 3)
    p_ref, _, _ = O.OracleISM(nx, ny, 16).solve(b, tol=1e-11)
    for prec in (ism.ISM_FP64, ism.ISM_MIXED):
        s, p, c, r, h, _ = gpu_solve(b, nx, ny, 16, (0, 0, 0, 0), prec, p0=p_ref)
        assert s == ism.ISM_OK and c == 0 and r <= 1e-8


def test_cycle_cap_reports_not_converged_with_last_iterate():
    nx = ny = 128
    b = smooth_rhs(nx, ny, 4)
    ref = O.OracleISM(nx, ny, 16)
    p5, c5, h5 = ref.solve(b, tol=1e-30, max_cycles=5)
    s, p, c, r, h, _ = gpu_solve(b, nx, ny, 16, (0, 0, 0, 0), ism.ISM_FP64, tol=1e-30, max_cycles=5)
    assert s == ism.ISM_ERR_NOT_CONVERGED and c == 5
    assert rel(p, p5) <= 1e-12 and abs(r - h5[-1]) <= 1e-9 * h5[-1]


def test_nonfinite_rhs_is_reported_and_p_untouched():
    b = smooth_rhs(64, 64, 5)
    b[10, 10] = np.nan
    p0 = random_field(64, 64, 6)
    for prec in (ism.ISM_FP64, ism.ISM_MIXED):
        s, p, c, r, h, _ = gpu_solve(b, 64, 64, 16, (0, 0, 0, 0), prec, p0=p0)
        assert s == ism.ISM_ERR_NONFINITE
        assert np.array_equal(p, p0)


@pytest.mark.parametrize("use_graphs", [0, 1, 2])
@pytest.mark.parametrize("check_every", [1, 7])
def test_loop_control_variants_agree(use_graphs, check_every):
    nx = ny = 128
    b = smooth_rhs(nx, ny, 7)
    p_ref, c_ref, _ = O.OracleISM(nx, ny, 16).solve(b, tol=1e-8)
    s, p, c, r, h, _ = gpu_solve(b, nx, ny, 16, (0, 0, 0, 0), ism.ISM_FP64,
                                 use_graphs=use_graphs, check_every=check_every)
    assert s == ism.ISM_OK and c == c_ref and rel(p, p_ref) <= 1e-12


@pytest.mark.parametrize("nu,k", [(8, 4), (8, 2), (4, 4), (6, 3), (1, 1)])
def test_mixed_sweep_fusion_options(nu, k):
    nx, ny = 192, 128
    b = smooth_rhs(nx, ny, 8)
    p_ex, _, _ = O.OracleISM(nx, ny, 32, nu=nu).solve(b, tol=1e-11)
    s, p, c, r, h, _ = gpu_solve(b, nx, ny, 32, (0, 0, 0, 0), ism.ISM_MIXED, nu=nu, sweeps_per_pass=k)
    assert s == ism.ISM_OK and r <= 1e-8 and rel(p, p_ex) <= 1e-9


def test_full_size_mixed_and_fp64_agree():
    """2048^2, 32h: the benchmark's solve.  Both precisions reach 1e-8 and
    agree; the oracle's FP64 residual of the mixed result confirms it."""
    nx = ny = 2048
    b = smooth_rhs(nx, ny, 0)
    s1, pm, cm, rm, _, _ = gpu_solve(b, nx, ny, 32, (0, 0, 0, 0), ism.ISM_MIXED)
    s2, pd, cd, rd, _, _ = gpu_solve(b, nx, ny, 32, (0, 0, 0, 0), ism.ISM_FP64)
    assert s1 == ism.ISM_OK and s2 == ism.ISM_OK and rm <= 1e-8 and rd <= 1e-8
    bb = b - b.mean()
    assert np.linalg.norm(O.residual(pm, bb, (0, 0, 0, 0))) / np.linalg.norm(bb) <= 1.01e-8
    assert rel(pm, pd) <= 1e-7


@pytest.mark.parametrize("nx,ny,m,bc,tcflag", [(2048, 2048, 32, (0, 0, 0, 0), 1), (512, 256, 16, (0, 1, 0, 0), 1),
                                                (160, 96, 32, (1, 1, 1, 1), 1), (2048, 2048, 16, (0, 0, 0, 0), 1),
                                                (4096, 2048, 16, (0, 1, 0, 0), 1), (512, 256, 16, (0, 1, 0, 0), 2)])
def test_mixed_coarse_on_tensor_cores_matches_cuda_cores(nx, ny, m, bc, tcflag):
    """The single-precision cycle with its coarse solve on the tensor cores
    (TF32; one CTA up to 64 x 64 coarse cells, the tiled chain above that and
    under coarse_tc 2) reaches the same FP64 tolerance as with the FP32
    CUDA-core coarse solve, to the same solution, within a few cycles."""
    b = smooth_rhs(nx, ny, 4) + (1e-6 if any(bc) else 0.0)
    s0, p0, c0, r0, _, _ = gpu_solve(b, nx, ny, m, bc, ism.ISM_MIXED, coarse_tc=0)
    s1, p1, c1, r1, _, _ = gpu_solve(b, nx, ny, m, bc, ism.ISM_MIXED, coarse_tc=tcflag)
    print(f"{nx}x{ny}/{m}: cycles CUDA cores {c0}, tensor cores {c1}")
    assert s0 == ism.ISM_OK and s1 == ism.ISM_OK and r0 <= 1e-8 and r1 <= 1e-8
    assert rel(p1, p0) <= 1e-8
    assert abs(c1 - c0) <= max(3, c0 // 10)


@pytest.mark.parametrize("prec", [0, 1])
def test_autotune_picks_a_working_candidate(prec):
    nx = ny = 256
    b = smooth_rhs(nx, ny, 9)
    ctx = setup(nx, ny, 32, (0, 0, 0, 0), prec=prec)
    s, o = ism.ism_autotune(ctx, dev64(b), 1e-8, 100000)
    assert s == ism.ISM_OK and o.nu % o.sweeps_per_pass == 0
    cur = ism.ism_get_options(ctx)
    assert (cur.nu, cur.sweeps_per_pass, cur.stream, cur.inner_tol, cur.tile_rows, cur.coarse_tc) == \
        (o.nu, o.sweeps_per_pass, o.stream, o.inner_tol, o.tile_rows, o.coarse_tc)
    assert o.coarse_tc in (0, 1, 2)
    p_ex, _, _ = O.OracleISM(nx, ny, 32, nu=o.nu).solve(b, tol=1e-11)
    p = dev64(np.zeros((ny, nx)))
    s, c, r = ism.ism_solve(ctx, dev64(b), p, 1e-8, 100000)
    assert s == ism.ISM_OK and r <= 1e-8 and rel(host(p), p_ex) <= 1e-9


def test_autotune_from_a_warm_start():
    """ism_autotune_from times solves started from a given guess (here the
    solution of a nearby right-hand side, as a time stepper's previous
    increment): the guess is not modified, the options it keeps solve that
    problem from that guess to the tolerance, and the result matches the
    oracle."""
    nx = ny = 256
    b0 = smooth_rhs(nx, ny, 9)
    b = b0 + 0.05 * smooth_rhs(nx, ny, 10)
    ctx = setup(nx, ny, 32, (0, 0, 0, 0), prec=ism.ISM_MIXED)
    p0 = dev64(np.zeros((ny, nx)))
    s, _, _ = ism.ism_solve(ctx, dev64(b0), p0, 1e-8, 100000)
    assert s == ism.ISM_OK
    keep = host(p0).copy()
    s, o = ism.ism_autotune_from(ctx, dev64(b), p0, 1e-8, 100000)
    assert s == ism.ISM_OK and o.nu % o.sweeps_per_pass == 0
    assert np.array_equal(host(p0), keep)
    cur = ism.ism_get_options(ctx)
    assert (cur.nu, cur.inner_tol, cur.coarse_tc) == (o.nu, o.inner_tol, o.coarse_tc)
    q = dev64(keep)
    s, c, r = ism.ism_solve(ctx, dev64(b), q, 1e-8, 100000)
    assert s == ism.ISM_OK and r <= 1e-8
    p_ex, _, _ = O.OracleISM(nx, ny, 32, nu=o.nu).solve(b, tol=1e-11)
    assert rel(host(q), p_ex) <= 1e-9


@pytest.mark.parametrize("nx,ny,expect", [(512, 512, (16, 32)), (144, 96, (16,)), (96, 64, (16, 32))])
def test_setup_chooses_coarsening(nx, ny, expect):
    """coarsen = 0: the library times solves with 16h and 32h (those that
    divide the grid) and keeps the faster; the context then solves to 1e-8."""
    s, ctx = ism.ism_setup(nx, ny, 1.0 / nx, (0, 0, 0, 0), 0, ism.ISM_MIXED)
    assert s == ism.ISM_OK
    m = ism.ism_coarsening(ctx)
    assert m in expect and ctx.m == m
    b = smooth_rhs(nx, ny, 31)
    p = dev64(np.zeros((ny, nx)))
    st, cyc, rr = ism.ism_solve(ctx, dev64(b), p, 1e-8, 100000)
    assert st == ism.ISM_OK and rr <= 1e-8
    p_ex, _, _ = O.OracleISM(nx, ny, m, nu=ism.ism_get_options(ctx).nu).solve(b, tol=1e-11)
    assert rel(host(p), p_ex) <= 1e-9
