"""Batched ensemble (many uneven problems advanced by one set of launches)
against the CPU oracle and against single-problem solves."""
import numpy as np
import pytest

import oracle as O
from synth.inputs import batch_shapes, smooth_rhs
from tests.gpu_util import dev64, ensure_built, host, ism, rel, setup

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def make_batch(shapes, ms, bcs, seed0=100, **opts):
    ctxs, rhs, ps, bs = [], [], [], []
    for k, ((nx, ny), m, bc) in enumerate(zip(shapes, ms, bcs)):
        ctxs.append(setup(nx, ny, m, bc, prec=ism.ISM_MIXED, **opts))
        b = smooth_rhs(nx, ny, seed0 + k) + (1e-6 if any(bc) else 0.0)
        bs.append(b)
        rhs.append(dev64(b))
        ps.append(dev64(np.zeros((ny, nx))))
    return ctxs, rhs, ps, bs


def test_batched_small_ensemble_matches_oracle_and_single_solves():
    shapes = batch_shapes(10, seed=3, lo=128, hi=320)
    ms = [16 if k % 2 else 32 for k in range(10)]
    bcs = [(0, 0, 0, 0)] * 8 + [(0, 1, 0, 0), (1, 1, 1, 1)]
    ctxs, rhs, ps, bs = make_batch(shapes, ms, bcs)
    s, cyc, rr = ism.ism_solve_batched(ctxs, rhs, ps, 1e-8, 100000)
    assert s == ism.ISM_OK, ism.status_str(s)
    for k, ((nx, ny), m, bc) in enumerate(zip(shapes, ms, bcs)):
        assert rr[k] <= 1e-8
        p = host(ps[k])
        ref = O.OracleISM(nx, ny, m, bc, nu=ism.ism_get_options(ctxs[k]).nu)
        p_ex, _, _ = ref.solve(bs[k], tol=1e-11)
        assert rel(p, p_ex) <= 1e-9, k
        # the same problem solved alone
        q = dev64(np.zeros((ny, nx)))
        s1, c1, r1 = ism.ism_solve(ctxs[k], rhs[k], q, 1e-8, 100000)
        assert s1 == ism.ISM_OK and abs(c1 - cyc[k]) <= 2
        assert rel(p, host(q)) <= 1e-9


def test_batched_repeat_and_zero_rhs():
    shapes = [(128, 128), (256, 128), (160, 96)]
    ctxs, rhs, ps, bs = make_batch(shapes, [16, 32, 32], [(0, 0, 0, 0)] * 3)
    rhs[1] = dev64(np.zeros((128, 256)))
    first = None
    for _ in range(2):                       # second call reuses the cached graph
        for p in ps:
            p.zero_()
        s, cyc, rr = ism.ism_solve_batched(ctxs, rhs, ps, 1e-8, 100000)
        assert s == ism.ISM_OK
        assert cyc[1] == 0 and np.all(host(ps[1]) == 0.0)
        out = [host(p) for p in ps]
        if first is not None:
            for a, b in zip(first, out):
                assert np.array_equal(a, b)
        first = out
    # a different set of problems rebuilds the plan
    s, cyc, rr = ism.ism_solve_batched(ctxs[::-1], rhs[::-1], ps[::-1], 1e-8, 100000)
    assert s == ism.ISM_OK and all(r <= 1e-8 for r in rr)


def test_batched_rejects_mixed_options_and_fp64():
    a = setup(128, 128, 16, prec=ism.ISM_MIXED)
    b = setup(128, 128, 16, prec=ism.ISM_MIXED, nu=8, sweeps_per_pass=4)
    c = setup(128, 128, 16, prec=ism.ISM_FP64)
    r = dev64(np.zeros((128, 128)))
    p = dev64(np.zeros((128, 128)))
    assert ism.ism_solve_batched([a, b], [r, r], [p, p])[0] == ism.ISM_ERR_ARG
    assert ism.ism_solve_batched([a, c], [r, r], [p, p])[0] == ism.ISM_ERR_ARG
    assert ism.ism_solve_batched([a, a], [r, r], [p, p])[0] == ism.ISM_ERR_ARG


def test_batched_full_ensemble_256():
    """256 uneven Neumann cavity problems (128..1024 per side, 16h / 32h by
    size): every problem reaches 1e-8 measured by the oracle's FP64 residual;
    three are compared with the oracle solution."""
    shapes = batch_shapes(256, seed=0)
    ms = [16 if min(nx, ny) < 512 else 32 for nx, ny in shapes]
    ctxs, rhs, ps, bs = make_batch(shapes, ms, [(0, 0, 0, 0)] * 256, seed0=1000)
    s, cyc, rr = ism.ism_solve_batched(ctxs, rhs, ps, 1e-8, 200000)
    assert s == ism.ISM_OK
    for k in range(256):
        p = host(ps[k])
        b = bs[k] - bs[k].mean()
        assert np.linalg.norm(O.residual(p, b, (0, 0, 0, 0))) / np.linalg.norm(b) <= 1.01e-8, k
    small = sorted(range(256), key=lambda k: shapes[k][0] * shapes[k][1])[:3]
    for k in small:
        nx, ny = shapes[k]
        p_ex, _, _ = O.OracleISM(nx, ny, ms[k], nu=ism.ism_get_options(ctxs[k]).nu).solve(bs[k], tol=1e-11)
        assert rel(host(ps[k]), p_ex) <= 1e-9


@pytest.mark.parametrize("nu", [72, 128])
def test_batched_many_passes_per_cycle(nu):
    """Cycles of nu / 8 > 8 fused passes (9 and 16 passes): every pass keeps
    its own argument table; results match single-problem solves."""
    shapes = [(256, 128), (160, 160), (384, 256)]
    ctxs, rhs, ps, bs = make_batch(shapes, [16, 32, 16], [(0, 0, 0, 0)] * 3, nu=nu, sweeps_per_pass=8)
    s, cyc, rr = ism.ism_solve_batched(ctxs, rhs, ps, 1e-8, 100000)
    assert s == ism.ISM_OK and all(r <= 1e-8 for r in rr)
    for k, (nx, ny) in enumerate(shapes):
        q = dev64(np.zeros((ny, nx)))
        s1, c1, r1 = ism.ism_solve(ctxs[k], rhs[k], q, 1e-8, 100000)
        assert s1 == ism.ISM_OK and abs(c1 - cyc[k]) <= 2
        assert rel(host(ps[k]), host(q)) <= 1e-9


def test_batched_tensor_core_and_cuda_core_coarse_agree():
    """The ensemble with its coarse solves on the tensor cores (coarse_tc 1:
    TF32, one CTA per problem; 2: the tiled split-TF32 chain over all
    problems' blocks) and on the CUDA cores (FP32): all reach 1e-8 per problem
    and agree to the refinement tolerance; the chain, accurate to about FP32
    rounding, takes the CUDA-core cycle counts within one cycle."""
    shapes = batch_shapes(8, seed=5, lo=128, hi=512)
    out = {}
    for tcflag in (0, 1, 2):
        ctxs, rhs, ps, bs = make_batch(shapes, [16] * 8, [(0, 0, 0, 0)] * 7 + [(0, 1, 0, 0)], seed0=300,
                                       coarse_tc=tcflag)
        s, cyc, rr = ism.ism_solve_batched(ctxs, rhs, ps, 1e-8, 100000)
        assert s == ism.ISM_OK and all(r <= 1e-8 for r in rr)
        out[tcflag] = ([host(p) for p in ps], cyc)
    for tcflag in (1, 2):
        for a, b in zip(out[0][0], out[tcflag][0]):
            assert rel(b, a) <= 1e-8
    assert all(abs(a - b) <= 1 for a, b in zip(out[0][1], out[2][1]))
    print("cycles CUDA cores", out[0][1], "tensor cores", out[1][1], "chain", out[2][1])


def test_batched_chain_on_coarse_grids_above_64():
    """Problems whose coarse grids exceed 64 x 64 (128 x 64, 96 x 96, 144 x 80
    at 16h) take the tiled chain under coarse_tc 1, batched like the rest:
    each result equals its single-problem solve (which takes the same chain)
    and the smallest the oracle's solution."""
    shapes = [(2048, 1024), (1536, 1536), (2304, 1280), (256, 256)]
    ctxs, rhs, ps, bs = make_batch(shapes, [16] * 4, [(0, 0, 0, 0), (0, 1, 0, 0), (0, 0, 0, 0), (0, 0, 0, 0)],
                                   seed0=700, coarse_tc=1)
    s, cyc, rr = ism.ism_solve_batched(ctxs, rhs, ps, 1e-8, 100000)
    assert s == ism.ISM_OK and all(r <= 1e-8 for r in rr)
    for k, (nx, ny) in enumerate(shapes):
        q = dev64(np.zeros((ny, nx)))
        s1, c1, r1 = ism.ism_solve(ctxs[k], rhs[k], q, 1e-8, 100000)
        assert s1 == ism.ISM_OK and abs(c1 - cyc[k]) <= 2
        assert rel(host(ps[k]), host(q)) <= 1e-9
    p_ex, _, _ = O.OracleISM(256, 256, 16, nu=ism.ism_get_options(ctxs[3]).nu).solve(bs[3], tol=1e-11)
    assert rel(host(ps[3]), p_ex) <= 1e-9


def test_autotune_batched_sets_a_common_nu():
    shapes = batch_shapes(6, seed=9, lo=128, hi=384)
    ctxs, rhs, ps, bs = make_batch(shapes, [16] * 6, [(0, 0, 0, 0)] * 6, seed0=500)
    s, nu = ism.ism_autotune_batched(ctxs, rhs, ps, 1e-8)
    assert s == ism.ISM_OK and nu in (16, 32, 64, 128)
    assert all(ism.ism_get_options(c).nu == nu for c in ctxs)
    tcs = {ism.ism_get_options(c).coarse_tc for c in ctxs}
    assert len(tcs) == 1 and tcs <= {0, 1, 2}
    for p in ps:
        p.zero_()
    s, cyc, rr = ism.ism_solve_batched(ctxs, rhs, ps, 1e-8, 100000)
    assert s == ism.ISM_OK and all(r <= 1e-8 for r in rr)
    for k, (nx, ny) in enumerate(shapes):
        p_ex, _, _ = O.OracleISM(nx, ny, 16, nu=nu).solve(bs[k], tol=1e-11)
        assert rel(host(ps[k]), p_ex) <= 1e-9
