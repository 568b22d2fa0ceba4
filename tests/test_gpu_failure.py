"""Failure detection on the GPU without a GPU fault.

Every wait of the tensor-core coarse solve has a time limit; when it runs
out the kernel records the failure, lets its bulk copies finish, frees its
tensor memory and returns, and the solve ends with ISM_ERR_CUDA.  The test
makes a wait run out on purpose (option fault_test: the kernel first waits
for an mbarrier phase that nothing completes -- a flag that nothing sets),
checks the status and the time it took, and then shows that the same context
and the device still work: a normal solve on the same context and a fresh
one, both checked against the oracle.
"""
import time

import numpy as np
import pytest

import oracle as O
from synth.inputs import smooth_rhs
from tests.gpu_util import dev64, ensure_built, host, ism, rel, setup, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


@pytest.mark.parametrize("use_graphs", [2, 0])
@pytest.mark.parametrize("coarse_tc", [1, 2])
def test_coarse_wait_that_runs_out_ends_the_solve_with_a_status(use_graphs, coarse_tc):
    nx = ny = 256
    m = 32                                   # 8 x 8 coarse grid: the tensor-core coarse solve
    b = smooth_rhs(nx, ny, 3)                # (coarse_tc 1: one CTA; 2: the tiled chain)
    ctx = setup(nx, ny, m, prec=ism.ISM_MIXED, coarse_tc=coarse_tc, fault_test=1, use_graphs=use_graphs)
    p0 = np.zeros((ny, nx))
    p = dev64(p0)
    t0 = time.perf_counter()
    s, cyc, _ = ism.ism_solve(ctx, dev64(b), p, 1e-8, 100000)
    dt = time.perf_counter() - t0
    assert s == ism.ISM_ERR_CUDA
    assert dt < 10.0                         # the loops stop after the failed coarse solve

    # the same context, the failure switched off: a normal solve
    o = ism.ism_get_options(ctx)
    o.fault_test = 0
    ism.check(ism.ism_set_options(ctx, o))
    p_ex, _, _ = O.OracleISM(nx, ny, m, nu=o.nu).solve(b, tol=1e-11)
    p = dev64(p0)
    s, cyc, rr = ism.ism_solve(ctx, dev64(b), p, 1e-8, 100000)
    assert s == ism.ISM_OK and rr <= 1e-8
    assert rel(host(p), p_ex) <= 1e-9

    # a fresh context and plain torch work on the same device
    ctx2 = setup(nx, ny, m, prec=ism.ISM_MIXED, coarse_tc=coarse_tc)
    p = dev64(p0)
    s, _, rr = ism.ism_solve(ctx2, dev64(b), p, 1e-8, 100000)
    assert s == ism.ISM_OK and rr <= 1e-8
    x = torch.arange(10, dtype=torch.float32, device="cuda:0")
    assert float(x.sum()) == 45.0


def test_fault_test_option_is_validated():
    ctx = setup(64, 64, 16, prec=ism.ISM_MIXED)
    o = ism.ism_get_options(ctx)
    assert o.fault_test == 0
    o.fault_test = 2
    assert ism.ism_set_options(ctx, o) == ism.ISM_ERR_ARG
