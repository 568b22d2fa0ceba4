"""The allocation-free residual + restriction entry point, for callers that
cannot allocate device memory when they need a residual (real-time loops
that cannot take cudaMalloc's implicit synchronisation, hosts whose device
memory belongs to their own arena), against the context-based
ism_residual_restrict and the oracle's residual and block sums, on two calls
in a row through the C ABI.  Named to be collected last."""
import numpy as np
import pytest

import oracle as O
from synth.inputs import random_field
from tests.gpu_util import dev64, ensure_built, host, ism, setup, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


@pytest.mark.parametrize("nx,ny,m,bc", [(160, 96, 32, (0, 0, 0, 0)), (256, 128, 16, (1, 0, 0, 1))])
def test_noalloc_matches_context_entry_point_twice(nx, ny, m, bc):
    ctx = setup(nx, ny, m, bc)
    for call, seed in enumerate((3, 11)):             # second call: new inputs, scratch reused
        p = dev64(random_field(nx, ny, seed))
        b = dev64(random_field(nx, ny, seed + 1))
        rc_ref = dev64(np.zeros((ny // m, nx // m)))
        s, rnorm, psum = ism.ism_residual_restrict(ctx, p, b, rc_ref)
        ism.check(s, "ism_residual_restrict")
        rc = torch.full_like(rc_ref, float("nan"))
        norms = torch.full((2,), float("nan"), dtype=torch.float64, device=p.device)
        s = ism.ism_residual_restrict_noalloc(nx, ny, m, bc, p, b, rc, norms)
        ism.check(s, "ism_residual_restrict_noalloc")
        torch.cuda.synchronize()
        np.testing.assert_allclose(host(rc), host(rc_ref), rtol=1e-12, atol=1e-12 * float(rc_ref.abs().max()))
        nh = host(norms)
        assert abs(nh[0] - rnorm) <= 1e-12 * rnorm, call
        assert abs(nh[1] - psum) <= 1e-12 * float(p.abs().sum()), call
        # and against the oracle's residual and block sums of the same fields
        ph, bh = host(p), host(b)
        r = O.residual(ph, bh, bc)
        ref = O.restrict(r, m)
        np.testing.assert_allclose(host(rc), ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
        assert abs(nh[0] - np.linalg.norm(r)) <= 1e-12 * np.linalg.norm(r), call


def test_noalloc_rejects_oversized_coarse_grid():
    p = torch.zeros(1, dtype=torch.float64, device="cuda:0")
    # 8192 x 4096 at 8h: 1024 x 512 coarse cells > 32768
    s = ism.ism_residual_restrict_noalloc(8192, 4096, 8, (0, 0, 0, 0), p, p, p, p)
    assert s == ism.ISM_ERR_ARG
