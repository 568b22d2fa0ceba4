"""Helpers shared by the GPU tests (no numerical method here)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1309_7128_gb300 import build as B  # noqa: E402
from paper_1309_7128_gb300 import ism  # noqa: E402

DEV = "cuda:0"


def ensure_built():
    B.build()
    ism.lib()


def dev64(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def dev32(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device=DEV)


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def setup(nx, ny, m, bc=(0, 0, 0, 0), prec=ism.ISM_FP64, h=None, **opts):
    s, ctx = ism.ism_setup(nx, ny, h if h is not None else 1.0 / nx, bc, m, prec)
    ism.check(s, "ism_setup")
    if opts:
        o = ism.ism_get_options(ctx)
        for k, v in opts.items():
            setattr(o, k, v)
        ism.check(ism.ism_set_options(ctx, o), "ism_set_options")
    return ctx


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
