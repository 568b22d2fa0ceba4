"""C-ABI checks that need no GPU: the library loads, exports every function
declared in include/ism.h, and rejects invalid arguments before touching
the device."""
import ctypes as C

import pytest

from paper_1309_7128_gb300 import build as B
from paper_1309_7128_gb300 import ism


@pytest.fixture(scope="module")
def L():
    B.build()
    return ism.lib()


def test_every_declared_function_is_exported(L):
    names = ism.declared_functions()
    assert "ism_setup" in names and "ism_solve" in names and "proj_step" in names
    raw = C.CDLL(ism.LIB_PATH)
    for n in names:
        assert hasattr(raw, n), n


def test_status_strings(L):
    assert ism.status_str(ism.ISM_OK) == "ok"
    assert ism.status_str(ism.ISM_ERR_NOT_CONVERGED) == "not converged"
    assert ism.status_str(99) == "unknown status"


@pytest.mark.parametrize("args", [
    (12, 64, 1.0, (0, 0, 0, 0), 16),     # nx smaller than m
    (70, 64, 1.0, (2, 2, 0, 0), 16),     # periodic axis not a multiple of m
    (64, 64, 1.0, (0, 0, 0, 0), 12),     # m not in {8, 16, 32}
    (64, 64, 0.0, (0, 0, 0, 0), 16),     # h <= 0
    (64, 64, 1.0, (0, 3, 0, 0), 16),     # bad face type
    (64, 64, 1.0, (0, 2, 0, 0), 16),     # periodic east face without a periodic west face
    (64, 64, 1.0, (0, 0, 2, 1), 16),     # periodic south face, Dirichlet north face
    (48, 64, 1.0, (2, 2, 0, 0), 16),     # periodic axis with 3 coarse cells
    (64, 96, 1.0, (0, 0, 2, 2), 32),     # periodic axis with 3 coarse cells
    (96, 48, 1.0, (0, 0, 2, 2), 0),      # autotuned: no m leaves 4 coarse cells on the periodic axis
    (0, 64, 1.0, (0, 0, 0, 0), 16),      # empty grid
    (64 * 2048, 64, 1.0, (0, 0, 0, 0), 32),  # coarse grid wider than 1024
    (100, 64, 1.0, (0, 0, 0, 0), 0),     # autotuned coarsening: neither 16 nor 32 divides nx
    (64, 64, 0.0, (0, 0, 0, 0), 0),      # autotuned coarsening, h <= 0
])
def test_setup_rejects_bad_arguments(L, args):
    nx, ny, h, bc, m = args
    out = C.c_void_p(0)
    bca = (C.c_int * 4)(*bc)
    assert L.ism_setup(nx, ny, h, bca, m, 0, None, C.byref(out)) == ism.ISM_ERR_ARG
    assert out.value is None


def test_mixed_setup_needs_rows_of_whole_float4_groups(L):
    out = C.c_void_p(0)
    bca = (C.c_int * 4)(0, 0, 0, 0)
    assert L.ism_setup(102, 64, 1.0, bca, 16, 1, None, C.byref(out)) == ism.ISM_ERR_ARG
    assert out.value is None


def test_setup_rejects_bad_precision_and_null_out(L):
    bca = (C.c_int * 4)(0, 0, 0, 0)
    out = C.c_void_p(0)
    assert L.ism_setup(64, 64, 1.0, bca, 16, 7, None, C.byref(out)) == ism.ISM_ERR_ARG
    assert L.ism_setup(64, 64, 1.0, bca, 16, 0, None, None) == ism.ISM_ERR_ARG


def test_null_context_is_rejected(L):
    c, r = C.c_int(), C.c_double()
    assert L.ism_solve(None, None, None, 1e-8, 10, C.byref(c), C.byref(r)) == ism.ISM_ERR_ARG
    assert L.proj_step(None, None, None, None, 0.1, 0.1) == ism.ISM_ERR_ARG
    assert L.ism_smooth(None, None, None, 1) == ism.ISM_ERR_ARG
    assert L.ism_solve_batched(-1, None, None, None, 1e-8, 10, None, None) == ism.ISM_ERR_ARG
    d = C.c_double()
    assert L.ism_residual_norms(None, None, None, C.byref(d), C.byref(d)) == ism.ISM_ERR_ARG
    assert L.ism_last_rhs(None, C.byref(d), None) == ism.ISM_ERR_ARG


def test_every_declared_function_has_a_binding():
    """The ctypes table covers exactly the functions of include/ism.h, and each
    has a Python function of the same name (ism_destroy runs from the context
    wrapper's finaliser, ism_status_str behind status_str)."""
    declared = set(ism.declared_functions())
    assert declared == set(ism._SIGS)
    wrapped = {n for n in dir(ism) if callable(getattr(ism, n))} | {"ism_destroy", "ism_status_str"}
    assert declared <= wrapped, sorted(declared - wrapped)
