"""Thin Python binding of the ISM C ABI (include/ism.h).

Argument marshalling only: torch tensors become device pointers, the current
torch CUDA stream becomes the context's ordering stream, and status codes
become return values (or exceptions via ``check``).  Every numerical step
runs in the CUDA library; when ``libism.so`` is missing the binding raises
instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os
import re
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libism.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "ism.h")

ISM_OK, ISM_ERR_ARG, ISM_ERR_NOT_CONVERGED, ISM_ERR_NONFINITE, ISM_ERR_CUDA, ISM_ERR_NOMEM = range(6)
ISM_BC_NEUMANN, ISM_BC_DIRICHLET0, ISM_BC_PERIODIC = 0, 1, 2
ISM_FP64, ISM_MIXED = 0, 1
ISM_COARSE_ISM, ISM_COARSE_ACM, ISM_COARSE_GMG, ISM_COARSE_ACMV = 0, 1, 2, 3
ISM_VEL_NOSLIP, ISM_VEL_FREESLIP, ISM_VEL_INFLOW, ISM_VEL_OUTFLOW, ISM_VEL_PERIODIC = 0, 1, 2, 3, 4


class IsmOptions(C.Structure):
    _fields_ = [("nu", C.c_int), ("sweeps_per_pass", C.c_int), ("kind", C.c_int),
                ("max_outer", C.c_int), ("inner_max", C.c_int), ("inner_tol", C.c_double),
                ("floor_mult", C.c_double), ("check_every", C.c_int), ("use_graphs", C.c_int),
                ("coarse_tc", C.c_int), ("cycle", C.c_int), ("accom_tol_c", C.c_double),
                ("accom_max_coarse", C.c_int),
                ("stream", C.c_int), ("fault_test", C.c_int), ("tile_rows", C.c_int), ("packed", C.c_int)]


class IsmError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {status_str(status)} ({status})")


_lock = threading.Lock()
_lib = None

_VP, _I, _D = C.c_void_p, C.c_int, C.c_double
_SIGS = {
    "ism_status_str": (C.c_char_p, [_I]),
    "ism_setup": (_I, [_I, _I, _D, C.POINTER(C.c_int), _I, _I, _VP, C.POINTER(_VP)]),
    "ism_destroy": (None, [_VP]),
    "ism_get_options": (_I, [_VP, C.POINTER(IsmOptions)]),
    "ism_set_options": (_I, [_VP, C.POINTER(IsmOptions)]),
    "ism_solve": (_I, [_VP, _VP, _VP, _D, _I, C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    "ism_last_history": (_I, [_VP, C.POINTER(C.c_double), _I]),
    "ism_last_counts": (_I, [_VP, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_longlong)]),
    "ism_smooth": (_I, [_VP, _VP, _VP, _I]),
    "ism_residual_restrict": (_I, [_VP, _VP, _VP, _VP, C.POINTER(C.c_double)]),
    "ism_residual_norms": (_I, [_VP, _VP, _VP, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "ism_last_rhs": (_I, [_VP, C.POINTER(C.c_double), C.POINTER(C.c_int)]),
    "ism_coarse_solve": (_I, [_VP, _VP, _VP]),
    "ism_prolong_add": (_I, [_VP, _VP, _VP]),
    "ism_set_flow": (_I, [_VP, C.POINTER(C.c_int), C.POINTER(C.c_double), _VP, _D]),
    "proj_step": (_I, [_VP, _VP, _VP, _VP, _D, _D]),
    "ism_proj_tol": (_I, [_VP, _D, _I, _I]),
    "ism_last_dp": (_VP, [_VP]),
    "ism_last_b": (_VP, [_VP]),
    "ism_set_warm_start": (_I, [_VP, _VP]),
    "ism_time_pass": (_I, [_VP, _VP, _VP, _I, _I, C.POINTER(C.c_double)]),
    "ism_time_restrict": (_I, [_VP, _VP, _VP, _VP, _I, C.POINTER(C.c_double)]),
    "ism_time_coarse": (_I, [_VP, _VP, _VP, _I, C.POINTER(C.c_double)]),
    "ism_autotune": (_I, [_VP, _VP, _D, _I, C.POINTER(IsmOptions)]),
    "ism_autotune_from": (_I, [_VP, _VP, _VP, _D, _I, C.POINTER(IsmOptions)]),
    "ism_residual_restrict_noalloc": (_I, [_I, _I, _I, C.POINTER(C.c_int), _VP, _VP, _VP, _VP, _VP]),
    "ism_solve_batched": (_I, [_I, C.POINTER(_VP), C.POINTER(_VP), C.POINTER(_VP), _D, _I,
                               C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    "ism_coarsening": (_I, [_VP]),
    "ism_autotune_batched": (_I, [_I, C.POINTER(_VP), C.POINTER(_VP), C.POINTER(_VP), _D, C.POINTER(C.c_int)]),
    "proj_step_adjoint": (_I, [_VP, _VP, _VP, _D, _D, _VP, _VP, _VP]),
    "ism_enstrophy": (_I, [_VP, _VP, _VP, C.POINTER(C.c_double), _VP, _VP]),
    "proj_rollout_grad": (_I, [_VP, _VP, _VP, _VP, _D, _D, _I, _I, C.POINTER(C.c_double),
                               _VP, _VP, _VP]),
}


def declared_functions(header: str = HEADER):
    """Names of the functions declared in include/ism.h."""
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b([a-z_][a-z0-9_]*)\s*\(", text)) - {"defined"})


def lib():
    """Load libism.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"ISM CUDA library not built ({LIB_PATH}); "
                                   "run __graft_entry__.build() or python -m paper_1309_7128_gb300.build")
            L = C.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def status_str(s: int) -> str:
    return lib().ism_status_str(int(s)).decode()


def check(status: int, where: str = "ism", ok=(ISM_OK,)):
    if status not in ok:
        raise IsmError(status, where)
    return status


def _ptr(t):
    return C.c_void_p(0 if t is None else t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return C.c_void_p(int(stream))


class Ctx:
    """Owning handle of an ism_ctx."""

    def __init__(self, handle, nx, ny, m, prec):
        self.handle = handle
        self.nx, self.ny, self.m, self.prec = nx, ny, m, prec

    def __del__(self):
        h, self.handle = getattr(self, "handle", None), None
        if h and _lib is not None:
            _lib.ism_destroy(h)

    @property
    def _as_parameter_(self):
        return self.handle


def ism_setup(nx, ny, h, bc, coarsen, prec=ISM_FP64, stream=None):
    """Returns (status, Ctx or None)."""
    L = lib()
    bca = (C.c_int * 4)(*[int(x) for x in bc])
    out = C.c_void_p()
    s = L.ism_setup(int(nx), int(ny), float(h), bca, int(coarsen), int(prec),
                    _stream(stream) if stream is not False else C.c_void_p(0), C.byref(out))
    if s != ISM_OK:
        return s, None
    return s, Ctx(out.value, nx, ny, L.ism_coarsening(out), prec)


def ism_get_options(ctx):
    o = IsmOptions()
    check(lib().ism_get_options(ctx.handle, C.byref(o)), "ism_get_options")
    return o


def ism_set_options(ctx, opt):
    return lib().ism_set_options(ctx.handle, C.byref(opt))


def ism_solve(ctx, rhs, p, tol=1e-8, max_cycles=100000):
    """Returns (status, cycles, relres)."""
    c = C.c_int(0)
    r = C.c_double(0.0)
    s = lib().ism_solve(ctx.handle, _ptr(rhs), _ptr(p), float(tol), int(max_cycles), C.byref(c), C.byref(r))
    return s, c.value, r.value


def ism_autotune(ctx, rhs, tol=1e-8, max_cycles=100000):
    """Returns (status, chosen IsmOptions)."""
    o = IsmOptions()
    s = lib().ism_autotune(ctx.handle, _ptr(rhs), float(tol), int(max_cycles), C.byref(o))
    return s, o


def ism_autotune_from(ctx, rhs, p0, tol=1e-8, max_cycles=100000):
    """ism_autotune with every timed solve started from p0 (device, or None
    for zero).  Returns (status, chosen IsmOptions)."""
    o = IsmOptions()
    s = lib().ism_autotune_from(ctx.handle, _ptr(rhs), _ptr(p0) if p0 is not None else None, float(tol),
                                int(max_cycles), C.byref(o))
    return s, o


def ism_last_history(ctx, cap=4096):
    buf = (C.c_double * cap)()
    n = lib().ism_last_history(ctx.handle, buf, cap)
    return list(buf[:n])


def ism_last_counts(ctx):
    o, c, l = C.c_int(), C.c_int(), C.c_longlong()
    check(lib().ism_last_counts(ctx.handle, C.byref(o), C.byref(c), C.byref(l)), "ism_last_counts")
    return o.value, c.value, l.value


def ism_smooth(ctx, p, b, sweeps):
    return lib().ism_smooth(ctx.handle, _ptr(p), _ptr(b), int(sweeps))


def ism_residual_restrict(ctx, p, b, rc):
    norms = (C.c_double * 2)()
    s = lib().ism_residual_restrict(ctx.handle, _ptr(p), _ptr(b), _ptr(rc), norms)
    return s, norms[0], norms[1]


def ism_residual_restrict_noalloc(nx, ny, coarsen, bc, p, b, rc, norms, stream=None):
    """Context-free FP64 residual + restriction; norms is a device tensor of
    2 doubles.  Returns the status."""
    bca = (C.c_int * 4)(*[int(x) for x in bc])
    return lib().ism_residual_restrict_noalloc(int(nx), int(ny), int(coarsen), bca, _ptr(p), _ptr(b),
                                               _ptr(rc), _ptr(norms), _stream(stream))


def ism_time_restrict(ctx, p, b, rc, reps):
    """Returns (status, mean device microseconds per residual + restriction pass)."""
    us = C.c_double(0.0)
    s = lib().ism_time_restrict(ctx.handle, _ptr(p), _ptr(b), _ptr(rc), int(reps), C.byref(us))
    return s, us.value


def ism_time_coarse(ctx, rc, ec, reps):
    """Returns (status, mean device microseconds per exact coarse solve)."""
    us = C.c_double(0.0)
    s = lib().ism_time_coarse(ctx.handle, _ptr(rc), _ptr(ec), int(reps), C.byref(us))
    return s, us.value


def ism_time_pass(ctx, p, b, sweeps, reps):
    """Returns (status, mean device microseconds per smoothing pass)."""
    us = C.c_double(0.0)
    s = lib().ism_time_pass(ctx.handle, _ptr(p), _ptr(b), int(sweeps), int(reps), C.byref(us))
    return s, us.value


def ism_residual_norms(ctx, rhs, p):
    """Returns (status, ||rhs - A_f p||_2, max |rhs - A_f p|) for FP64 device tensors."""
    l2 = C.c_double(0.0)
    mx = C.c_double(0.0)
    s = lib().ism_residual_norms(ctx.handle, _ptr(rhs), _ptr(p), C.byref(l2), C.byref(mx))
    return s, l2.value, mx.value


def ism_last_rhs(ctx):
    """Returns (status, mean removed from the last right-hand side, incompatible flag)."""
    mu = C.c_double(0.0)
    flag = C.c_int(0)
    s = lib().ism_last_rhs(ctx.handle, C.byref(mu), C.byref(flag))
    return s, mu.value, bool(flag.value)


def ism_coarse_solve(ctx, rc, ec):
    return lib().ism_coarse_solve(ctx.handle, _ptr(rc), _ptr(ec))


def ism_prolong_add(ctx, ec, p):
    return lib().ism_prolong_add(ctx.handle, _ptr(ec), _ptr(p))


def ism_set_flow(ctx, vel_bc, wall_u=(0.0, 0.0, 0.0, 0.0), u_in=None, conv_u=1.0):
    vb = (C.c_int * 4)(*[int(x) for x in vel_bc])
    wu = (C.c_double * 4)(*[float(x) for x in wall_u])
    return lib().ism_set_flow(ctx.handle, vb, wu, _ptr(u_in), float(conv_u))


def ism_proj_tol(ctx, tol=1e-8, max_cycles=100000, warm_start=False):
    return lib().ism_proj_tol(ctx.handle, float(tol), int(max_cycles), int(bool(warm_start)))


def proj_step(ctx, u, v, p, dt, nu):
    return lib().proj_step(ctx.handle, _ptr(u), _ptr(v), _ptr(p), float(dt), float(nu))


def ism_last_dp(ctx):
    """Device address of the context's last pressure increment (nx*ny doubles)."""
    return lib().ism_last_dp(ctx.handle)


def ism_set_warm_start(ctx, dp0):
    """Next warm-started proj_step starts from dp0 (device, nx*ny doubles)."""
    return lib().ism_set_warm_start(ctx.handle, _ptr(dp0))


def device_view(ptr, shape, dtype="float64"):
    """A torch tensor aliasing library-owned device memory (ism_last_dp,
    ism_last_b): no copy; valid until the next call on the owning context."""
    import torch

    class _Arr:
        __cuda_array_interface__ = {"shape": tuple(shape), "typestr": {"float64": "<f8", "float32": "<f4"}[dtype],
                                    "data": (int(ptr), False), "version": 3, "strides": None}
    return torch.as_tensor(_Arr(), device="cuda")


def ism_last_b(ctx):
    """Device address of the right-hand side of the context's last pressure
    solve (nx*ny doubles, mean removed when all faces are Neumann)."""
    return lib().ism_last_b(ctx.handle)


def ism_solve_batched(ctxs, rhs, p, tol=1e-8, max_cycles=100000):
    """Returns (status, cycles list, relres list)."""
    n = len(ctxs)
    ca = (C.c_void_p * n)(*[c.handle for c in ctxs])
    ra = (C.c_void_p * n)(*[t.data_ptr() for t in rhs])
    pa = (C.c_void_p * n)(*[t.data_ptr() for t in p])
    cyc = (C.c_int * n)()
    rel = (C.c_double * n)()
    s = lib().ism_solve_batched(n, ca, ra, pa, float(tol), int(max_cycles), cyc, rel)
    return s, list(cyc), list(rel)


def proj_step_adjoint(ctx, u, v, dt, nu, gu, gv, gp):
    """Overwrite (gu, gv, gp), the adjoints of one step's outputs, with the
    adjoints of its inputs; (u, v) are the step's input velocities."""
    return lib().proj_step_adjoint(ctx.handle, _ptr(u), _ptr(v), float(dt), float(nu),
                                   _ptr(gu), _ptr(gv), _ptr(gp))


def ism_enstrophy(ctx, u, v, gu=None, gv=None):
    """Returns (status, enstrophy); gu, gv (optional) receive its gradient."""
    val = C.c_double(0.0)
    s = lib().ism_enstrophy(ctx.handle, _ptr(u), _ptr(v), C.byref(val), _ptr(gu), _ptr(gv))
    return s, val.value


def proj_rollout_grad(ctx, u0, v0, p0, dt, nu, steps, every=20, gu=None, gv=None, gp=None):
    """Returns (status, loss); with gu, gv, gp given they receive the gradient
    of the final enstrophy with respect to (u0, v0, p0)."""
    val = C.c_double(0.0)
    s = lib().proj_rollout_grad(ctx.handle, _ptr(u0), _ptr(v0), _ptr(p0), float(dt), float(nu),
                                int(steps), int(every), C.byref(val), _ptr(gu), _ptr(gv), _ptr(gp))
    return s, val.value


def ism_coarsening(ctx):
    """Coarsening factor m of the context (as chosen by ism_setup)."""
    return lib().ism_coarsening(ctx.handle)


def ism_autotune_batched(ctxs, rhs, p, tol=1e-8):
    """Returns (status, nu chosen for the ensemble)."""
    n = len(ctxs)
    ca = (C.c_void_p * n)(*[c.handle for c in ctxs])
    ra = (C.c_void_p * n)(*[t.data_ptr() for t in rhs])
    pa = (C.c_void_p * n)(*[t.data_ptr() for t in p])
    nu = C.c_int(0)
    s = lib().ism_autotune_batched(n, ca, ra, pa, float(tol), C.byref(nu))
    return s, nu.value
