"""TEST INFRASTRUCTURE ONLY: the CPU oracle of the ISM pressure solve.

Plain, slow and sequential.  The per-cell loops live in ``ism_oracle.c``
(IEEE double, fixed loop order, no fused multiply-add); this module builds it,
wraps it with ctypes and drives the multigrid cycle in the paper's order.  The
exact coarse solve uses a dense LU factorisation from LAPACK (scipy) of the
assembled coarse operator, a library primitive standing in for the paper's
iterative coarse solve (Sec. 4: block Gauss-Seidel to a coarse tolerance).

Readings of points the paper leaves open (each one is restated where it is
used):
* cycle: correction scheme, r = b - A_f p, r_c = R r, e_c = A_c^+ r_c exactly,
  p += P e_c, then nu red-black Gauss-Seidel sweeps (no pre-smoothing), mean
  of p removed when every face is Neumann, stop on the relative L2 residual
  ||b - A_f p|| / ||b|| <= tol (the paper's accommodative cycle, Sec. 4.3.1,
  with an exact coarse solve);
* the cycle count is the number of coarse corrections applied;
* Neumann compatibility: the mean of b is removed before the solve.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg use this module.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np
import scipy.linalg

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ism_oracle.c")
_SO = os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_lib = None

VEL_NOSLIP, VEL_FREESLIP, VEL_INFLOW, VEL_OUTFLOW, VEL_PERIODIC = 0, 1, 2, 3, 4

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_fp = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle's C part in place (gcc, no fused multiply-add)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
                               "-fPIC", "-shared", "-std=c99", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            i, d = C.c_int, C.c_double
            sig = {
                "or_apply_af": [i, i, _ip, _dp, _dp],
                "or_residual": [i, i, _ip, _dp, _dp, _dp],
                "or_rbgs_sweep": [i, i, _ip, _dp, _dp],
                "or_restrict": [i, i, i, _dp, _dp],
                "or_prolong_add": [i, i, i, _ip, _dp, _dp],
                "or_prolong_const_add": [i, i, i, _dp, _dp],
                "or_coarse_operator": [i, i, i, _ip, i, _dp],
                "or_coarse_gs4": [i, i, _dp, _dp, _dp, C.c_double, i, i],
                "or_coarse_operator_coo": [i, i, i, _ip, i, _ip, _ip, _dp],
                "or_residual_f32": [i, i, _ip, _fp, _fp, _fp],
                "or_rbgs_sweep_f32": [i, i, _ip, _fp, _fp],
                "or_restrict_f32": [i, i, i, _fp, _dp],
                "or_prolong_add_f32": [i, i, i, _ip, _dp, _fp],
                "or_predictor": [i, i, d, d, d, _ip, _dp, _dp, d, _dp, _dp, _dp, _dp, _dp],
                "or_divergence": [i, i, d, d, _dp, _dp, _dp],
                "or_correct": [i, i, d, d, _ip, _dp, _dp, _dp, _dp],
                "or_set_threads": [i],
                "or_get_threads": [],
            }
            for name, args in sig.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = C.c_int if name in ("or_coarse_operator", "or_coarse_gs4", "or_set_threads",
                                                "or_get_threads") else None
            L.or_coarse_operator_coo.restype = C.c_long
            # sequential unless a caller asks for threads (set_threads): the
            # test grids are small, where thread start-up costs more than it saves
            L.or_set_threads(1)
            _lib = L
    return _lib


BC_NEUMANN, BC_DIRICHLET0, BC_PERIODIC = 0, 1, 2


def _blas_one_thread():
    """Run the OpenBLAS libraries that numpy and scipy load on one thread.
    The oracle's BLAS calls (norms, the coarse LU solve) are small; OpenBLAS
    worker threads that keep spinning between them take the cores the
    threaded row loops need (a 256^2 solve on 16 threads was 15x slower than
    on one).  Searches the loaded libraries (/proc/self/maps) for the
    OpenBLAS thread setter under the names these builds export."""
    try:
        with open("/proc/self/maps") as f:
            libs = sorted({ln.split()[-1] for ln in f if "openblas" in ln.lower() and "/" in ln})
    except OSError:
        return
    for path in libs:
        try:
            L = C.CDLL(path)
        except OSError:
            continue
        for name in ("openblas_set_num_threads", "openblas_set_num_threads64_",
                     "scipy_openblas_set_num_threads", "scipy_openblas_set_num_threads64_"):
            fn = getattr(L, name, None)
            if fn is not None:
                fn.argtypes = [C.c_int]
                fn.restype = None
                fn(1)


def set_threads(n: int) -> int:
    """Threads of the C part's row loops (n <= 0: all host cores); returns the
    count in use.  Results are bit-identical for any count.  BLAS stays on
    one thread (see _blas_one_thread)."""
    if int(n) != 1:
        import scipy.linalg  # noqa: F401  (load scipy's OpenBLAS before limiting it)
        _blas_one_thread()
    return int(lib().or_set_threads(int(n)))


def get_threads() -> int:
    return int(lib().or_get_threads())


def _faces(k):
    return np.ascontiguousarray(np.asarray(k, dtype=np.int32).reshape(4))


def _bc(bc):
    """Pressure face types (west, east, south, north): 0 Neumann,
    1 Dirichlet-0, 2 periodic (on both faces of an axis)."""
    a = _faces(bc)
    if ((a[0] == BC_PERIODIC) != (a[1] == BC_PERIODIC)) or ((a[2] == BC_PERIODIC) != (a[3] == BC_PERIODIC)):
        raise ValueError("a periodic face needs its opposite face periodic too")
    if np.any((a < 0) | (a > 2)):
        raise ValueError("face type must be 0, 1 or 2")
    return a


def ncoarse(n, m):
    """Coarse cells along an axis of n fine cells: ceil(n / m), the last one
    narrower when m does not divide n."""
    return -(-n // m)


def is_singular(bc):
    """A_f is singular (null space: constants) iff no face is Dirichlet."""
    return not np.any(_bc(bc) == BC_DIRICHLET0)


def periodic_axes(bc):
    """bit 0: x periodic, bit 1: y periodic."""
    a = _bc(bc)
    return int(a[0] == BC_PERIODIC) | (int(a[2] == BC_PERIODIC) << 1)


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# --------------------------------------------------------------------------
# thin wrappers (fields are (ny, nx) float64 arrays)
# --------------------------------------------------------------------------

def apply_af(p, bc):
    ny, nx = p.shape
    out = np.empty_like(p, dtype=np.float64)
    lib().or_apply_af(nx, ny, _bc(bc), _c64(p), out)
    return out


def residual(p, b, bc):
    ny, nx = p.shape
    r = np.empty((ny, nx), dtype=np.float64)
    lib().or_residual(nx, ny, _bc(bc), _c64(p), _c64(b), r)
    return r


def rbgs_sweep(p, b, bc):
    """One red-black Gauss-Seidel sweep in place (Sec. 3.1)."""
    ny, nx = p.shape
    assert p.dtype == np.float64 and p.flags.c_contiguous
    lib().or_rbgs_sweep(nx, ny, _bc(bc), p, _c64(b))


def restrict(r, m):
    ny, nx = r.shape
    rc = np.empty((ncoarse(ny, m), ncoarse(nx, m)), dtype=np.float64)
    lib().or_restrict(nx, ny, m, _c64(r), rc)
    return rc


def prolong_add(p, q, m, bc):
    ny, nx = p.shape
    assert p.dtype == np.float64 and p.flags.c_contiguous
    lib().or_prolong_add(nx, ny, m, _bc(bc), _c64(q), p)


def prolong_const_add(p, q, m):
    ny, nx = p.shape
    assert p.dtype == np.float64 and p.flags.c_contiguous
    lib().or_prolong_const_add(nx, ny, m, _c64(q), p)


def coarse_operator(nx, ny, m, bc, kind="ism"):
    """Dense coarse operator A_c; kind 'ism' (face-flux sums of the bilinear
    interpolant, Sec. 3.3, Eq. 5-7), 'acm' (face-flux sums of the piecewise
    constant interpolant, Sec. 3.2) or 'gmg' (the five-point operator
    re-discretised on the coarse grid, the comparator of Sec. 3.3 / Table 5:
    the fine operator's rule applied to coarse cells)."""
    nc = ncoarse(nx, m) * ncoarse(ny, m)
    if kind == "gmg":
        if nx % m or ny % m:
            raise ValueError("the re-discretised coarse operator needs uniform coarse cells")
        ncx, ncy = nx // m, ny // m
        eye = np.eye(nc)
        Ac = np.empty((nc, nc), dtype=np.float64)
        for k in range(nc):
            Ac[:, k] = apply_af(eye[k].reshape(ncy, ncx), bc).ravel()
        return Ac
    Ac = np.empty((nc, nc), dtype=np.float64)
    rc = lib().or_coarse_operator(nx, ny, m, _bc(bc), 0 if kind == "ism" else 1, Ac)
    if rc != 0:
        raise MemoryError("oracle coarse operator allocation failed")
    return Ac


def coarse_operator_sparse(nx, ny, m, bc, kind="ism"):
    """The coarse operator of kind 'ism' or 'acm' as a scipy CSR matrix,
    assembled column by column with the same face-flux sums as
    coarse_operator (walls only: no periodic face).  For coarse grids too
    large for a dense matrix."""
    import scipy.sparse
    if kind not in ("ism", "acm"):
        raise ValueError("sparse assembly: kinds 'ism' and 'acm'")
    nc = ncoarse(nx, m) * ncoarse(ny, m)
    rows = np.empty(9 * nc, dtype=np.int32)
    cols = np.empty(9 * nc, dtype=np.int32)
    vals = np.empty(9 * nc, dtype=np.float64)
    got = lib().or_coarse_operator_coo(nx, ny, m, _bc(bc), 0 if kind == "ism" else 1, rows, cols, vals)
    if got < 0:
        raise ValueError("sparse assembly failed (periodic face or allocation)")
    keep = rows >= 0
    return scipy.sparse.csr_matrix((vals[keep], (rows[keep], cols[keep])), shape=(nc, nc))


# --------------------------------------------------------------------------
# the two-level solver
# --------------------------------------------------------------------------

class OracleISM:
    """Two-level ISM (kind='ism'), ACM (kind='acm') or GMG (kind='gmg',
    re-discretised five-point coarse operator with the bilinear correction)
    solver.

    Sec. 3.3-3.4: aggressive m x m coarsening (16h / 32h), interpolated
    nine-point coarse stencil (ISM) or summed five-point coarse equations with
    piecewise-constant correction (ACM), red-black Gauss-Seidel smoothing.
    """

    # coarse grids above this many cells are factorised as sparse matrices
    SPARSE_ABOVE = 4096

    def __init__(self, nx, ny, m, bc=(0, 0, 0, 0), kind="ism", nu=8, coarse="auto"):
        if kind == "gmg" and (nx % m or ny % m):
            raise ValueError("the GMG comparator needs a grid that is a multiple of the coarsening factor")
        bca = _bc(bc)
        if (bca[0] == BC_PERIODIC and nx % m) or (bca[2] == BC_PERIODIC and ny % m):
            raise ValueError("a periodic axis must be a multiple of the coarsening factor")
        self.nx, self.ny, self.m = nx, ny, m
        self.bc = _bc(bc)
        self.kind = kind
        self.nu = nu
        self.singular = is_singular(self.bc)
        nc = ncoarse(nx, m) * ncoarse(ny, m)
        if coarse == "auto":
            coarse = "sparse" if (nc > self.SPARSE_ABOVE and kind in ("ism", "acm")
                                  and not np.any(bca == BC_PERIODIC)) else "dense"
        self.coarse = coarse
        if coarse == "sparse":
            self._setup_sparse(nc)
            return
        self.Ac = coarse_operator(nx, ny, m, self.bc, kind)
        M = -self.Ac
        if self.singular:
            # all-Neumann: A_c 1 = 0.  (-A_c + 1 1^T / nc) is nonsingular and,
            # for a right-hand side with zero sum, returns minus the mean-free
            # solution of A_c e = r_c.
            M = M + np.full((nc, nc), 1.0 / nc)
        self._lu = scipy.linalg.lu_factor(M, check_finite=False)

    def _setup_sparse(self, nc):
        """Sparse LU (SuperLU, a library routine) of -A_c; with all faces
        Neumann of the bordered matrix [[-A_c, 1], [1^T, 0]], whose solution
        for a zero-sum right-hand side is minus the mean-free solution of
        A_c e = r_c (the Lagrange multiplier is then 0)."""
        import scipy.sparse
        import scipy.sparse.linalg
        self.Ac = coarse_operator_sparse(self.nx, self.ny, self.m, self.bc, self.kind)
        M = -self.Ac
        if self.singular:
            one = scipy.sparse.csr_matrix(np.ones((nc, 1)))
            M = scipy.sparse.bmat([[M, one], [one.T, None]], format="csr")
        self._splu = scipy.sparse.linalg.splu(M.tocsc())
        self._nc = nc

    # e_c = A_c^+ r_c (exact coarse solve)
    def coarse_solve(self, rc):
        if self.coarse == "sparse":
            rhs = rc.reshape(-1)
            if self.singular:
                rhs = np.concatenate([rhs, [0.0]])
            x = self._splu.solve(rhs)[: self._nc]
            return (-x).reshape(rc.shape)
        x = scipy.linalg.lu_solve(self._lu, rc.reshape(-1), check_finite=False)
        return (-x).reshape(rc.shape)

    def _correct(self, p, ec):
        if self.kind != "acm":
            prolong_add(p, ec, self.m, self.bc)
        else:
            prolong_const_add(p, ec, self.m)

    def cycle(self, p, b):
        """One cycle (reading: correction scheme, exact coarse solve, then nu
        post-smoothing sweeps, no pre-smoothing; mean of p removed when all
        faces are Neumann)."""
        r = residual(p, b, self.bc)
        rc = restrict(r, self.m)
        ec = self.coarse_solve(rc)
        self._correct(p, ec)
        for _ in range(self.nu):
            rbgs_sweep(p, b, self.bc)
        if self.singular:
            p -= p.mean()

    def prepare_rhs(self, b):
        b = np.array(b, dtype=np.float64, order="C", copy=True)
        if self.singular:
            b -= b.mean()
        return b

    def solve(self, b, p0=None, tol=1e-8, max_cycles=10000):
        """FP64 solve.  Returns (p, cycles, relres_history)."""
        b = self.prepare_rhs(b)
        p = np.zeros_like(b) if p0 is None else np.array(p0, dtype=np.float64, order="C", copy=True)
        if self.singular:
            p -= p.mean()
        bn = np.linalg.norm(b)
        if bn == 0.0:
            return np.zeros_like(b), 0, [0.0]
        hist = [np.linalg.norm(residual(p, b, self.bc)) / bn]
        cycles = 0
        while hist[-1] > tol and cycles < max_cycles:
            self.cycle(p, b)
            cycles += 1
            hist.append(np.linalg.norm(residual(p, b, self.bc)) / bn)
        return p, cycles, hist

    # ---------------- mixed precision (emulated single-precision inner) ----

    def inner_cycle_f32(self, e, r32):
        """One inner cycle on A_f e = r32 with float loops; the exact coarse
        solve runs in double and is rounded to float by the prolongation."""
        L = lib()
        nx, ny, m = self.nx, self.ny, self.m
        rin = np.empty_like(e)
        L.or_residual_f32(nx, ny, self.bc, e, r32, rin)
        rc = np.empty((ncoarse(ny, m), ncoarse(nx, m)), dtype=np.float64)
        L.or_restrict_f32(nx, ny, m, rin, rc)
        ec = self.coarse_solve(rc)
        L.or_prolong_add_f32(nx, ny, m, self.bc, np.ascontiguousarray(ec), e)
        for _ in range(self.nu):
            L.or_rbgs_sweep_f32(nx, ny, self.bc, e, r32)
        if self.singular:
            e -= np.float32(e.astype(np.float64).mean())

    def inner_residual_norm_f32(self, e, r32):
        rin = np.empty_like(e)
        lib().or_residual_f32(self.nx, self.ny, self.bc, e, r32, rin)
        return float(np.linalg.norm(rin.astype(np.float64)))

    # Single-precision rounding floor of the inner residual: every Gauss-Seidel
    # update rounds e to float (relative error up to 2^-24), and the five-point
    # stencil maps that noise to a residual of about 1.5e-7 ||e||.  The inner
    # solve stops once it is within FLOOR_MULT * 2^-23 ||e|| of that floor.
    FLOOR_UNIT = 2.0 ** -23
    FLOOR_MULT = 4.0

    def solve_mixed(self, b, p0=None, tol=1e-8, max_outer=50, inner_tol=1e-3,
                    inner_max=10000):
        """FP64 iterative refinement around single-precision inner cycles.

        Outer step (FP64): r = b - A_f p, relres = ||r|| / ||b||.  Inner solve
        (float): cycles on A_f e = r (e_0 = 0) until the float residual is
        below max(inner_tol ||r||, FLOOR_MULT 2^-23 ||e||) or ``inner_max``
        cycles.  Then p += e (FP64) and the mean of p is removed (all-Neumann).
        Returns (p, outer_iterations, inner_cycles_total, relres_history).
        """
        b = self.prepare_rhs(b)
        p = np.zeros_like(b) if p0 is None else np.array(p0, dtype=np.float64, order="C", copy=True)
        if self.singular:
            p -= p.mean()
        bn = np.linalg.norm(b)
        if bn == 0.0:
            return np.zeros_like(b), 0, 0, [0.0]
        r = residual(p, b, self.bc)
        hist = [np.linalg.norm(r) / bn]
        outer = inner_total = 0
        while hist[-1] > tol and outer < max_outer:
            r32 = np.ascontiguousarray(r, dtype=np.float32)
            r32n = float(np.linalg.norm(r32.astype(np.float64)))
            e = np.zeros_like(r32)
            for _ in range(inner_max):
                self.inner_cycle_f32(e, r32)
                inner_total += 1
                en = float(np.linalg.norm(e.astype(np.float64)))
                lim = max(inner_tol * r32n, self.FLOOR_MULT * self.FLOOR_UNIT * en)
                if self.inner_residual_norm_f32(e, r32) <= lim:
                    break
            p += e.astype(np.float64)
            if self.singular:
                p -= p.mean()
            outer += 1
            r = residual(p, b, self.bc)
            hist.append(np.linalg.norm(r) / bn)
        return p, outer, inner_total, hist


class OracleACMV:
    """The additive correction multigrid of Sec. 3.2 as a deep V-cycle (the
    paper's comparator, Sec. 4.3): coarse equations are sums of 2 x 2 blocks
    of the finer equations (agglomeration), the correction is piecewise
    constant, levels go from h down to the coarsening factor m = 2^L.

    Cycle (reading: correction scheme, no pre-smoothing, one post-smoothing
    sweep per intermediate level, exact solve at the coarsest level):
    r_0 = b - A_f p; r_{l+1} = R_2 r_l; e_L = A_L^+ r_L;
    for l = L-1 .. 1: e_l = P_2 e_{l+1}, one red-black sweep on A_l e_l = r_l;
    p += P_2 e_1; nu sweeps on A_f p = b; mean of p removed when all faces
    are Neumann.  A_l = 2^l x (five-point operator of level l) (the
    agglomerated operator), so a sweep on level l is a five-point sweep with
    right-hand side r_l / 2^l."""

    def __init__(self, nx, ny, m, bc=(0, 0, 0, 0), nu=8):
        if nx % m or ny % m or m & (m - 1) or m < 2:
            raise ValueError("m must be a power of two dividing the grid")
        self.nx, self.ny, self.m, self.nu = nx, ny, m, nu
        self.L = m.bit_length() - 1
        self.bc = _bc(bc)
        self.singular = is_singular(self.bc)
        self.top = OracleISM(nx, ny, m, bc, kind="acm", nu=nu)     # exact level-L solve of A_L = m x five-point

    def cycle(self, p, b):
        r = residual(p, b, self.bc)
        rs = [r]
        for _ in range(self.L):
            rs.append(restrict(rs[-1], 2))
        e = self.top.coarse_solve(rs[self.L])
        for lev in range(self.L - 1, 0, -1):
            el = np.zeros_like(rs[lev])
            prolong_const_add(el, e, 2)
            rbgs_sweep(el, rs[lev] / float(2 ** lev), self.bc)
            e = el
        prolong_const_add(p, e, 2)
        for _ in range(self.nu):
            rbgs_sweep(p, b, self.bc)
        if self.singular:
            p -= p.mean()

    def solve(self, b, p0=None, tol=1e-8, max_cycles=10000):
        """FP64 solve.  Returns (p, cycles, relres_history)."""
        b = self.top.prepare_rhs(b)
        p = np.zeros_like(b) if p0 is None else np.array(p0, dtype=np.float64, order="C", copy=True)
        if self.singular:
            p -= p.mean()
        bn = np.linalg.norm(b)
        if bn == 0.0:
            return np.zeros_like(b), 0, [0.0]
        hist = [np.linalg.norm(residual(p, b, self.bc)) / bn]
        cycles = 0
        while hist[-1] > tol and cycles < max_cycles:
            self.cycle(p, b)
            cycles += 1
            hist.append(np.linalg.norm(residual(p, b, self.bc)) / bn)
        return p, cycles, hist


class OracleAccommodative:
    """The paper's accommodative strategy for one pressure solve (Sec. 4.3.1),
    in its simplest form: iterate on the coarse grid first, prolongate when
    the coarse residual is small enough, then iterate on the fine grid until
    the fine criterion holds.  Readings: the coarse equations are the ISM
    equations A_c e = R r (sums of fine equations) solved by four-colour
    Gauss-Seidel from e = 0 until max |R r - A_c e| <= tol_c; the correction
    is bilinear (Eq. 5); the fine iteration is red-black Gauss-Seidel until
    max |b - A_f p| <= tol_f; both criteria are absolute maximum norms (the
    paper's 1e-6 with h = 1); one coarse-then-fine pass per solve."""

    def __init__(self, nx, ny, m, bc=(0, 0, 0, 0)):
        self.nx, self.ny, self.m = nx, ny, m
        self.bc = _bc(bc)
        self.singular = is_singular(self.bc)
        self.Ac = np.ascontiguousarray(coarse_operator(nx, ny, m, self.bc, "ism"))

    def solve(self, b, p0=None, tol_f=1e-6, tol_c=1e-5, cap_c=100000, cap_f=1000000):
        """Returns (p, coarse iterations, fine sweeps, final max |r|)."""
        b = np.array(b, dtype=np.float64, order="C", copy=True)
        if self.singular:
            b -= b.mean()
        p = np.zeros_like(b) if p0 is None else np.array(p0, dtype=np.float64, order="C", copy=True)
        if self.singular:
            p -= p.mean()
        r = residual(p, b, self.bc)
        if np.abs(r).max() <= tol_f:
            return p, 0, 0, float(np.abs(r).max())
        rc = np.ascontiguousarray(restrict(r, self.m))
        ec = np.zeros_like(rc)
        nc_it = lib().or_coarse_gs4(rc.shape[1], rc.shape[0], self.Ac, rc, ec, float(tol_c), int(cap_c),
                                    periodic_axes(self.bc))
        prolong_add(p, ec, self.m, self.bc)
        if self.singular:
            p -= p.mean()
        nf = 0
        mx = float(np.abs(residual(p, b, self.bc)).max())
        while mx > tol_f and nf < cap_f:
            rbgs_sweep(p, b, self.bc)
            nf += 1
            mx = float(np.abs(residual(p, b, self.bc)).max())
        if self.singular:
            p -= p.mean()
        return p, nc_it, nf, mx


# --------------------------------------------------------------------------
# projection time step (Sec. 2.2-2.3, Eq. 3-4)
# --------------------------------------------------------------------------

def predictor(u, v, p, h, dt, nu, vel_bc, wall_u=(0, 0, 0, 0), u_in=None, conv_u=1.0):
    ny, nx = p.shape
    us = np.empty((ny, nx + 1)); vs = np.empty((ny + 1, nx))
    uin = np.zeros(ny) if u_in is None else _c64(u_in)
    lib().or_predictor(nx, ny, h, dt, nu, _faces(vel_bc), _c64(np.asarray(wall_u, float)),
                       uin, conv_u, _c64(u), _c64(v), _c64(p), us, vs)
    return us, vs


def divergence(u, v, h, dt):
    ny, nx = v.shape[0] - 1, u.shape[1] - 1
    b = np.empty((ny, nx))
    lib().or_divergence(nx, ny, h, dt, _c64(u), _c64(v), b)
    return b


def correct(u, v, p, dp, h, dt, vel_bc):
    ny, nx = p.shape
    for a in (u, v, p):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    lib().or_correct(nx, ny, h, dt, _faces(vel_bc), _c64(dp), u, v, p)


def pressure_bc(vel_bc):
    """Dirichlet-0 pressure on outflow faces, periodic on periodic faces,
    Neumann elsewhere."""
    return tuple(1 if k == VEL_OUTFLOW else (BC_PERIODIC if k == VEL_PERIODIC else 0) for k in vel_bc)


def proj_step(u, v, p, h, dt, nu, vel_bc, solver: OracleISM, wall_u=(0, 0, 0, 0),
              u_in=None, conv_u=1.0, tol=1e-8, max_cycles=10000, dp0=None):
    """One Goda incremental pressure-correction step (Sec. 2.2) in place on
    (u, v, p).  Returns (dp, cycles, relres_history)."""
    us, vs = predictor(u, v, p, h, dt, nu, vel_bc, wall_u, u_in, conv_u)
    b = divergence(us, vs, h, dt)
    dp, cycles, hist = solver.solve(b, p0=dp0, tol=tol, max_cycles=max_cycles)
    u[...] = us
    v[...] = vs
    correct(u, v, p, dp, h, dt, vel_bc)
    return dp, cycles, hist
