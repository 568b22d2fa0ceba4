"""Pins of the oracle on grids that are not a multiple of the coarsening
factor (the last coarse cell along an axis is narrower, Sec. 3.3: padding and
interpolation rectangles of different sizes).

Each check uses an independent construction: numpy block sums, numpy linear
interpolation between the nonuniform coarse centres, dense matrices R, A_f, P
assembled here, a dense pseudo-inverse, and convergence properties.
"""
import numpy as np
import pytest

import oracle as O
from synth.inputs import random_field, smooth_rhs
from tests.conftest import ALL_BCS

RAGGED = [(70, 50, 16), (100, 36, 32), (45, 77, 8), (129, 64, 16)]


def second_difference(n, lo, hi):
    T = -2.0 * np.eye(n) + np.eye(n, k=1) + np.eye(n, k=-1)
    T[0, 0] = -1.0 if lo == 0 else -3.0
    T[-1, -1] = -1.0 if hi == 0 else -3.0
    return T


def dense_laplacian(nx, ny, bc):
    return (np.kron(np.eye(ny), second_difference(nx, bc[0], bc[1]))
            + np.kron(second_difference(ny, bc[2], bc[3]), np.eye(nx)))


def centres(n, m):
    lo = np.arange(0, n, m)
    hi = np.minimum(lo + m, n)
    return (lo + hi) / 2.0


def interp1(q, n, m, face_lo, face_hi):
    """Linear interpolation along the last axis of q from the coarse centres
    (block midpoints) to the fine centres, with ghost centres mirrored across
    the walls (even at Neumann, odd at Dirichlet-0)."""
    xc = centres(n, m)
    xe = np.concatenate([[-xc[0]], xc, [2 * n - xc[-1]]])
    x = np.arange(n) + 0.5
    out = np.empty(q.shape[:-1] + (n,))
    for idx in np.ndindex(q.shape[:-1]):
        row = q[idx]
        gl = -row[0] if face_lo == 1 else row[0]
        gh = -row[-1] if face_hi == 1 else row[-1]
        out[idx] = np.interp(x, xe, np.concatenate([[gl], row, [gh]]))
    return out


def P_dense(nx, ny, m, bc):
    ncx, ncy = O.ncoarse(nx, m), O.ncoarse(ny, m)
    P = np.zeros((nx * ny, ncx * ncy))
    for k in range(ncx * ncy):
        q = np.zeros(ncx * ncy)
        q[k] = 1.0
        a = interp1(q.reshape(ncy, ncx), nx, m, bc[0], bc[1])
        P[:, k] = np.swapaxes(interp1(np.swapaxes(a, 0, 1), ny, m, bc[2], bc[3]), 0, 1).ravel()
    return P


def R_dense(nx, ny, m):
    ncx = O.ncoarse(nx, m)
    R = np.zeros((ncx * O.ncoarse(ny, m), nx * ny))
    for j in range(ny):
        for i in range(nx):
            R[(j // m) * ncx + i // m, j * nx + i] = 1.0
    return R


@pytest.mark.parametrize("nx,ny,m", RAGGED)
def test_restriction_is_block_sum_with_narrow_last_cell(nx, ny, m):
    r = random_field(nx, ny, 1)
    want = np.add.reduceat(np.add.reduceat(r, np.arange(0, ny, m), axis=0), np.arange(0, nx, m), axis=1)
    np.testing.assert_allclose(O.restrict(r, m), want, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("nx,ny,m", RAGGED)
@pytest.mark.parametrize("bc", ALL_BCS)
def test_prolongation_is_linear_interpolation_between_block_midpoints(nx, ny, m, bc):
    q = random_field(O.ncoarse(nx, m), O.ncoarse(ny, m), 2)
    p = np.zeros((ny, nx))
    O.prolong_add(p, q, m, bc)
    a = interp1(q, nx, m, bc[0], bc[1])
    want = np.swapaxes(interp1(np.swapaxes(a, 0, 1), ny, m, bc[2], bc[3]), 0, 1)
    np.testing.assert_allclose(p, want, atol=1e-14)


def test_prolongation_reproduces_constants_and_linear_functions():
    nx, ny, m = 70, 50, 16
    xc, yc = centres(nx, m), centres(ny, m)
    f = lambda X, Y: 0.3 + 1.7 * X - 0.4 * Y
    p = np.zeros((ny, nx))
    O.prolong_add(p, f(xc[None, :], yc[:, None]), m, (0, 0, 0, 0))
    x, y = np.arange(nx) + 0.5, np.arange(ny) + 0.5
    ix = (x >= xc[0]) & (x <= xc[-1])
    iy = (y >= yc[0]) & (y <= yc[-1])
    np.testing.assert_allclose(p[np.ix_(iy, ix)], f(x[None, :], y[:, None])[np.ix_(iy, ix)], rtol=1e-13)
    p = np.zeros((ny, nx))
    O.prolong_add(p, np.ones((len(yc), len(xc))), m, (0, 0, 0, 0))
    np.testing.assert_allclose(p, 1.0, rtol=1e-14)


@pytest.mark.parametrize("nx,ny,m", [(40, 28, 8), (45, 33, 16)])
@pytest.mark.parametrize("bc", ALL_BCS)
def test_coarse_operator_equals_R_Af_P(nx, ny, m, bc):
    R = R_dense(nx, ny, m)
    A = dense_laplacian(nx, ny, bc)
    np.testing.assert_allclose(O.coarse_operator(nx, ny, m, bc, "ism"), R @ A @ P_dense(nx, ny, m, bc),
                               atol=1e-12)
    # ACM: piecewise-constant interpolant
    Pc = R.T.copy()
    np.testing.assert_allclose(O.coarse_operator(nx, ny, m, bc, "acm"), R @ A @ Pc, atol=1e-12)


def one_d(n, m, lo, hi):
    """1-D factors: W = R1 P1 and T = R1 T1 P1 (bilinear P1 with the ghost
    rule), and the ACM pair (diag of cell widths, R1 T1 R1^T)."""
    nc = O.ncoarse(n, m)
    R1 = np.zeros((nc, n))
    for i in range(n):
        R1[i // m, i] = 1.0
    P1 = interp1(np.eye(nc), n, m, lo, hi).T
    T1 = second_difference(n, lo, hi)
    return R1 @ P1, R1 @ T1 @ P1, R1 @ R1.T, R1 @ T1 @ R1.T


@pytest.mark.parametrize("nx,ny,m", RAGGED)
@pytest.mark.parametrize("bc", ALL_BCS)
def test_coarse_operator_is_a_sum_of_two_kronecker_products(nx, ny, m, bc):
    """A_c = W_y (x) T_x + T_y (x) W_x with the 1-D factors W = R P, T = R T1 P:
    the structure the GPU's separable coarse solve relies on (R, P and A_f
    are all tensor products or Kronecker sums)."""
    Wx, Tx, Wcx, Tcx = one_d(nx, m, bc[0], bc[1])
    Wy, Ty, Wcy, Tcy = one_d(ny, m, bc[2], bc[3])
    np.testing.assert_allclose(O.coarse_operator(nx, ny, m, bc, "ism"),
                               np.kron(Wy, Tx) + np.kron(Ty, Wx), atol=1e-12)
    np.testing.assert_allclose(O.coarse_operator(nx, ny, m, bc, "acm"),
                               np.kron(Wcy, Tcx) + np.kron(Tcy, Wcx), atol=1e-12)


@pytest.mark.parametrize("n,m", [(70, 16), (100, 32), (77, 8), (1000, 32), (1001, 16), (33, 32)])
@pytest.mark.parametrize("lo,hi", [(0, 0), (0, 1), (1, 1)])
def test_one_dimensional_pencils_have_real_eigenvalues(n, m, lo, hi):
    """W^-1 T has real eigenvalues in (-inf, 0] for every tested ragged
    length (a reading the GPU's setup checks again at run time: W is
    nonsymmetric when the last cell is narrower, so this is not automatic)."""
    W, T, _, _ = one_d(n, m, lo, hi)
    ev = np.linalg.eigvals(np.linalg.solve(W, T))
    assert np.abs(ev.imag).max() == 0.0
    assert ev.real.max() <= 1e-12
    assert len(np.unique(np.round(ev.real, 12))) == len(ev)


@pytest.mark.parametrize("bc", ALL_BCS)
def test_coarse_correction_annihilates_restricted_residual(bc):
    nx, ny, m = 100, 70, 16
    s = O.OracleISM(nx, ny, m, bc)
    b = s.prepare_rhs(smooth_rhs(nx, ny, 7))
    p = random_field(nx, ny, 8)
    rc = O.restrict(O.residual(p, b, bc), m)
    O.prolong_add(p, s.coarse_solve(rc), m, bc)
    after = O.restrict(O.residual(p, b, bc), m)
    assert np.abs(after).max() <= 1e-11 * np.abs(rc).max()


@pytest.mark.parametrize("bc", ALL_BCS)
@pytest.mark.parametrize("nx,ny,m", [(20, 28, 8), (18, 13, 4)])
def test_solve_matches_dense_pseudo_inverse(bc, nx, ny, m):
    b = smooth_rhs(nx, ny, 11)
    if O.is_singular(bc):
        b = b - b.mean()
    # pseudo-inverse through the symmetric eigen-decomposition (A_f is
    # symmetric; null space: constants when no face is Dirichlet)
    w, V = np.linalg.eigh(dense_laplacian(nx, ny, bc))
    ex = V @ (np.where(np.abs(w) > 1e-10, 1.0 / np.where(w == 0, 1.0, w), 0.0) * (V.T @ b.ravel()))
    p, _, _ = O.OracleISM(nx, ny, m, bc).solve(b, tol=1e-13)
    np.testing.assert_allclose(p.ravel(), ex, atol=1e-10 * np.abs(ex).max())


@pytest.mark.parametrize("bc", [(0, 0, 0, 0), (0, 1, 0, 0)])
def test_ism_converges_in_fewer_cycles_than_acm(bc):
    nx, ny, m = 200, 150, 16
    b = smooth_rhs(nx, ny, 15) + (0.0 if O.is_singular(bc) else 1e-6)
    n_ism = O.OracleISM(nx, ny, m, bc, "ism").solve(b, tol=1e-8)[1]
    n_acm = O.OracleISM(nx, ny, m, bc, "acm").solve(b, tol=1e-8)[1]
    assert n_ism < n_acm


def test_periodic_axis_must_be_a_multiple_of_m():
    with pytest.raises(ValueError):
        O.OracleISM(70, 64, 16, (2, 2, 0, 0))
    with pytest.raises(ValueError):
        O.OracleISM(70, 64, 16, (0, 0, 0, 0), kind="gmg")
