"""Pins of the oracle's periodic faces (face type 2 on both faces of an axis).

Each check is against something other than the oracle itself: a circulant
(np.roll) Laplacian, the discrete Fourier diagonalisation of the periodic
five-point operator, numpy's periodic linear interpolation, a closed form of
the coarse operator with circulant factors, a dense Gauss-Seidel written from
the matrix, and translation invariance of one cycle.
"""
import numpy as np
import pytest

import oracle as O
from synth.inputs import random_field, smooth_rhs
from tests.conftest import PERIODIC_BCS


def second_difference(n, lo, hi):
    """1-D cell-centred second difference: circulant on a periodic axis,
    otherwise end diagonal -1 (Neumann) or -3 (Dirichlet-0)."""
    T = -2.0 * np.eye(n) + np.eye(n, k=1) + np.eye(n, k=-1)
    if lo == 2:
        T[0, -1] += 1.0
        T[-1, 0] += 1.0
    else:
        T[0, 0] = -1.0 if lo == 0 else -3.0
        T[-1, -1] = -1.0 if hi == 0 else -3.0
    return T


def dense_laplacian(nx, ny, bc):
    return (np.kron(np.eye(ny), second_difference(nx, bc[0], bc[1]))
            + np.kron(second_difference(ny, bc[2], bc[3]), np.eye(nx)))


def S1(n, lo, hi):
    """1-D factor of the ISM coarse operator: tridiag(1, 2, 1), circulant on
    a periodic axis, else end diagonal 3 (Neumann) or 1 (Dirichlet-0)."""
    return second_difference(n, lo, hi) + 4.0 * np.eye(n)


def test_face_type_validation():
    with pytest.raises(ValueError):
        O.OracleISM(64, 64, 16, (2, 0, 0, 0))
    with pytest.raises(ValueError):
        O.OracleISM(64, 64, 16, (0, 0, 0, 2))
    assert O.is_singular((2, 2, 0, 0)) and O.is_singular((2, 2, 2, 2))
    assert not O.is_singular((2, 2, 1, 0))
    assert O.periodic_axes((2, 2, 1, 1)) == 1 and O.periodic_axes((0, 0, 2, 2)) == 2


@pytest.mark.parametrize("bc", PERIODIC_BCS)
def test_fine_operator_is_kronecker_sum_with_circulant_factors(bc):
    nx, ny = 12, 10
    p = random_field(nx, ny, 3)
    np.testing.assert_allclose(O.apply_af(p, bc).ravel(), dense_laplacian(nx, ny, bc) @ p.ravel(),
                               atol=1e-13)


def test_fully_periodic_operator_is_the_rolled_laplacian():
    p = random_field(16, 8, 4)
    lap = (np.roll(p, 1, 1) + np.roll(p, -1, 1) + np.roll(p, 1, 0) + np.roll(p, -1, 0)) - 4.0 * p
    np.testing.assert_allclose(O.apply_af(p, (2, 2, 2, 2)), lap, atol=1e-13)


def dense_gs_sweep(A, p, b, nx, ny):
    """Red then black point Gauss-Seidel on the dense matrix A."""
    p = p.ravel().copy()
    for colour in (0, 1):
        for j in range(ny):
            for i in range(nx):
                if (i + j) % 2 != colour:
                    continue
                k = j * nx + i
                p[k] = (b.ravel()[k] - (A[k] @ p - A[k, k] * p[k])) / A[k, k]
    return p.reshape(ny, nx)


@pytest.mark.parametrize("bc", PERIODIC_BCS)
def test_rbgs_sweep_is_dense_red_black_gauss_seidel(bc):
    nx, ny = 8, 6
    p, b = random_field(nx, ny, 5), random_field(nx, ny, 6)
    want = dense_gs_sweep(dense_laplacian(nx, ny, bc), p, b, nx, ny)
    got = p.copy()
    O.rbgs_sweep(got, b, bc)
    np.testing.assert_allclose(got, want, atol=1e-13)


def periodic_fft_solve(b):
    """Exact mean-free solve of the fully periodic five-point equation: the
    DFT diagonalises it with eigenvalues -4 sin^2(pi k/nx) - 4 sin^2(pi l/ny)."""
    ny, nx = b.shape
    kx, ky = np.arange(nx), np.arange(ny)
    lam = (-4 * np.sin(np.pi * kx / nx) ** 2)[None, :] + (-4 * np.sin(np.pi * ky / ny) ** 2)[:, None]
    bh = np.fft.fft2(b)
    lam[0, 0] = 1.0
    ph = bh / lam
    ph[0, 0] = 0.0
    return np.fft.ifft2(ph).real


@pytest.mark.parametrize("m", [8, 16])
def test_fully_periodic_solve_matches_fft_exact_solution(m):
    nx, ny = 128, 64
    b = smooth_rhs(nx, ny, 9)
    s = O.OracleISM(nx, ny, m, (2, 2, 2, 2))
    p, cycles, _ = s.solve(b, tol=1e-12)
    ex = periodic_fft_solve(b - b.mean())
    assert cycles > 0
    assert np.linalg.norm(p - ex) <= 1e-10 * np.linalg.norm(ex)


@pytest.mark.parametrize("bc", PERIODIC_BCS)
@pytest.mark.parametrize("m", [4, 8])
def test_solve_matches_dense_pseudo_inverse_16x16(bc, m):
    nx = ny = 16
    b = smooth_rhs(nx, ny, 11)
    A = dense_laplacian(nx, ny, bc)
    if O.is_singular(bc):
        b = b - b.mean()
    ex = np.linalg.pinv(A) @ b.ravel()
    p, _, _ = O.OracleISM(nx, ny, m, bc).solve(b, tol=1e-13)
    np.testing.assert_allclose(p.ravel(), ex, atol=1e-10 * np.abs(ex).max())


def interp_axis(q, n, m, face_lo, face_hi, axis):
    """Linear interpolation of coarse centres ((I + 1/2) m) to fine centres
    along `axis` of q: numpy's periodic interpolation on a periodic axis,
    otherwise the mirror ghost rule (even at Neumann, odd at Dirichlet-0)."""
    q = np.moveaxis(q, axis, -1)
    nc = q.shape[-1]
    xc = (np.arange(nc) + 0.5) * m
    x = np.arange(n) + 0.5
    out = np.empty(q.shape[:-1] + (n,))
    for idx in np.ndindex(q.shape[:-1]):
        row = q[idx]
        if face_lo == 2:
            out[idx] = np.interp(x, xc, row, period=n)
        else:
            gl = -row[0] if face_lo == 1 else row[0]
            gh = -row[-1] if face_hi == 1 else row[-1]
            out[idx] = np.interp(x, np.concatenate([[xc[0] - m], xc, [xc[-1] + m]]),
                                 np.concatenate([[gl], row, [gh]]))
    return np.moveaxis(out, -1, axis)


@pytest.mark.parametrize("bc", PERIODIC_BCS)
def test_prolongation_is_separable_periodic_linear_interpolation(bc):
    """Eq. 5 is the tensor product of 1-D linear interpolations; across a
    periodic face it interpolates between the last and the first coarse
    centre."""
    m, ncx, ncy = 8, 6, 4
    nx, ny = m * ncx, m * ncy
    q = random_field(ncx, ncy, 12)
    p = np.zeros((ny, nx))
    O.prolong_add(p, q, m, bc)
    want = interp_axis(interp_axis(q, nx, m, bc[0], bc[1], 1), ny, m, bc[2], bc[3], 0)
    np.testing.assert_allclose(p, want, atol=1e-14)


@pytest.mark.parametrize("bc", PERIODIC_BCS)
@pytest.mark.parametrize("m", [8, 16])
def test_ism_coarse_operator_closed_form(bc, m):
    """A_c = 1/4 (S_y kron S_x) - 4 I with a circulant S on a periodic axis."""
    ncx, ncy = 6, 4
    Ac = O.coarse_operator(ncx * m, ncy * m, m, bc, "ism")
    cf = 0.25 * np.kron(S1(ncy, bc[2], bc[3]), S1(ncx, bc[0], bc[1])) - 4.0 * np.eye(ncx * ncy)
    np.testing.assert_allclose(Ac, cf, atol=1e-12)


@pytest.mark.parametrize("bc", PERIODIC_BCS)
def test_acm_and_gmg_coarse_operators_are_periodic_five_point(bc):
    m, ncx, ncy = 16, 6, 4
    L = dense_laplacian(ncx, ncy, bc)
    np.testing.assert_allclose(O.coarse_operator(ncx * m, ncy * m, m, bc, "acm"), m * L, atol=1e-12)
    np.testing.assert_allclose(O.coarse_operator(ncx * m, ncy * m, m, bc, "gmg"), L, atol=1e-12)


@pytest.mark.parametrize("bc", [(2, 2, 2, 2), (2, 2, 1, 0)])
def test_coarse_operator_equals_R_Af_P(bc):
    m, ncx, ncy = 8, 4, 4
    nx, ny = m * ncx, m * ncy
    nc = ncx * ncy
    P = np.zeros((nx * ny, nc))
    for k in range(nc):
        q = np.zeros(nc)
        q[k] = 1.0
        P[:, k] = interp_axis(interp_axis(q.reshape(ncy, ncx), nx, m, bc[0], bc[1], 1),
                              ny, m, bc[2], bc[3], 0).ravel()
    R = np.zeros((nc, nx * ny))
    for j in range(ny):
        for i in range(nx):
            R[(j // m) * ncx + i // m, j * nx + i] = 1.0
    RAP = R @ dense_laplacian(nx, ny, bc) @ P
    np.testing.assert_allclose(O.coarse_operator(nx, ny, m, bc, "ism"), RAP, atol=1e-12)


def test_one_cycle_commutes_with_a_shift_by_the_coarsening_factor():
    """On a fully periodic grid a shift by m cells maps coarse cells to
    coarse cells and keeps the red-black colouring, so one cycle commutes
    with it."""
    nx, ny, m = 96, 64, 16
    s = O.OracleISM(nx, ny, m, (2, 2, 2, 2))
    b = s.prepare_rhs(smooth_rhs(nx, ny, 13))
    p = random_field(nx, ny, 14)
    p -= p.mean()
    for axis in (0, 1):
        a, c = p.copy(), np.ascontiguousarray(np.roll(p, m, axis))
        s.cycle(a, b)
        s.cycle(c, np.ascontiguousarray(np.roll(b, m, axis)))
        np.testing.assert_allclose(c, np.roll(a, m, axis), atol=1e-12 * np.abs(a).max())


@pytest.mark.parametrize("bc", PERIODIC_BCS)
def test_coarse_correction_annihilates_restricted_residual(bc):
    m, nx, ny = 16, 96, 64
    s = O.OracleISM(nx, ny, m, bc)
    b = s.prepare_rhs(smooth_rhs(nx, ny, 7))
    p = random_field(nx, ny, 8)
    rc = O.restrict(O.residual(p, b, bc), m)
    O.prolong_add(p, s.coarse_solve(rc), m, bc)
    after = O.restrict(O.residual(p, b, bc), m)
    assert np.abs(after).max() <= 1e-11 * np.abs(rc).max()


@pytest.mark.parametrize("bc", [(2, 2, 2, 2), (2, 2, 1, 0), (1, 1, 2, 2)])
def test_ism_converges_in_fewer_cycles_than_acm(bc):
    nx, ny, m = 128, 128, 16
    b = smooth_rhs(nx, ny, 15)
    n_ism = O.OracleISM(nx, ny, m, bc, "ism").solve(b, tol=1e-8)[1]
    n_acm = O.OracleISM(nx, ny, m, bc, "acm").solve(b, tol=1e-8)[1]
    assert n_ism < n_acm


@pytest.mark.parametrize("bc", [(2, 2, 2, 2), (0, 1, 2, 2)])
def test_deep_acm_exact_solution_is_fixed_point(bc):
    nx, ny, m = 64, 64, 8
    s = O.OracleACMV(nx, ny, m, bc)
    p = random_field(nx, ny, 16)
    if O.is_singular(bc):
        p -= p.mean()
    b = O.apply_af(p, bc)
    q = p.copy()
    s.cycle(q, b)
    assert np.abs(q - p).max() <= 1e-12 * np.abs(p).max()


@pytest.mark.parametrize("bc", [(2, 2, 2, 2), (2, 2, 1, 0)])
def test_coarse_gauss_seidel_converges_to_the_exact_coarse_solution(bc):
    nx, ny, m = 96, 64, 8
    s = O.OracleISM(nx, ny, m, bc)
    rc = random_field(nx // m, ny // m, 5)
    if O.is_singular(bc):
        rc -= rc.mean()
    ec = np.zeros_like(rc)
    it = O.lib().or_coarse_gs4(nx // m, ny // m, np.ascontiguousarray(s.Ac), np.ascontiguousarray(rc), ec,
                               1e-13, 100000, O.periodic_axes(bc))
    assert 0 < it < 100000
    ex = s.coarse_solve(rc)
    if O.is_singular(bc):
        ec -= ec.mean()
        ex -= ex.mean()
    assert np.abs(ec - ex).max() <= 1e-11 * np.abs(ex).max()


@pytest.mark.parametrize("bc", [(2, 2, 2, 2), (2, 2, 0, 1)])
def test_accommodative_solve_meets_the_maximum_norm_criterion(bc):
    nx, ny, m = 128, 96, 16
    b = smooth_rhs(nx, ny, 17)
    s = O.OracleAccommodative(nx, ny, m, bc)
    p, nc_it, nf, mx = s.solve(b, tol_f=1e-6, tol_c=1e-5)
    assert nc_it > 0 and nf > 0 and mx <= 1e-6
    bb = b - b.mean() if O.is_singular(bc) else b
    assert np.abs(O.residual(p, bb, bc)).max() <= 1e-6
