/*
 * ism_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * The plain, slow, sequential CPU oracle of the interpolated stencil
 * multigrid (ISM) pressure solve and of the projection time step it sits in
 * (Tegze & Toth, "A GPU cluster optimized multigrid scheme for computing
 * unsteady incompressible fluid flow").  Only the test suite, the smoke check
 * and the CPU-baseline leg of the benchmark load this file; the product path
 * (the CUDA library) never does, and the two share no code.
 *
 * Every loop runs over cells in a fixed order (rows j = 0..ny-1 outer,
 * columns i = 0..nx-1 inner) in IEEE double, except the *_f32 variants, which
 * emulate the single-precision inner solver of the mixed path with float
 * loops.  Build with -ffp-contract=off so that no multiply-add is fused on
 * any host.
 *
 * Threads (OpenMP, when built with it): the row loops of the cell-wise
 * operations may be split over threads.  Every cell's value is computed by
 * one thread with the same arithmetic in the same order, and a row only
 * writes its own cells: a Gauss-Seidel colour reads only cells of the other
 * colour (fixed during that colour), every sum of the restriction belongs to
 * one coarse cell.  Results are therefore bit-identical for any number of
 * threads; or_set_threads(1) gives the sequential program.
 *
 * Conventions (Sec. 2.3, Sec. 3.3):
 *   cell-centred field p[j*nx + i], cell (i, j), i along x, j along y;
 *   face order bc[0..3] = west, east, south, north;
 *   bc = 0: homogeneous Neumann wall (no flux through the face);
 *   bc = 1: Dirichlet p = 0 on the face (ghost value -p_c);
 *   bc = 2: periodic, given on both faces of an axis (west and east, or
 *           south and north): the neighbour across the face is the cell at
 *           the other end of the row / column.
 *   The fine operator is the finite-volume flux sum of the five-point
 *   Laplacian (Sec. 3.3: the Gauss theorem turns the cell integral into face
 *   fluxes), in units where a face flux is (p_neighbour - p_cell):
 *       (A_f p)_c = sum over faces of flux,
 *   a Neumann face contributing 0, a Dirichlet-0 face (-p_c - p_c) and a
 *   periodic face the flux to the wrapped neighbour.
 *   The equation solved is A_f p = b.
 *
 * Coarse cells (Sec. 3.3): coarse cell I along an axis of n fine cells covers
 * fine cells [I m, min(n, (I + 1) m)); when n is not a multiple of m the last
 * coarse cell is narrower (the paper pads the grid and lets the interpolation
 * rectangles differ in size), nc = ceil(n / m).
 */
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Number of threads for the row loops (n <= 0: all host cores); returns the
   count in use (1 without OpenMP). */
int or_set_threads(int n)
{
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : omp_get_num_procs());
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

int or_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* row loop split over threads (each iteration writes its own row) */
#define ROWS_PARALLEL _Pragma("omp parallel for schedule(static)")

#define F_W 0
#define F_E 1
#define F_S 2
#define F_N 3

#define BC_DIR 1
#define BC_PER 2

#define AT(a, i, j) (a)[(size_t)(j) * (size_t)nx + (size_t)(i)]

/* ------------------------------------------------------------------------ */
/* Fine operator, Sec. 2.3 / Sec. 3.3: five-point flux sum.                  */
/* ------------------------------------------------------------------------ */

static double cell_flux_sum(int nx, int ny, const int *bc, const double *p,
                            int i, int j)
{
    double pc = AT(p, i, j);
    double s = 0.0;
    if (i > 0) s += AT(p, i - 1, j) - pc;
    else if (bc[F_W] == BC_PER) s += AT(p, nx - 1, j) - pc;
    else if (bc[F_W] == BC_DIR) s += -pc - pc;
    if (i < nx - 1) s += AT(p, i + 1, j) - pc;
    else if (bc[F_E] == BC_PER) s += AT(p, 0, j) - pc;
    else if (bc[F_E] == BC_DIR) s += -pc - pc;
    if (j > 0) s += AT(p, i, j - 1) - pc;
    else if (bc[F_S] == BC_PER) s += AT(p, i, ny - 1) - pc;
    else if (bc[F_S] == BC_DIR) s += -pc - pc;
    if (j < ny - 1) s += AT(p, i, j + 1) - pc;
    else if (bc[F_N] == BC_PER) s += AT(p, i, 0) - pc;
    else if (bc[F_N] == BC_DIR) s += -pc - pc;
    return s;
}

/* out = A_f p */
void or_apply_af(int nx, int ny, const int *bc, const double *p, double *out)
{
    ROWS_PARALLEL
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i)
            AT(out, i, j) = cell_flux_sum(nx, ny, bc, p, i, j);
}

/* r = b - A_f p */
void or_residual(int nx, int ny, const int *bc, const double *p,
                 const double *b, double *r)
{
    ROWS_PARALLEL
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i)
            AT(r, i, j) = AT(b, i, j) - cell_flux_sum(nx, ny, bc, p, i, j);
}

/* ------------------------------------------------------------------------ */
/* Red-black Gauss-Seidel sweep, Sec. 3.1: the point update solves the cell's */
/* own equation for p_c with the neighbours held fixed:                       */
/*   p_c = (sum of neighbours - b_c) / d_c,                                   */
/*   d_c = (#neighbours) + 2 (#Dirichlet-0 faces),                            */
/* a periodic face's wrapped cell counting as a neighbour.  Red cells         */
/* ((i + j) even) are updated first, then black; a periodic axis has an even  */
/* number of cells, so wrapped neighbours have the other colour.              */
/* ------------------------------------------------------------------------ */

static void gs_colour(int nx, int ny, const int *bc, double *p, const double *b,
                      int colour)
{
    ROWS_PARALLEL
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            if (((i + j) & 1) != colour) continue;
            double s = 0.0;
            int d = 0;
            if (i > 0) { s += AT(p, i - 1, j); d += 1; }
            else if (bc[F_W] == BC_PER) { s += AT(p, nx - 1, j); d += 1; }
            else if (bc[F_W] == BC_DIR) d += 2;
            if (i < nx - 1) { s += AT(p, i + 1, j); d += 1; }
            else if (bc[F_E] == BC_PER) { s += AT(p, 0, j); d += 1; }
            else if (bc[F_E] == BC_DIR) d += 2;
            if (j > 0) { s += AT(p, i, j - 1); d += 1; }
            else if (bc[F_S] == BC_PER) { s += AT(p, i, ny - 1); d += 1; }
            else if (bc[F_S] == BC_DIR) d += 2;
            if (j < ny - 1) { s += AT(p, i, j + 1); d += 1; }
            else if (bc[F_N] == BC_PER) { s += AT(p, i, 0); d += 1; }
            else if (bc[F_N] == BC_DIR) d += 2;
            AT(p, i, j) = (s - AT(b, i, j)) / (double)d;
        }
    }
}

void or_rbgs_sweep(int nx, int ny, const int *bc, double *p, const double *b)
{
    gs_colour(nx, ny, bc, p, b, 0);
    gs_colour(nx, ny, bc, p, b, 1);
}

static int ncoarse(int n, int m) { return (n + m - 1) / m; }
static int block_end(int I, int n, int m) { return (I + 1) * m < n ? (I + 1) * m : n; }

/* ------------------------------------------------------------------------ */
/* Restriction, Sec. 3.2-3.3: the coarse right-hand side is the sum of the    */
/* fine equations over the coarse cell (agglomeration, as in ACM).            */
/* ------------------------------------------------------------------------ */

void or_restrict(int nx, int ny, int m, const double *r, double *rc)
{
    int ncx = ncoarse(nx, m), ncy = ncoarse(ny, m);
    ROWS_PARALLEL
    for (int J = 0; J < ncy; ++J)
        for (int I = 0; I < ncx; ++I) {
            double s = 0.0;
            for (int j = J * m; j < block_end(J, ny, m); ++j)
                for (int i = I * m; i < block_end(I, nx, m); ++i)
                    s += AT(r, i, j);
            rc[(size_t)J * ncx + I] = s;
        }
}

/* ------------------------------------------------------------------------ */
/* Bilinear interpolation from coarse centres, Eq. 5.                          */
/* Q11, Q21, Q12, Q22 are the corner values of the interpolation rectangle    */
/* (Delta_x, Delta_y: the distances between neighbouring coarse centres, m    */
/* fine cells except next to a narrower last coarse cell), (x, y) the         */
/* fine-cell centre measured from Q11.  Outside the hull of coarse centres    */
/* the rule near the boundary is a ghost centre mirrored across the wall      */
/* (distance m beyond the edge centre when the edge cell is m wide; the paper */
/* leaves this rule open): even (Q_ghost = Q_edge) at a Neumann face, odd     */
/* (Q_ghost = -Q_edge) at a Dirichlet-0 face; across a periodic face the      */
/* ghost is the coarse centre at the other end (the periodic extension).      */
/* ------------------------------------------------------------------------ */

/* fine coordinate of coarse centre I along an axis of n fine cells; I = -1
   and I = nc give the ghost centres */
static double centre(int I, int n, int m, int periodic)
{
    int nc = ncoarse(n, m);
    if (I < 0) return periodic ? centre(I + nc, n, m, 0) - n : -centre(0, n, m, 0);
    if (I >= nc) return periodic ? centre(I - nc, n, m, 0) + n : 2.0 * n - centre(nc - 1, n, m, 0);
    return 0.5 * (double)(I * m + block_end(I, n, m));
}

/* the coarse centre at or before fine centre i + 1/2 (possibly a ghost) */
static int left_centre(int i, int n, int m, int periodic)
{
    int I = i / m;
    if (centre(I, n, m, periodic) > (double)i + 0.5) --I;
    return I;
}

static double coarse_or_ghost(int ncx, int ncy, const int *bc, const double *q,
                              int I, int J)
{
    double sgn = 1.0;
    if (I < 0) { if (bc[F_W] == BC_PER) I += ncx; else { I = 0; if (bc[F_W] == BC_DIR) sgn = -sgn; } }
    if (I >= ncx) { if (bc[F_E] == BC_PER) I -= ncx; else { I = ncx - 1; if (bc[F_E] == BC_DIR) sgn = -sgn; } }
    if (J < 0) { if (bc[F_S] == BC_PER) J += ncy; else { J = 0; if (bc[F_S] == BC_DIR) sgn = -sgn; } }
    if (J >= ncy) { if (bc[F_N] == BC_PER) J -= ncy; else { J = ncy - 1; if (bc[F_N] == BC_DIR) sgn = -sgn; } }
    return sgn * q[(size_t)J * ncx + I];
}

/* value of the interpolant P q at fine cell (i, j) */
static double bilinear_at(int nx, int ny, int m, const int *bc, const double *q,
                          int i, int j)
{
    int ncx = ncoarse(nx, m), ncy = ncoarse(ny, m);
    int px = bc[F_W] == BC_PER, py = bc[F_S] == BC_PER;
    /* lower-left corner of the interpolation rectangle: the coarse centre at
       or left of / below the fine centre */
    int I0 = left_centre(i, nx, m, px);
    int J0 = left_centre(j, ny, m, py);
    double cx0 = centre(I0, nx, m, px), cy0 = centre(J0, ny, m, py);
    double Dx = centre(I0 + 1, nx, m, px) - cx0, Dy = centre(J0 + 1, ny, m, py) - cy0;
    double x = ((double)i + 0.5) - cx0;
    double y = ((double)j + 0.5) - cy0;
    double Q11 = coarse_or_ghost(ncx, ncy, bc, q, I0, J0);
    double Q21 = coarse_or_ghost(ncx, ncy, bc, q, I0 + 1, J0);
    double Q12 = coarse_or_ghost(ncx, ncy, bc, q, I0, J0 + 1);
    double Q22 = coarse_or_ghost(ncx, ncy, bc, q, I0 + 1, J0 + 1);
    return (Q11 * (Dx - x) * (Dy - y) + Q21 * x * (Dy - y)
            + Q12 * (Dx - x) * y + Q22 * x * y) / (Dx * Dy);
}

/* p += P q (bilinear prolongation with the same rule, Sec. 3.3) */
void or_prolong_add(int nx, int ny, int m, const int *bc, const double *q, double *p)
{
    ROWS_PARALLEL
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i)
            AT(p, i, j) += bilinear_at(nx, ny, m, bc, q, i, j);
}

/* p += q[block] (piecewise-constant correction of ACM, Sec. 3.2) */
void or_prolong_const_add(int nx, int ny, int m, const double *q, double *p)
{
    int ncx = ncoarse(nx, m);
    ROWS_PARALLEL
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i)
            AT(p, i, j) += q[(size_t)(j / m) * ncx + (i / m)];
}

/* ------------------------------------------------------------------------ */
/* Coarse operator, Sec. 3.3 (Eq. 5-7, Fig. 1).                                */
/* Column J of A_c is obtained by interpolating the unit coarse vector e_J to */
/* the fine grid and summing, for every coarse cell K, the fine face fluxes    */
/* (p_out - p_in) that cross the boundary of K; fluxes inside K cancel.  With */
/* kind = 0 (ISM) the fine values come from the bilinear rule above; with      */
/* kind = 1 (ACM) p is constant inside each coarse cell, which reproduces the  */
/* summation of the fine equations.  The result is dense row-major nc x nc,    */
/* row K = coarse equation, column J = coarse unknown.                         */
/* ------------------------------------------------------------------------ */

static double face_sums(int nx, int ny, int m, const int *bc, const double *p,
                        int KI, int KJ)
{
    int x0 = KI * m, x1 = block_end(KI, nx, m), y0 = KJ * m, y1 = block_end(KJ, ny, m);
    double s = 0.0;
    for (int j = y0; j < y1; ++j) {                     /* west face */
        if (x0 > 0) s += AT(p, x0 - 1, j) - AT(p, x0, j);
        else if (bc[F_W] == BC_PER) s += AT(p, nx - 1, j) - AT(p, x0, j);
        else if (bc[F_W] == BC_DIR) s += -AT(p, x0, j) - AT(p, x0, j);
    }
    for (int j = y0; j < y1; ++j) {                     /* east face */
        if (x1 < nx) s += AT(p, x1, j) - AT(p, x1 - 1, j);
        else if (bc[F_E] == BC_PER) s += AT(p, 0, j) - AT(p, x1 - 1, j);
        else if (bc[F_E] == BC_DIR) s += -AT(p, x1 - 1, j) - AT(p, x1 - 1, j);
    }
    for (int i = x0; i < x1; ++i) {                     /* south face */
        if (y0 > 0) s += AT(p, i, y0 - 1) - AT(p, i, y0);
        else if (bc[F_S] == BC_PER) s += AT(p, i, ny - 1) - AT(p, i, y0);
        else if (bc[F_S] == BC_DIR) s += -AT(p, i, y0) - AT(p, i, y0);
    }
    for (int i = x0; i < x1; ++i) {                     /* north face */
        if (y1 < ny) s += AT(p, i, y1) - AT(p, i, y1 - 1);
        else if (bc[F_N] == BC_PER) s += AT(p, i, 0) - AT(p, i, y1 - 1);
        else if (bc[F_N] == BC_DIR) s += -AT(p, i, y1 - 1) - AT(p, i, y1 - 1);
    }
    return s;
}

int or_coarse_operator(int nx, int ny, int m, const int *bc, int kind, double *Ac)
{
    int ncx = ncoarse(nx, m), ncy = ncoarse(ny, m), nc = ncx * ncy;
    double *p = (double *)calloc((size_t)nx * ny, sizeof(double));
    double *q = (double *)calloc((size_t)nc, sizeof(double));
    if (!p || !q) { free(p); free(q); return -1; }
    memset(Ac, 0, sizeof(double) * (size_t)nc * nc);
    for (int JJ = 0; JJ < ncy; ++JJ) {
        for (int JI = 0; JI < ncx; ++JI) {
            int col = JJ * ncx + JI;
            q[col] = 1.0;
            /* the interpolant of e_J vanishes outside coarse cells JI-1..JI+1,
               JJ-1..JJ+1 (the hat spans from centre to neighbouring centre);
               along a periodic axis the hat wraps, so the whole axis is
               swept there */
            int bi0 = JI - 1 < 0 ? 0 : JI - 1, bi1 = JI + 1 >= ncx ? ncx - 1 : JI + 1;
            int bj0 = JJ - 1 < 0 ? 0 : JJ - 1, bj1 = JJ + 1 >= ncy ? ncy - 1 : JJ + 1;
            if (bc[F_W] == BC_PER) { bi0 = 0; bi1 = ncx - 1; }
            if (bc[F_S] == BC_PER) { bj0 = 0; bj1 = ncy - 1; }
            for (int j = bj0 * m; j < block_end(bj1, ny, m); ++j)
                for (int i = bi0 * m; i < block_end(bi1, nx, m); ++i)
                    AT(p, i, j) = (kind == 0) ? bilinear_at(nx, ny, m, bc, q, i, j)
                                              : q[(size_t)(j / m) * ncx + (i / m)];
            for (int KJ = bj0; KJ <= bj1; ++KJ)
                for (int KI = bi0; KI <= bi1; ++KI)
                    Ac[(size_t)(KJ * ncx + KI) * nc + col] =
                        face_sums(nx, ny, m, bc, p, KI, KJ);
            for (int j = bj0 * m; j < block_end(bj1, ny, m); ++j)
                for (int i = bi0 * m; i < block_end(bi1, nx, m); ++i)
                    AT(p, i, j) = 0.0;
            q[col] = 0.0;
        }
    }
    free(p);
    free(q);
    return 0;
}

/* The same assembly for large coarse grids, returned as (row, column,     */
/* value) triples instead of a dense matrix: the interpolant of e_J is       */
/* evaluated on a window of the coarse cells J-1..J+1 with a border of one   */
/* zero cell (the interpolant vanishes beyond them), and the face sums of    */
/* every coarse cell K of the window are taken there with the same rules and */
/* the same order of operations as face_sums.  Walls only (no periodic       */
/* face: its wrapped neighbours lie outside the window).  rows, cols, vals   */
/* hold 9 nc entries; returns the number written, or -1 (allocation failed,  */
/* or a periodic face).  The columns are independent, so they may be split   */
/* over threads; each triple is computed by one thread as in the dense form. */
/* ------------------------------------------------------------------------ */

#define WIN(a, i, j) (a)[(size_t)((j) - wy0 + 1) * (size_t)(wx + 2) + (size_t)((i) - wx0 + 1)]

static double face_sums_window(int nx, int ny, int m, const int *bc, const double *w,
                               int wx0, int wy0, int wx, int KI, int KJ)
{
    int x0 = KI * m, x1 = block_end(KI, nx, m), y0 = KJ * m, y1 = block_end(KJ, ny, m);
    double s = 0.0;
    for (int j = y0; j < y1; ++j) {                     /* west face */
        if (x0 > 0) s += WIN(w, x0 - 1, j) - WIN(w, x0, j);
        else if (bc[F_W] == BC_DIR) s += -WIN(w, x0, j) - WIN(w, x0, j);
    }
    for (int j = y0; j < y1; ++j) {                     /* east face */
        if (x1 < nx) s += WIN(w, x1, j) - WIN(w, x1 - 1, j);
        else if (bc[F_E] == BC_DIR) s += -WIN(w, x1 - 1, j) - WIN(w, x1 - 1, j);
    }
    for (int i = x0; i < x1; ++i) {                     /* south face */
        if (y0 > 0) s += WIN(w, i, y0 - 1) - WIN(w, i, y0);
        else if (bc[F_S] == BC_DIR) s += -WIN(w, i, y0) - WIN(w, i, y0);
    }
    for (int i = x0; i < x1; ++i) {                     /* north face */
        if (y1 < ny) s += WIN(w, i, y1) - WIN(w, i, y1 - 1);
        else if (bc[F_N] == BC_DIR) s += -WIN(w, i, y1 - 1) - WIN(w, i, y1 - 1);
    }
    return s;
}

long or_coarse_operator_coo(int nx, int ny, int m, const int *bc, int kind,
                            int *rows, int *cols, double *vals)
{
    int ncx = ncoarse(nx, m), ncy = ncoarse(ny, m);
    long nc = (long)ncx * ncy;
    for (int f = 0; f < 4; ++f)
        if (bc[f] == BC_PER) return -1;
    long count = 0;
    int fail = 0;
    /* each column writes its own 9 slots: column c owns entries 9c .. 9c+8 */
    _Pragma("omp parallel")
    {
        const size_t wmax = (size_t)(3 * m + 2) * (size_t)(3 * m + 2);
        double *w = (double *)calloc(wmax, sizeof(double));
        double *q = (double *)calloc((size_t)nc, sizeof(double));
        if (!w || !q) {
            _Pragma("omp atomic write")
            fail = 1;
        } else {
            _Pragma("omp for schedule(static)")
            for (long col = 0; col < nc; ++col) {
                int JI = (int)(col % ncx), JJ = (int)(col / ncx);
                int bi0 = JI - 1 < 0 ? 0 : JI - 1, bi1 = JI + 1 >= ncx ? ncx - 1 : JI + 1;
                int bj0 = JJ - 1 < 0 ? 0 : JJ - 1, bj1 = JJ + 1 >= ncy ? ncy - 1 : JJ + 1;
                int wx0 = bi0 * m, wy0 = bj0 * m;
                int wx = block_end(bi1, nx, m) - wx0, wy = block_end(bj1, ny, m) - wy0;
                memset(w, 0, (size_t)(wx + 2) * (size_t)(wy + 2) * sizeof(double));
                q[col] = 1.0;
                for (int j = wy0; j < wy0 + wy; ++j)
                    for (int i = wx0; i < wx0 + wx; ++i)
                        WIN(w, i, j) = (kind == 0) ? bilinear_at(nx, ny, m, bc, q, i, j)
                                                   : q[(size_t)(j / m) * ncx + (i / m)];
                q[col] = 0.0;
                int k = 0;
                for (int KJ = bj0; KJ <= bj1; ++KJ)
                    for (int KI = bi0; KI <= bi1; ++KI, ++k) {
                        rows[9 * col + k] = KJ * ncx + KI;
                        cols[9 * col + k] = (int)col;
                        vals[9 * col + k] = face_sums_window(nx, ny, m, bc, w, wx0, wy0, wx, KI, KJ);
                    }
                for (; k < 9; ++k) {             /* unused slots (edge columns) */
                    rows[9 * col + k] = -1;
                    cols[9 * col + k] = -1;
                    vals[9 * col + k] = 0.0;
                }
            }
        }
        free(w);
        free(q);
    }
    if (fail) return -1;
    count = 9 * nc;
    return count;
}

#undef WIN

/* ------------------------------------------------------------------------ */
/* Gauss-Seidel on the coarse equations A_c e = r (the paper's iterative      */
/* coarse solve, Sec. 4.3.1), four-colour ordering of the nine-point stencil: */
/* colour (I mod 2) + 2 (J mod 2), colours 0..3 in turn; the matrix is the    */
/* assembled dense A_c (nc x nc), its nine neighbours taken in the order      */
/* dJ = -1..1, dI = -1..1.  Runs full iterations until max |r - A_c e| <=     */
/* tol (checked after each iteration) or `cap` iterations; returns the count. */
/* per: bit 0 x periodic, bit 1 y periodic: the neighbours wrap around that   */
/* axis (which then has an even number >= 4 of coarse cells, so the nine are  */
/* distinct and the four colours stay independent).                            */
/* ------------------------------------------------------------------------ */
static int gs4_wrap(int K, int n, int periodic)
{
    if (!periodic) return K;
    return K < 0 ? K + n : (K >= n ? K - n : K);
}

int or_coarse_gs4(int ncx, int ncy, const double *Ac, const double *r, double *e,
                  double tol, int cap, int per)
{
    const size_t nc = (size_t)ncx * ncy;
    int it = 0;
    for (;;) {
        double mx = 0.0;
        for (int J = 0; J < ncy; ++J)
            for (int I = 0; I < ncx; ++I) {
                const size_t row = (size_t)J * ncx + I;
                double s = 0.0;
                for (int dJ = -1; dJ <= 1; ++dJ)
                    for (int dI = -1; dI <= 1; ++dI) {
                        const int K = gs4_wrap(J + dJ, ncy, per & 2), L = gs4_wrap(I + dI, ncx, per & 1);
                        if (K < 0 || K >= ncy || L < 0 || L >= ncx) continue;
                        const size_t col = (size_t)K * ncx + L;
                        s += Ac[row * nc + col] * e[col];
                    }
                const double d = fabs(r[row] - s);
                if (d > mx) mx = d;
            }
        if (mx <= tol || it >= cap) return it;
        for (int colour = 0; colour < 4; ++colour)
            for (int J = colour >> 1; J < ncy; J += 2)
                for (int I = colour & 1; I < ncx; I += 2) {
                    const size_t row = (size_t)J * ncx + I;
                    double s = 0.0;
                    for (int dJ = -1; dJ <= 1; ++dJ)
                        for (int dI = -1; dI <= 1; ++dI) {
                            const int K = gs4_wrap(J + dJ, ncy, per & 2), L = gs4_wrap(I + dI, ncx, per & 1);
                            if ((dI == 0 && dJ == 0) || K < 0 || K >= ncy || L < 0 || L >= ncx) continue;
                            const size_t col = (size_t)K * ncx + L;
                            s += Ac[row * nc + col] * e[col];
                        }
                    e[row] = (r[row] - s) / Ac[row * nc + row];
                }
        ++it;
    }
}

/* ------------------------------------------------------------------------ */
/* Single-precision emulation of the inner solver of the mixed path.          */
/* Same steps as above in float arithmetic; sums of the restriction and of    */
/* norms are accumulated in double.                                           */
/* ------------------------------------------------------------------------ */

static float cell_flux_sum_f(int nx, int ny, const int *bc, const float *p,
                             int i, int j)
{
    float pc = AT(p, i, j);
    float s = 0.0f;
    if (i > 0) s += AT(p, i - 1, j) - pc;
    else if (bc[F_W] == BC_PER) s += AT(p, nx - 1, j) - pc;
    else if (bc[F_W] == BC_DIR) s += -pc - pc;
    if (i < nx - 1) s += AT(p, i + 1, j) - pc;
    else if (bc[F_E] == BC_PER) s += AT(p, 0, j) - pc;
    else if (bc[F_E] == BC_DIR) s += -pc - pc;
    if (j > 0) s += AT(p, i, j - 1) - pc;
    else if (bc[F_S] == BC_PER) s += AT(p, i, ny - 1) - pc;
    else if (bc[F_S] == BC_DIR) s += -pc - pc;
    if (j < ny - 1) s += AT(p, i, j + 1) - pc;
    else if (bc[F_N] == BC_PER) s += AT(p, i, 0) - pc;
    else if (bc[F_N] == BC_DIR) s += -pc - pc;
    return s;
}

void or_residual_f32(int nx, int ny, const int *bc, const float *p,
                     const float *b, float *r)
{
    ROWS_PARALLEL
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i)
            AT(r, i, j) = AT(b, i, j) - cell_flux_sum_f(nx, ny, bc, p, i, j);
}

static void gs_colour_f(int nx, int ny, const int *bc, float *p, const float *b,
                        int colour)
{
    ROWS_PARALLEL
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            if (((i + j) & 1) != colour) continue;
            float s = 0.0f;
            int d = 0;
            if (i > 0) { s += AT(p, i - 1, j); d += 1; }
            else if (bc[F_W] == BC_PER) { s += AT(p, nx - 1, j); d += 1; }
            else if (bc[F_W] == BC_DIR) d += 2;
            if (i < nx - 1) { s += AT(p, i + 1, j); d += 1; }
            else if (bc[F_E] == BC_PER) { s += AT(p, 0, j); d += 1; }
            else if (bc[F_E] == BC_DIR) d += 2;
            if (j > 0) { s += AT(p, i, j - 1); d += 1; }
            else if (bc[F_S] == BC_PER) { s += AT(p, i, ny - 1); d += 1; }
            else if (bc[F_S] == BC_DIR) d += 2;
            if (j < ny - 1) { s += AT(p, i, j + 1); d += 1; }
            else if (bc[F_N] == BC_PER) { s += AT(p, i, 0); d += 1; }
            else if (bc[F_N] == BC_DIR) d += 2;
            AT(p, i, j) = (s - AT(b, i, j)) / (float)d;
        }
    }
}

void or_rbgs_sweep_f32(int nx, int ny, const int *bc, float *p, const float *b)
{
    gs_colour_f(nx, ny, bc, p, b, 0);
    gs_colour_f(nx, ny, bc, p, b, 1);
}

void or_restrict_f32(int nx, int ny, int m, const float *r, double *rc)
{
    int ncx = ncoarse(nx, m), ncy = ncoarse(ny, m);
    ROWS_PARALLEL
    for (int J = 0; J < ncy; ++J)
        for (int I = 0; I < ncx; ++I) {
            double s = 0.0;
            for (int j = J * m; j < block_end(J, ny, m); ++j)
                for (int i = I * m; i < block_end(I, nx, m); ++i)
                    s += (double)AT(r, i, j);
            rc[(size_t)J * ncx + I] = s;
        }
}

void or_prolong_add_f32(int nx, int ny, int m, const int *bc, const double *q, float *p)
{
    ROWS_PARALLEL
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i)
            AT(p, i, j) = AT(p, i, j) + (float)bilinear_at(nx, ny, m, bc, q, i, j);
}

/* ------------------------------------------------------------------------ */
/* Projection time step, Sec. 2.2-2.3 (Eq. 3-4), physical signs:              */
/*   v* = v^n + dt [ -(v.grad) v + nu lap v - grad p^n ]     (forward Euler)  */
/*   A_f dp = h (div_flux v*) / dt                                            */
/*   v^{n+1} = v* - dt grad dp,   p^{n+1} = p^n + dp                          */
/* on the staggered (MAC) grid: u[j*(nx+1) + i] on x-faces (i = 0..nx),       */
/* v[j*nx + i] on y-faces (j = 0..ny).  Second-order central differences,     */
/* advective form, face-averaged transverse velocity.                          */
/*                                                                             */
/* Face kinds (vel_bc[face]): 0 no-slip wall moving tangentially with          */
/* wall_u[face]; 1 free-slip wall; 2 inflow (west face only, profile u_in[j]); */
/* 3 convective outflow (east face only, speed conv_u); 4 periodic (on both    */
/* faces of an axis: the neighbour across the face is at the other end, and   */
/* the last face of the axis, kept equal to the first, is the same face).     */
/* The pressure is Dirichlet-0 on outflow faces, periodic on periodic faces   */
/* and Neumann elsewhere.                                                      */
/* ------------------------------------------------------------------------ */

#define UU(i, j) u[(size_t)(j) * (size_t)(nx + 1) + (size_t)(i)]
#define VV(i, j) v[(size_t)(j) * (size_t)nx + (size_t)(i)]
#define US(i, j) us[(size_t)(j) * (size_t)(nx + 1) + (size_t)(i)]
#define VS(i, j) vs[(size_t)(j) * (size_t)nx + (size_t)(i)]
#define PP(i, j) p[(size_t)(j) * (size_t)nx + (size_t)(i)]

#define VEL_PER 4

static int wrapn(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

/* ghost value of a tangential velocity component beyond a face */
static double tangential_ghost(int kind, double wall_u, double inner)
{
    switch (kind) {
    case 0: return 2.0 * wall_u - inner;   /* no-slip: mean of inner and ghost = wall speed */
    case 1: return inner;                  /* free slip: zero normal gradient */
    case 2: return -inner;                 /* inflow: no tangential velocity at the inlet */
    default: return inner;                 /* outflow: zero normal gradient */
    }
}

void or_predictor(int nx, int ny, double h, double dt, double nu,
                  const int *vel_bc, const double *wall_u, const double *u_in,
                  double conv_u, const double *u, const double *v,
                  const double *p, double *us, double *vs)
{
    double ih = 1.0 / h, ih2 = 1.0 / (h * h);
    int px = vel_bc[F_W] == VEL_PER, py = vel_bc[F_S] == VEL_PER;
    /* x-faces; with x periodic, face 0 is computed like an interior face
       (west neighbours wrap) and face nx is the same face */
    ROWS_PARALLEL
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i <= nx; ++i) {
            double uc = UU(i, j);
            if (px && i == nx) continue;
            if (!px && i == 0) {
                US(i, j) = (vel_bc[F_W] == 2) ? u_in[j] : 0.0;
                continue;
            }
            if (!px && i == nx) {
                if (vel_bc[F_E] == 3) {
                    double pin = PP(nx - 1, j);
                    double gp = (-pin - pin) * ih;                /* ghost -p: Dirichlet 0 */
                    US(i, j) = uc + dt * (-conv_u * (uc - UU(nx - 1, j)) * ih - gp);
                } else {
                    US(i, j) = 0.0;
                }
                continue;
            }
            int im = wrapn(i - 1, nx), ip = px ? wrapn(i + 1, nx) : i + 1, jp = py ? wrapn(j + 1, ny) : j + 1;
            double uw = UU(im, j), ue = UU(ip, j);
            double usx = (j > 0) ? UU(i, j - 1) : (py ? UU(i, ny - 1) : tangential_ghost(vel_bc[F_S], wall_u[F_S], uc));
            double unx = (j < ny - 1) ? UU(i, j + 1) : (py ? UU(i, 0) : tangential_ghost(vel_bc[F_N], wall_u[F_N], uc));
            double vbar = 0.25 * (VV(im, j) + VV(i, j) + VV(im, jp) + VV(i, jp));
            double adv = uc * (ue - uw) * (0.5 * ih) + vbar * (unx - usx) * (0.5 * ih);
            double lap = (ue + uw + unx + usx - 4.0 * uc) * ih2;
            double gp = (PP(i, j) - PP(im, j)) * ih;
            US(i, j) = uc + dt * (-adv + nu * lap - gp);
        }
        if (px) US(nx, j) = US(0, j);
    }
    /* y-faces: south and north are walls (zero normal velocity) unless y is
       periodic (then face 0 is computed like an interior face and face ny is
       the same face) */
    ROWS_PARALLEL
    for (int j = 0; j <= ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            double vc = VV(i, j);
            if (py && j == ny) { VS(i, j) = 0.0; continue; }      /* set from face 0 below */
            if (!py && (j == 0 || j == ny)) { VS(i, j) = 0.0; continue; }
            int jm = wrapn(j - 1, ny), jp = py ? wrapn(j + 1, ny) : j + 1, ip = px ? wrapn(i + 1, nx) : i + 1;
            double vsy = VV(i, jm), vny = VV(i, jp);
            double vw = (i > 0) ? VV(i - 1, j) : (px ? VV(nx - 1, j) : tangential_ghost(vel_bc[F_W], wall_u[F_W], vc));
            double ve = (i < nx - 1) ? VV(i + 1, j) : (px ? VV(0, j) : tangential_ghost(vel_bc[F_E], wall_u[F_E], vc));
            double ubar = 0.25 * (UU(i, jm) + UU(ip, jm) + UU(i, j) + UU(ip, j));
            double adv = ubar * (ve - vw) * (0.5 * ih) + vc * (vny - vsy) * (0.5 * ih);
            double lap = (ve + vw + vny + vsy - 4.0 * vc) * ih2;
            double gp = (PP(i, j) - PP(i, jm)) * ih;
            VS(i, j) = vc + dt * (-adv + nu * lap - gp);
        }
    }
    if (py)
        for (int i = 0; i < nx; ++i) VS(i, ny) = VS(i, 0);
}

/* b = h (u_e - u_w + v_n - v_s) / dt : right-hand side of A_f dp = b (Eq. 4) */
void or_divergence(int nx, int ny, double h, double dt, const double *u,
                   const double *v, double *b)
{
    ROWS_PARALLEL
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i)
            b[(size_t)j * nx + i] = h * ((UU(i + 1, j) - UU(i, j))
                                         + (VV(i, j + 1) - VV(i, j))) / dt;
}

/* v^{n+1} = v* - dt grad dp on every face whose normal velocity is not
   prescribed (across a periodic face the gradient takes the cell at the
   other end, and the last face copies the first); p += dp */
void or_correct(int nx, int ny, double h, double dt, const int *vel_bc,
                const double *dp, double *u, double *v, double *p)
{
    double s = dt / h;
    int px = vel_bc[F_W] == VEL_PER, py = vel_bc[F_S] == VEL_PER;
    ROWS_PARALLEL
    for (int j = 0; j < ny; ++j) {
        for (int i = 1; i < nx; ++i)
            UU(i, j) -= s * (dp[(size_t)j * nx + i] - dp[(size_t)j * nx + i - 1]);
        if (px) {
            UU(0, j) -= s * (dp[(size_t)j * nx] - dp[(size_t)j * nx + nx - 1]);
            UU(nx, j) = UU(0, j);
        }
        if (vel_bc[F_E] == 3) {
            double pin = dp[(size_t)j * nx + nx - 1];
            UU(nx, j) -= s * (-pin - pin);
        }
    }
    ROWS_PARALLEL
    for (int j = 1; j < ny; ++j)
        for (int i = 0; i < nx; ++i)
            VV(i, j) -= s * (dp[(size_t)j * nx + i] - dp[(size_t)(j - 1) * nx + i]);
    if (py)
        for (int i = 0; i < nx; ++i) {
            VV(i, 0) -= s * (dp[i] - dp[(size_t)(ny - 1) * nx + i]);
            VV(i, ny) = VV(i, 0);
        }
    for (size_t k = 0; k < (size_t)nx * ny; ++k) p[k] += dp[k];
}
