// ism_pencil.cu -- host numerics of the coarse level when the grid is not a
// multiple of the coarsening factor (Sec. 3.3: the grid is padded and the
// interpolation rectangles next to the last, narrower coarse cell differ in
// size).
//
// The restriction R (block sums), the interpolation P (bilinear, Eq. 5) and
// the fine operator A_f are tensor products / a Kronecker sum of 1-D
// operators, so the coarse operator R A_f P is
//     A_c = W_y (x) T_x + T_y (x) W_x,     W = R1 P1,  T = R1 T1 P1
// with the 1-D block sum R1, interpolation P1 and second difference T1 of
// each axis (ACM: P1 piecewise constant).  W and T are tridiagonal; W is not
// symmetric when the last coarse cell is narrower.  With the 1-D pencils
// T V = W V diag(lam) and L = (W V)^-1:
//     A_c = (W_y V_y (x) W_x V_x) (diag(lam_y) (+) diag(lam_x)) (V_y (x) V_x)^-1
//     A_c^-1 = (V_y (x) V_x) diag(1 / (lam_y[l] + lam_x[k])) (L_y (x) L_x),
// the same four-product form as the uniform case (there V = Q orthonormal).
// The eigenvalues are found by bisection on the pivot signs of T - lam W:
// for lam <= 0 every off-diagonal product of T - lam W is positive, so the
// matrix is diagonally similar to a symmetric one and its pivots count its
// negative eigenvalues; the count is checked to run from 0 to n over the
// bracket, every eigenvector is checked by its residual, and any failed
// check rejects the grid (the caller returns ISM_ERR_ARG).
#include <math.h>

#include <algorithm>
#include <vector>

#include "ism_internal.cuh"

namespace {

int ncoarse(int n, int m) { return (n + m - 1) / m; }
int block_end(int I, int n, int m) { return std::min(n, (I + 1) * m); }

// fine coordinate of coarse centre I (I = -1, nc: ghosts mirrored across the walls)
double centre(int I, int n, int m)
{
    const int nc = ncoarse(n, m);
    if (I < 0) return -centre(0, n, m);
    if (I >= nc) return 2.0 * n - centre(nc - 1, n, m);
    return 0.5 * (double)(I * m + block_end(I, n, m));
}

struct Tri {   // tridiagonal n x n: l[k] = A[k][k-1], d[k] = A[k][k], u[k] = A[k][k+1]
    std::vector<double> l, d, u;
    explicit Tri(int n) : l(n, 0.0), d(n, 0.0), u(n, 0.0) {}
    void add(int r, int c, double v)
    {
        if (c == r) d[r] += v;
        else if (c == r - 1) l[r] += v;
        else if (c == r + 1) u[r] += v;
        else if (v != 0.0) bad = true;
    }
    bool bad = false;
};

// row i of P1: up to two (coarse index, weight) pairs, ghost indices folded
// back with the wall's sign (even at Neumann, odd at Dirichlet-0)
int p_row(int i, int n, int m, int lo_dir, int hi_dir, bool constant, int *idx, double *w)
{
    const int nc = ncoarse(n, m);
    if (constant) { idx[0] = i / m; w[0] = 1.0; return 1; }
    int I0 = i / m;
    const double x = i + 0.5;
    if (centre(I0, n, m) > x) --I0;
    const double c0 = centre(I0, n, m), t = (x - c0) / (centre(I0 + 1, n, m) - c0);
    int k = 0;
    for (int s = 0; s < 2; ++s) {
        int I = I0 + s;
        double v = s ? t : 1.0 - t;
        if (I < 0) { I = 0; if (lo_dir) v = -v; }
        if (I >= nc) { I = nc - 1; if (hi_dir) v = -v; }
        idx[k] = I; w[k] = v; ++k;
    }
    return k;
}

// (n x n) tridiagonal solve with partial pivoting, b overwritten by x
void tri_solve(const std::vector<double> &dl0, const std::vector<double> &d0, const std::vector<double> &du0,
               std::vector<double> &b)
{
    const int n = (int)d0.size();
    std::vector<double> u0(n), u1(n, 0.0), u2(n, 0.0);
    const double tiny = 1e-300;
    double cd = d0[0], cu = n > 1 ? du0[0] : 0.0;
    for (int i = 0; i + 1 < n; ++i) {
        const double nl = dl0[i + 1], nd = d0[i + 1], nu = (i + 2 < n) ? du0[i + 1] : 0.0;
        if (fabs(cd) >= fabs(nl)) {
            const double piv = cd != 0.0 ? cd : tiny, f = nl / piv;
            u0[i] = piv; u1[i] = cu; u2[i] = 0.0;
            cd = nd - f * cu;
            cu = nu;
            b[i + 1] -= f * b[i];
        } else {
            const double f = cd / nl;
            u0[i] = nl; u1[i] = nd; u2[i] = nu;
            const double bi = b[i];
            b[i] = b[i + 1];
            b[i + 1] = bi - f * b[i + 1];
            cd = cu - f * nd;
            cu = -f * nu;
        }
    }
    u0[n - 1] = cd != 0.0 ? cd : tiny;
    for (int i = n - 1; i >= 0; --i) {
        double s = b[i];
        if (i + 1 < n) s -= u1[i] * b[i + 1];
        if (i + 2 < n) s -= u2[i] * b[i + 2];
        b[i] = s / u0[i];
    }
}

// number of negative pivots of T - lam W
int neg_count(const Tri &T, const Tri &W, double lam)
{
    const int n = (int)T.d.size();
    int c = 0;
    double piv = T.d[0] - lam * W.d[0];
    for (int k = 0;; ++k) {
        if (piv == 0.0) piv = -1e-300;
        if (piv < 0.0) ++c;
        if (k + 1 == n) break;
        const double b = T.u[k] - lam * W.u[k], cc = T.l[k + 1] - lam * W.l[k + 1];
        piv = (T.d[k + 1] - lam * W.d[k + 1]) - b * cc / piv;
    }
    return c;
}

// dense inverse by Gauss-Jordan elimination with partial pivoting; false if singular
bool invert(std::vector<double> A, int n, std::vector<double> &X)
{
    X.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) X[(size_t)i * n + i] = 1.0;
    for (int c = 0; c < n; ++c) {
        int p = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(A[(size_t)r * n + c]) > fabs(A[(size_t)p * n + c])) p = r;
        if (A[(size_t)p * n + c] == 0.0) return false;
        if (p != c)
            for (int k = 0; k < n; ++k) {
                std::swap(A[(size_t)p * n + k], A[(size_t)c * n + k]);
                std::swap(X[(size_t)p * n + k], X[(size_t)c * n + k]);
            }
        const double inv = 1.0 / A[(size_t)c * n + c];
        for (int k = 0; k < n; ++k) { A[(size_t)c * n + k] *= inv; X[(size_t)c * n + k] *= inv; }
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            const double f = A[(size_t)r * n + c];
            if (f == 0.0) continue;
            for (int k = 0; k < n; ++k) {
                A[(size_t)r * n + k] -= f * A[(size_t)c * n + k];
                X[(size_t)r * n + k] -= f * X[(size_t)c * n + k];
            }
        }
    }
    return true;
}

}  // namespace

namespace {
// W = R1 P1 and T = R1 T1 P1 of one axis, accumulated over its fine cells
bool axis_tri(int n, int m, int lo_dir, int hi_dir, bool constant, Tri &W, Tri &T)
{
    for (int i = 0; i < n; ++i) {
        int idx[2], jdx[2];
        double w[2], wj[2];
        const int np = p_row(i, n, m, lo_dir, hi_dir, constant, idx, w);
        const int K = i / m;
        for (int s = 0; s < np; ++s) W.add(K, idx[s], w[s]);
        // row i of T1: in-domain neighbours 1, diagonal -(neighbours) - 2 per Dirichlet face
        double diag = 0.0;
        for (int di = -1; di <= 1; di += 2) {
            const int j = i + di;
            if (j < 0 || j >= n) {
                if ((j < 0 && lo_dir) || (j >= n && hi_dir)) diag -= 2.0;
                continue;
            }
            diag -= 1.0;
            const int npj = p_row(j, n, m, lo_dir, hi_dir, constant, jdx, wj);
            for (int s = 0; s < npj; ++s) T.add(K, jdx[s], wj[s]);
        }
        for (int s = 0; s < np; ++s) T.add(K, idx[s], diag * w[s]);
    }
    return !(W.bad || T.bad);
}
}  // namespace

bool ism_axis_tridiag(int n, int m, int lo, int hi, int kind, double *W3, double *T3)
{
    const int nc = ncoarse(n, m);
    if (nc < 2 || lo == ISM_BC_PERIODIC || hi == ISM_BC_PERIODIC) return false;
    Tri W(nc), T(nc);
    if (!axis_tri(n, m, lo == ISM_BC_DIRICHLET0, hi == ISM_BC_DIRICHLET0, kind == ISM_COARSE_ACM, W, T)) return false;
    for (int k = 0; k < nc; ++k) {
        W3[3 * k] = W.l[k]; W3[3 * k + 1] = W.d[k]; W3[3 * k + 2] = W.u[k];
        T3[3 * k] = T.l[k]; T3[3 * k + 1] = T.d[k]; T3[3 * k + 2] = T.u[k];
    }
    return true;
}

bool ism_axis_factor(int n, int m, int lo, int hi, int kind, IsmAxisFactor &F)
{
    const int nc = ncoarse(n, m);
    if (nc < 2 || lo == ISM_BC_PERIODIC || hi == ISM_BC_PERIODIC) return false;
    const int lo_dir = lo == ISM_BC_DIRICHLET0, hi_dir = hi == ISM_BC_DIRICHLET0;
    Tri W(nc), T(nc);
    if (!axis_tri(n, m, lo_dir, hi_dir, kind == ISM_COARSE_ACM, W, T)) return false;

    // eigenvalues: bracket (-inf, 0], bisection on the pivot count
    double lb = -1.0;
    for (int it = 0; neg_count(T, W, lb) > 0; ++it) {
        if (it > 200) return false;
        lb *= 2.0;
    }
    double scale = fabs(lb);
    const double ub = 1e-14 * scale;
    if (neg_count(T, W, ub) != nc) return false;
    F.lam.assign(nc, 0.0);
    for (int k = 0; k < nc; ++k) {
        double a = lb, b = ub;
        for (int it = 0; it < 200 && b - a > 1e-15 * std::max(fabs(a), fabs(b)) + 1e-300; ++it) {
            const double mid = 0.5 * (a + b);
            if (neg_count(T, W, mid) > k) b = mid;
            else a = mid;
        }
        F.lam[k] = 0.5 * (a + b);
    }
    for (int k = 1; k < nc; ++k)
        if (!(F.lam[k] > F.lam[k - 1])) return false;   // distinct
    // the null mode of the all-Neumann axis is exactly the constant, eigenvalue 0
    if (!lo_dir && !hi_dir && fabs(F.lam[nc - 1]) < 1e-10 * scale) F.lam[nc - 1] = 0.0;

    // eigenvectors: inverse iteration with T - (lam + shift) W
    F.V.assign((size_t)nc * nc, 0.0);
    std::vector<double> dl(nc), dd(nc), du(nc), x(nc), y(nc);
    double tnorm = 0.0;
    for (int k = 0; k < nc; ++k)
        tnorm = std::max(tnorm, fabs(T.l[k]) + fabs(T.d[k]) + fabs(T.u[k]));
    for (int k = 0; k < nc; ++k) {
        const double gap = std::min(k > 0 ? F.lam[k] - F.lam[k - 1] : 1e300,
                                    k + 1 < nc ? F.lam[k + 1] - F.lam[k] : 1e300);
        const double sigma = F.lam[k] + 1e-6 * std::min(gap, scale);
        for (int i = 0; i < nc; ++i) {
            dl[i] = T.l[i] - sigma * W.l[i];
            dd[i] = T.d[i] - sigma * W.d[i];
            du[i] = T.u[i] - sigma * W.u[i];
            x[i] = 1.0 + 0.25 * sin(0.7 * i + 1.3 * k + 0.1);
        }
        for (int it = 0; it < 4; ++it) {
            for (int i = 0; i < nc; ++i)   // y = W x
                y[i] = W.d[i] * x[i] + (i > 0 ? W.l[i] * x[i - 1] : 0.0) + (i + 1 < nc ? W.u[i] * x[i + 1] : 0.0);
            tri_solve(dl, dd, du, y);
            double nrm = 0.0;
            for (int i = 0; i < nc; ++i) nrm += y[i] * y[i];
            nrm = sqrt(nrm);
            if (!(nrm > 0.0) || !isfinite(nrm)) return false;
            for (int i = 0; i < nc; ++i) x[i] = y[i] / nrm;
        }
        // residual check: || T x - lam W x ||_inf <= 1e-9 ||T||
        double res = 0.0;
        for (int i = 0; i < nc; ++i) {
            const double tx = T.d[i] * x[i] + (i > 0 ? T.l[i] * x[i - 1] : 0.0) + (i + 1 < nc ? T.u[i] * x[i + 1] : 0.0);
            const double wx = W.d[i] * x[i] + (i > 0 ? W.l[i] * x[i - 1] : 0.0) + (i + 1 < nc ? W.u[i] * x[i + 1] : 0.0);
            res = std::max(res, fabs(tx - F.lam[k] * wx));
        }
        if (!(res <= 1e-9 * tnorm)) return false;
        for (int i = 0; i < nc; ++i) F.V[(size_t)i * nc + k] = x[i];
    }
    // L = (W V)^-1, checked
    std::vector<double> WV((size_t)nc * nc);
    for (int i = 0; i < nc; ++i)
        for (int k = 0; k < nc; ++k)
            WV[(size_t)i * nc + k] = W.d[i] * F.V[(size_t)i * nc + k] +
                                     (i > 0 ? W.l[i] * F.V[(size_t)(i - 1) * nc + k] : 0.0) +
                                     (i + 1 < nc ? W.u[i] * F.V[(size_t)(i + 1) * nc + k] : 0.0);
    if (!invert(WV, nc, F.L)) return false;
    double err = 0.0;
    for (int i = 0; i < nc; ++i)
        for (int k = 0; k < nc; ++k) {
            double s = 0.0;
            for (int j = 0; j < nc; ++j) s += F.L[(size_t)i * nc + j] * WV[(size_t)j * nc + k];
            err = std::max(err, fabs(s - (i == k ? 1.0 : 0.0)));
        }
    return err <= 1e-8;
}
