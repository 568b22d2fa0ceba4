// ism_core.cu -- setup, control kernels and solve drivers of the ISM library.
//
// The two-level cycle (Sec. 3.4, Fig. 2b; cycle of Sec. 4.3.1 restated with
// an exact coarse solve):
//   r = b - A_f p;  r_c = R r (m x m block sums);  e_c = A_c^+ r_c;
//   p += P e_c (bilinear, Eq. 5);  nu red-black Gauss-Seidel sweeps;
// repeated until ||b - A_f p|| <= tol ||b||.  Convergence is decided on the
// device by one-CTA control kernels, so a chunk of cycles runs as one CUDA
// graph with a single host read of the state per chunk.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "ism_kernels.cuh"
#include "ism_sweep32.cuh"
#include "ism_stream32.cuh"
#include "ism_restrict_stream.cuh"

// Dynamic shared memory of the streaming restriction (m = 8, 16, 32).
template <typename T>
static void restrict_stream_attrs()
{
    const int sm = (int)RestrictShape<T>::smem;
    cudaFuncSetAttribute(k_restrict_stream<T, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_restrict_stream<T, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_restrict_stream<T, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
}

// ================================================================ control

__global__ void __launch_bounds__(256) k_ctl(IsmState *st, const double *partials, int nblk,
                                             int nq, int mode, unsigned long long cond)
{
    __shared__ double S[ISM_NQ];
    if ((mode == CTL_FP64_AFTER || mode == CTL_OUTER_AFTER) && st->done) return;
    if (mode == CTL_INNER && st->inner_done) return;
    ctl_reduce(partials, nblk, nq, S);
    if (threadIdx.x == 0) {
        ctl_decide(st, S, mode);
        ctl_set_condition(st, mode, cond);
    }
}

// ================================================================ rhs preparation

// partial sums of x and |x| (mode 0) or of (x - mean)^2 with y = x - mean
// (mode 1, second column 0)
__global__ void k_rhs_stats(const double *__restrict__ x, double *__restrict__ y, long long n,
                            const IsmState *st, int mode, int sub_mean, double *partials)
{
    double s = 0.0, sa = 0.0;
    const double mu = (mode == 1 && sub_mean) ? st->mean : 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        double v = x[i];
        if (mode == 0) {
            s += v;
            sa += fabs(v);
        } else {
            v -= mu;
            y[i] = v;
            s += v * v;
        }
    }
    double v2[2] = {s, sa};
    block_partials<2>(v2, partials, gridDim.x, blockIdx.x);
}

// ================================================================ mixed-path outer kernels

// FP64 refinement step on the ping-pong pair p0/p1 (st->c64 selects the
// current iterate), in two kernels so that every FP64 operation is done once
// per cell (the FP64 pipe of this GPU is 1/64 of the FP32 rate):
//   k_refine_add:   p_out = p_in + e (e = inner iterate selected by st->cur);
//   k_refine_resid: r = b - A_f p in FP64 on p_out (after an update) or p_in
//                   (first residual), r32 = (float) r, partials
//                   (||r||^2, sum p).
// nx % 4 == 0 (the mixed path's fields are whole float4 groups per row).
__global__ void k_refine_add(double *p0, double *p1, const float *e0, const float *e1, long long n4,
                             const IsmState *st)
{
    const float4 *__restrict__ e = reinterpret_cast<const float4 *>(st->cur ? e1 : e0);
    const double2 *__restrict__ pi = reinterpret_cast<const double2 *>(st->c64 ? p1 : p0);
    double2 *__restrict__ po = reinterpret_cast<double2 *>(st->c64 ? p0 : p1);
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n4;
         k += (long long)gridDim.x * blockDim.x) {
        const float4 ev = e[k];
        const double2 a = pi[2 * k], c = pi[2 * k + 1];
        po[2 * k] = make_double2(a.x + (double)ev.x, a.y + (double)ev.y);
        po[2 * k + 1] = make_double2(c.x + (double)ev.z, c.y + (double)ev.w);
    }
}

constexpr int RF_ROWS = 4;       // rows per thread of k_refine_resid
constexpr int RF_THREADS = 128;  // 4 columns each

// One thread: 4 adjacent columns of RF_ROWS rows.  The neighbour sum takes
// the terms in the order west, east, south, north with 0 for a wall face
// (x + 0 == x: the same value as the sum over in-domain neighbours).
__global__ void __launch_bounds__(RF_THREADS) k_refine_resid(const double *p0, const double *p1,
                                                             const double *__restrict__ b, float *__restrict__ r32,
                                                             double *partials, int nx, int ny, int bcmask,
                                                             const IsmState *st, int after_update)
{
    const double *__restrict__ p = (after_update ? !st->c64 : st->c64) ? p1 : p0;
    const int i = 4 * (blockIdx.x * RF_THREADS + threadIdx.x);
    const int j0 = blockIdx.y * RF_ROWS;
    const bool per_x = (bcmask & ISM_PER_X) != 0, per_y = (bcmask & ISM_PER_Y) != 0;
    double r2 = 0.0, ps = 0.0;
    if (i < nx) {
        // west / east neighbours of the 4-column group
        const bool hasw = i > 0 || per_x, hase = i + 4 < nx || per_x;
        const int iw = i > 0 ? i - 1 : nx - 1, ie = i + 4 < nx ? i + 4 : 0;
        // diagonal count per column without the south / north faces
        double dcol[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int d = 4;
            if (!per_x && i + q == 0) d += (bcmask & 1) ? 1 : -1;
            if (!per_x && i + q == nx - 1) d += (bcmask & 2) ? 1 : -1;
            dcol[q] = (double)d;
        }
        for (int jj = 0; jj < RF_ROWS; ++jj) {
            const int j = j0 + jj;
            if (j >= ny) break;
            const bool hass = j > 0 || per_y, hasn = j < ny - 1 || per_y;
            const int js = j > 0 ? j - 1 : ny - 1, jn = j < ny - 1 ? j + 1 : 0;
            const double *row = p + (size_t)j * nx;
            const double2 c01 = *reinterpret_cast<const double2 *>(row + i);
            const double2 c23 = *reinterpret_cast<const double2 *>(row + i + 2);
            double2 s01 = make_double2(0.0, 0.0), s23 = s01, n01 = s01, n23 = s01;
            if (hass) {
                s01 = *reinterpret_cast<const double2 *>(p + (size_t)js * nx + i);
                s23 = *reinterpret_cast<const double2 *>(p + (size_t)js * nx + i + 2);
            }
            if (hasn) {
                n01 = *reinterpret_cast<const double2 *>(p + (size_t)jn * nx + i);
                n23 = *reinterpret_cast<const double2 *>(p + (size_t)jn * nx + i + 2);
            }
            const double w = hasw ? row[iw] : 0.0, e = hase ? row[ie] : 0.0;
            const double pc[4] = {c01.x, c01.y, c23.x, c23.y};
            const double so[4] = {s01.x, s01.y, s23.x, s23.y};
            const double no[4] = {n01.x, n01.y, n23.x, n23.y};
            const double2 b01 = *reinterpret_cast<const double2 *>(b + (size_t)j * nx + i);
            const double2 b23 = *reinterpret_cast<const double2 *>(b + (size_t)j * nx + i + 2);
            const double bv[4] = {b01.x, b01.y, b23.x, b23.y};
            // south / north wall faces of this row (uniform across the block)
            int drow = 0;
            if (!per_y && j == 0) drow += (bcmask & 4) ? 1 : -1;
            if (!per_y && j == ny - 1) drow += (bcmask & 8) ? 1 : -1;
            float rr[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const double lf = q == 0 ? w : pc[q - 1], rt = q == 3 ? e : pc[q + 1];
                const double d = drow ? dcol[q] + (double)drow : dcol[q];
                const double sum = ((lf + rt) + so[q]) + no[q];
                const double r = bv[q] - (sum - d * pc[q]);
                rr[q] = (float)r;
                r2 = fma(r, r, r2);
                ps += pc[q];
            }
            *reinterpret_cast<float4 *>(r32 + (size_t)j * nx + i) = make_float4(rr[0], rr[1], rr[2], rr[3]);
        }
    }
    double v[2] = {r2, ps};
    block_partials<2>(v, partials, gridDim.x * gridDim.y, blockIdx.y * gridDim.x + blockIdx.x);
}

static inline dim3 refine_grid(int nx, int ny)
{
    return dim3((nx / 4 + RF_THREADS - 1) / RF_THREADS, (ny + RF_ROWS - 1) / RF_ROWS);
}

// Norms of the residual r = rhs - A_f p (FP64) of a given iterate: per block
// the sum of r^2 (fixed order) and max |r| (a non-finite residual counts as
// +inf), written to partials[blk] and partials[nblk + blk].  Grid
// (ceil(nx/256), ny).
__global__ void __launch_bounds__(256) k_resnorms(const double *__restrict__ p, const double *__restrict__ b,
                                                  double *partials, int nx, int ny, int bcmask)
{
    const int j = blockIdx.y, i = blockIdx.x * blockDim.x + threadIdx.x;
    double r2 = 0.0, rm = 0.0;
    if (i < nx) {
        const size_t idx = (size_t)j * nx + i;
        const double s = nb_sum<double>([&](long long k) -> double { return p[k]; }, (long long)idx, i, j, nx, ny,
                                        bcmask);
        const double r = b[idx] - (s - (double)diag_count(i, j, nx, ny, bcmask) * p[idx]);
        r2 = r * r;
        rm = isfinite(r) ? fabs(r) : INFINITY;
    }
    __shared__ double mx[8];
    double m = rm;
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(FULLMASK, m, o));
    if ((threadIdx.x & 31) == 0) mx[threadIdx.x >> 5] = m;
    const int nblk = gridDim.x * gridDim.y, bid = blockIdx.y * gridDim.x + blockIdx.x;
    double v[1] = {r2};
    block_partials<1>(v, partials, nblk, bid);      // its barriers also publish mx[]
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t = fmax(t, mx[k]);
        partials[(size_t)nblk + bid] = t;
    }
}

// out = in - mean (mean of the final iterate when all faces are Neumann);
// zeros when the right-hand side vanished.  in_alt replaces in when st->c64.
__global__ void k_finalize(const double *in, const double *in_alt, double *out, long long n,
                           const IsmState *st, int sub_mean)
{
    if (in_alt && st->c64) in = in_alt;
    const double mu = sub_mean ? st->mean : 0.0;
    const bool zero = st->zero_rhs != 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = zero ? 0.0 : in[i] - mu;
}

// ================================================================ host: setup

extern "C" const char *ism_status_str(ism_status s)
{
    switch (s) {
    case ISM_OK: return "ok";
    case ISM_ERR_ARG: return "invalid argument";
    case ISM_ERR_NOT_CONVERGED: return "not converged";
    case ISM_ERR_NONFINITE: return "non-finite value";
    case ISM_ERR_CUDA: return "CUDA error";
    case ISM_ERR_NOMEM: return "out of memory";
    }
    return "unknown status";
}

static void default_options(ism_options *o, int prec)
{
    // FP64: 8 sweeps per cycle (the reading used by the oracle).  Mixed: 64
    // sweeps per cycle in eight fused passes of 8 -- the total number of
    // sweeps to a given tolerance hardly depends on nu, while every cycle adds
    // a fixed cost (coarse solve, fused prolongation and residual, control).
    o->nu = prec == ISM_MIXED ? 64 : 8;
    o->sweeps_per_pass = prec == ISM_MIXED ? 8 : 4;
    o->kind = ISM_COARSE_ISM;
    o->max_outer = 50;
    o->inner_max = 10000;
    o->inner_tol = 1e-3;
    o->floor_mult = 4.0;
    o->check_every = 16;
    o->use_graphs = 2;
    o->coarse_tc = prec == ISM_MIXED ? 1 : 0;
    o->cycle = 0;
    o->accom_tol_c = 1e-5;
    o->accom_max_coarse = 100000;
    o->stream = 0;
    o->fault_test = 0;
    o->tile_rows = 128;
    o->packed = 2;
}

static const double kPi = 3.14159265358979323846;

// Eigenbasis of S = tridiag(1, 2, 1) of size n with end diagonals 3 (Neumann)
// or 1 (Dirichlet-0): with the ghost x_{-1} = +-x_0 and x_n = +-x_{n-1},
// (S x)_i = x_{i-1} + 2 x_i + x_{i+1} everywhere, so the cosine/sine modes
// below are eigenvectors with eigenvalue 2 + 2 cos(theta):
//   N-N: cos(theta (i+1/2)), theta = pi k / n          (DCT-II)
//   D-D: sin(theta (i+1/2)), theta = pi (k+1) / n      (DST-II)
//   N-D: cos(theta (i+1/2)), theta = pi (k+1/2) / n    (DCT-IV)
//   D-N: sin(theta (i+1/2)), theta = pi (k+1/2) / n    (DST-IV)
// On a periodic axis S is circulant, diagonalised by the real Fourier modes
// (n even): column 0 the constant, columns 2t-1, 2t (t = 1..n/2-1)
// cos(theta i), sin(theta i) with theta = 2 pi t / n, column n-1 (-1)^i;
// eigenvalue 2 + 2 cos(theta) (0 for the last).
// Q[i*n + k] is component i of unit eigenvector k.  lo, hi: ism_bc of the
// two ends.
static void s_eigen(int n, int lo, int hi, std::vector<double> &Q, std::vector<double> &lam)
{
    Q.assign((size_t)n * n, 0.0);
    lam.assign(n, 0.0);
    if (lo == ISM_BC_PERIODIC) {
        for (int k = 0; k < n; ++k) {
            const int t = (k + 1) / 2;                 // frequency of column k
            const double th = 2.0 * kPi * t / n;
            lam[k] = 2.0 + 2.0 * cos(th);
            double nrm = 0.0;
            for (int i = 0; i < n; ++i) {
                const double v = (k == 0) ? 1.0 : (k == n - 1) ? ((i & 1) ? -1.0 : 1.0)
                                 : (k & 1) ? cos(th * i) : sin(th * i);
                Q[(size_t)i * n + k] = v;
                nrm += v * v;
            }
            nrm = 1.0 / sqrt(nrm);
            for (int i = 0; i < n; ++i) Q[(size_t)i * n + k] *= nrm;
        }
        lam[n - 1] = 0.0;                              // 2 + 2 cos(pi), exactly
        return;
    }
    const int lo_dir = lo == ISM_BC_DIRICHLET0, hi_dir = hi == ISM_BC_DIRICHLET0;
    for (int k = 0; k < n; ++k) {
        double th;
        bool use_sin = lo_dir != 0;
        if (!lo_dir && !hi_dir) th = kPi * k / n;
        else if (lo_dir && hi_dir) th = kPi * (k + 1) / n;
        else th = kPi * (k + 0.5) / n;
        lam[k] = 2.0 + 2.0 * cos(th);
        double nrm = 0.0;
        for (int i = 0; i < n; ++i) {
            double v = use_sin ? sin(th * (i + 0.5)) : cos(th * (i + 0.5));
            Q[(size_t)i * n + k] = v;
            nrm += v * v;
        }
        nrm = 1.0 / sqrt(nrm);
        for (int i = 0; i < n; ++i) Q[(size_t)i * n + k] *= nrm;
    }
}

// The coarse solve e_c = A_c^+ r_c in the four-product form
// E = Qy [(QyT R Qx) . Minv] QxT (R, E: ncy x ncx row-major).
struct EigenHost {
    std::vector<double> Qx, QxT, Qy, QyT, Minv;
};

static void transpose(const std::vector<double> &A, int n, std::vector<double> &At)
{
    At.resize((size_t)n * n);
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k) At[(size_t)k * n + i] = A[(size_t)i * n + k];
}

// Uniform coarse cells: eigenvalues of A_c on the orthonormal (Qy x Qx):
// ISM A_c = 1/4 (S_y x S_x) - 4 I (closed form of summing the Eq. 6-7 face
// fluxes), ACM A_c = m (T_y (+) T_x) with T = S - 4 I (the five-point coarse
// operator of the summed equations), GMG the same without the factor m.
static EigenHost eigen_uniform(const ism_ctx *ctx, int kind)
{
    EigenHost E;
    std::vector<double> lx, ly;
    s_eigen(ctx->ncx, ctx->bc[0], ctx->bc[1], E.Qx, lx);
    s_eigen(ctx->ncy, ctx->bc[2], ctx->bc[3], E.Qy, ly);
    const int ncx = ctx->ncx, ncy = ctx->ncy;
    transpose(E.Qx, ncx, E.QxT);
    transpose(E.Qy, ncy, E.QyT);
    E.Minv.resize((size_t)ncx * ncy);
    for (int l = 0; l < ncy; ++l)
        for (int k = 0; k < ncx; ++k) {
            double mu = (kind == ISM_COARSE_ISM) ? 0.25 * lx[k] * ly[l] - 4.0 : (lx[k] - 4.0) + (ly[l] - 4.0);
            if (kind == ISM_COARSE_ACM || kind == ISM_COARSE_ACMV) mu *= ctx->m;
            E.Minv[(size_t)l * ncx + k] = fabs(mu) < 1e-10 ? 0.0 : 1.0 / mu;
        }
    return E;
}

// 1-D factor T V = W V diag(lam), L = (W V)^-1 of one axis (see ism_pencil.cu).
// A periodic axis (a multiple of m) in closed form: V = Q (Fourier basis of S),
// W = m (S + 4 I) / 8 and T = (S - 4 I) / m for ISM, W = m I and T = S - 4 I
// for ACM, so lam = t / w and L = diag(1 / w) Q^T.
static bool axis_factor(const ism_ctx *ctx, int n, int lo, int hi, int kind, IsmAxisFactor &F)
{
    if (lo != ISM_BC_PERIODIC) return ism_axis_factor(n, ctx->m, lo, hi, kind, F);
    const int nc = n / ctx->m;
    const double m = ctx->m;
    std::vector<double> s;
    s_eigen(nc, lo, hi, F.V, s);
    F.lam.resize(nc);
    F.L.resize((size_t)nc * nc);
    for (int k = 0; k < nc; ++k) {
        const double w = (kind == ISM_COARSE_ISM) ? m * (s[k] + 4.0) / 8.0 : m;
        const double t = (kind == ISM_COARSE_ISM) ? (s[k] - 4.0) / m : s[k] - 4.0;
        F.lam[k] = t / w;
        for (int i = 0; i < nc; ++i) F.L[(size_t)k * nc + i] = F.V[(size_t)i * nc + k] / w;
    }
    return true;
}

// A narrower last coarse cell along an axis: A_c = W_y x T_x + T_y x W_x, so
// A_c^+ = (V_y x V_x) diag(1 / (lam_y + lam_x)) (L_y x L_x) with the null mode
// (every face Neumann or periodic: lam_y + lam_x = 0 for the constants) dropped.
static bool eigen_general(const ism_ctx *ctx, int kind, EigenHost &E)
{
    IsmAxisFactor fx, fy;
    if (!axis_factor(ctx, ctx->nx, ctx->bc[0], ctx->bc[1], kind, fx) ||
        !axis_factor(ctx, ctx->ny, ctx->bc[2], ctx->bc[3], kind, fy))
        return false;
    const int ncx = ctx->ncx, ncy = ctx->ncy;
    transpose(fx.L, ncx, E.Qx);   // R Qx = R L_x^T
    transpose(fx.V, ncx, E.QxT);
    E.Qy = fy.V;
    E.QyT = fy.L;
    double mx = 0.0;
    for (int l = 0; l < ncy; ++l)
        for (int k = 0; k < ncx; ++k) mx = std::max(mx, fabs(fy.lam[l] + fx.lam[k]));
    E.Minv.resize((size_t)ncx * ncy);
    for (int l = 0; l < ncy; ++l)
        for (int k = 0; k < ncx; ++k) {
            const double mu = fy.lam[l] + fx.lam[k];
            E.Minv[(size_t)l * ncx + k] = fabs(mu) <= 1e-12 * mx ? 0.0 : 1.0 / mu;
        }
    return true;
}

static ism_status build_eigen(const ism_ctx *ctx, int kind, EigenHost &E)
{
    if (!ctx->ragged) {
        E = eigen_uniform(ctx, kind);
        return ISM_OK;
    }
    return eigen_general(ctx, kind, E) ? ISM_OK : ISM_ERR_ARG;
}

static ism_status upload_coarse(ism_ctx *ctx, const EigenHost &E)
{
    auto up = [&](double *d64, float *d32, const std::vector<double> &h) -> ism_status {
        std::vector<float> f(h.size());
        for (size_t i = 0; i < h.size(); ++i) f[i] = (float)h[i];
        ISM_CUDA_TRY(cudaMemcpy(d64, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice));
        ISM_CUDA_TRY(cudaMemcpy(d32, f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice));
        return ISM_OK;
    };
    ism_status s;
    if ((s = up(ctx->Qx64, ctx->Qx32, E.Qx)) != ISM_OK) return s;
    if ((s = up(ctx->QxT64, ctx->QxT32, E.QxT)) != ISM_OK) return s;
    if ((s = up(ctx->Qy64, ctx->Qy32, E.Qy)) != ISM_OK) return s;
    if ((s = up(ctx->QyT64, ctx->QyT32, E.QyT)) != ISM_OK) return s;
    if ((s = up(ctx->Minv64, ctx->Minv32, E.Minv)) != ISM_OK) return s;
    return ism_coarse_tc_upload(ctx, E.Qx, E.QxT, E.Qy, E.QyT, E.Minv);
}

static void free_graphs(ism_ctx *ctx)
{
    if (ctx->g_fp64) cudaGraphExecDestroy(ctx->g_fp64);
    if (ctx->g_inner) cudaGraphExecDestroy(ctx->g_inner);
    if (ctx->gc_fp64) cudaGraphExecDestroy(ctx->gc_fp64);
    if (ctx->gc_mixed) cudaGraphExecDestroy(ctx->gc_mixed);
    ctx->g_fp64 = ctx->g_inner = ctx->gc_fp64 = ctx->gc_mixed = nullptr;
}

void ism_batch_free(void *plan);   // ism_batched.cu

extern "C" void ism_destroy(ism_ctx *ctx)
{
    if (!ctx) return;
    if (ctx->batch) ism_batch_free(ctx->batch);
    if (ctx->ws) cudaStreamSynchronize(ctx->ws);
    if (ctx->ws2) cudaStreamSynchronize(ctx->ws2);
    free_graphs(ctx);
    void *bufs[] = {ctx->Qx64, ctx->QxT64, ctx->Qy64, ctx->QyT64, ctx->Minv64, ctx->Qx32,
                    ctx->QxT32, ctx->Qy32, ctx->QyT32, ctx->Minv32, ctx->b64, ctx->p64[0],
                    ctx->p64[1], ctx->e32[0], ctx->e32[1], ctx->r32, ctx->rc64, ctx->ec64,
                    ctx->T64, ctx->rc32, ctx->ec32, ctx->T32, ctx->partials, ctx->st,
                    ctx->st_k, ctx->us, ctx->vs, ctx->dp, ctx->rcpart, ctx->roll, ctx->scal,
                    ctx->tc_block, ctx->tct_block, ctx->G64, ctx->ac_tri};
    for (void *b : bufs)
        if (b) cudaFree(b);
    for (int l = 0; l < 6; ++l) {
        if (ctx->lvl_r[l]) cudaFree(ctx->lvl_r[l]);
        if (ctx->lvl_e[l]) cudaFree(ctx->lvl_e[l]);
    }
    for (int K = 0; K <= SMAXK; ++K)
        for (int r = 0; r < 2; ++r)
            for (int t = 0; t < 2; ++t)
                if (ctx->plans[t][K][r].edge) cudaFree(ctx->plans[t][K][r].edge);
    if (ctx->st_host) cudaFreeHost(ctx->st_host);
    if (ctx->ev_in) cudaEventDestroy(ctx->ev_in);
    if (ctx->ev_out) cudaEventDestroy(ctx->ev_out);
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
    if (ctx->ws2) cudaStreamDestroy(ctx->ws2);
    if (ctx->ws) cudaStreamDestroy(ctx->ws);
    free(ctx);
}

static ism_status make_plans(ism_ctx *ctx);

// Dynamic shared memory of every fused-pass kernel of a region of NW warps.
template <int NW>
static void set_sweep_smem()
{
    const int smb = (int)sweep_smem_bytes(NW);
    cudaFuncSetAttribute(k_sweep32<NW, true, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smb);
    cudaFuncSetAttribute(k_sweep32<NW, true, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smb);
    cudaFuncSetAttribute(k_sweep32<NW, false, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smb);
    cudaFuncSetAttribute(k_sweep32<NW, false, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smb);
    cudaFuncSetAttribute(k_sweep32<NW, true, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smb);
    cudaFuncSetAttribute(k_sweep32<NW, true, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smb);
    cudaFuncSetAttribute(k_sweep32<NW, false, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smb);
    cudaFuncSetAttribute(k_sweep32<NW, false, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smb);
    cudaFuncSetAttribute(k_sweep32<NW, true, true, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smb);
    cudaFuncSetAttribute(k_sweep32<NW, true, false, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smb);
    cudaFuncSetAttribute(k_sweep32<NW, false, true, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smb);
    cudaFuncSetAttribute(k_sweep32<NW, false, false, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smb);
}


ism_status ism_setup_fixed(int nx, int ny, double h, const int bc[4], int coarsen, ism_precision prec,
                           void *stream, ism_ctx **out)
{
    if (!out || !bc) return ISM_ERR_ARG;
    if (coarsen != 8 && coarsen != 16 && coarsen != 32) return ISM_ERR_ARG;
    if (nx < coarsen || ny < coarsen) return ISM_ERR_ARG;
    if ((long long)nx * ny > (1LL << 31) || nx > (1 << 20) || ny > (1 << 20)) return ISM_ERR_ARG;
    const int ncx = (nx + coarsen - 1) / coarsen, ncy = (ny + coarsen - 1) / coarsen;
    if (ncx > 1024 || ncy > 1024) return ISM_ERR_ARG;
    const bool ragged = nx % coarsen || ny % coarsen;
    // a narrower last coarse cell needs a full one before it; the single-precision
    // pass moves aligned groups of 4 cells along x
    if ((nx % coarsen && ncx < 2) || (ny % coarsen && ncy < 2)) return ISM_ERR_ARG;
    if (prec == ISM_MIXED && nx % 4) return ISM_ERR_ARG;
    if (!(h > 0.0) || !isfinite(h)) return ISM_ERR_ARG;
    const int mask = ism_bc_mask(bc);
    if (mask < 0) return ISM_ERR_ARG;
    if ((mask & ISM_PER_X) && (nx % coarsen || ncx < 4)) return ISM_ERR_ARG;
    if ((mask & ISM_PER_Y) && (ny % coarsen || ncy < 4)) return ISM_ERR_ARG;
    if (prec != ISM_FP64 && prec != ISM_MIXED) return ISM_ERR_ARG;

    ism_ctx *ctx = (ism_ctx *)calloc(1, sizeof(ism_ctx));
    if (!ctx) return ISM_ERR_NOMEM;
    ctx->nx = nx;
    ctx->ny = ny;
    ctx->m = coarsen;
    ctx->ncx = ncx;
    ctx->ncy = ncy;
    ctx->ragged = ragged;
    ctx->n = (long long)nx * ny;
    ctx->h = h;
    ctx->bcmask = mask;
    for (int f = 0; f < 4; ++f) ctx->bc[f] = bc[f];
    ctx->singular = (mask & 15) == 0;
    {
        static unsigned long long next_uid = 1;
        ctx->uid = __atomic_fetch_add(&next_uid, 1ULL, __ATOMIC_RELAXED);
    }
    ctx->prec = prec;
    ctx->user_stream = (cudaStream_t)stream;
    default_options(&ctx->opt, prec);
    ctx->proj_tol = 1e-8;
    ctx->proj_max_cycles = 100000;
    ctx->conv_u = 1.0;

    const size_t N = (size_t)ctx->n, nc = (size_t)ctx->ncx * ctx->ncy;
    const int tiles = ((nx + sweep_tile_w(SMAXK, true) - 1) / sweep_tile_w(SMAXK, true)) *
                      ((ny + sweep_tile_h(SMAXK, true) - 1) / sweep_tile_h(SMAXK, true));   // largest tile grid
    ctx->max_blocks = std::max({(int)nc, tiles, ((nx + 255) / 256) * ny, 1024});

#define ALLOC(ptr, bytes)                                                        \
    do {                                                                         \
        if (cudaMalloc((void **)&(ptr), (bytes)) != cudaSuccess) {               \
            cudaGetLastError();                                                  \
            ism_destroy(ctx);                                                    \
            return ISM_ERR_NOMEM;                                                \
        }                                                                        \
    } while (0)
    const size_t ncx2 = (size_t)ctx->ncx * ctx->ncx, ncy2 = (size_t)ctx->ncy * ctx->ncy;
    ALLOC(ctx->Qx64, ncx2 * 8); ALLOC(ctx->QxT64, ncx2 * 8);
    ALLOC(ctx->Qy64, ncy2 * 8); ALLOC(ctx->QyT64, ncy2 * 8);
    ALLOC(ctx->Minv64, nc * 8);
    ALLOC(ctx->Qx32, ncx2 * 4); ALLOC(ctx->QxT32, ncx2 * 4);
    ALLOC(ctx->Qy32, ncy2 * 4); ALLOC(ctx->QyT32, ncy2 * 4);
    ALLOC(ctx->Minv32, nc * 4);
    ALLOC(ctx->b64, N * 8);
    ALLOC(ctx->p64[0], N * 8);
    ALLOC(ctx->rc64, nc * 8); ALLOC(ctx->ec64, nc * 8); ALLOC(ctx->T64, nc * 8);
    ALLOC(ctx->rc32, nc * 4); ALLOC(ctx->ec32, nc * 4); ALLOC(ctx->T32, nc * 4);
    ALLOC(ctx->rcpart, nc * 4 * 4);
    if (prec == ISM_FP64) ALLOC(ctx->G64, (size_t)ctx->ncy * nx * 8);
    if (prec == ISM_MIXED) {
        ALLOC(ctx->p64[1], N * 8);
        ALLOC(ctx->e32[0], N * 4);
        ALLOC(ctx->e32[1], N * 4);
        ALLOC(ctx->r32, N * 4);
    }
    ALLOC(ctx->partials, (size_t)ISM_NQ * ctx->max_blocks * 8);
    ALLOC(ctx->st, sizeof(IsmState));
    ALLOC(ctx->st_k, sizeof(IsmState));
#undef ALLOC
    if (cudaMallocHost((void **)&ctx->st_host, sizeof(IsmState)) != cudaSuccess) {
        cudaGetLastError();
        ism_destroy(ctx);
        return ISM_ERR_NOMEM;
    }
    if (cudaStreamCreateWithFlags(&ctx->ws, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&ctx->ws2, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_out, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        ism_destroy(ctx);
        return ISM_ERR_CUDA;
    }
    if (cudaMemset(ctx->st, 0, sizeof(IsmState)) != cudaSuccess ||
        cudaMemset(ctx->st_k, 0, sizeof(IsmState)) != cudaSuccess) {
        ism_destroy(ctx);
        return ISM_ERR_CUDA;
    }
    EigenHost E;
    ism_status s = build_eigen(ctx, ctx->opt.kind, E);
    if (s == ISM_OK) s = upload_coarse(ctx, E);
    if (s != ISM_OK) {
        ism_destroy(ctx);
        return s;
    }
    // the fused sweep pass uses 91 KB (128-row region) or 180 KB (256-row)
    // of dynamic shared memory
    ism_coarse_tc_prepare();
    restrict_stream_attrs<float>();
    restrict_stream_attrs<double>();
    set_sweep_smem<8>();
    set_sweep_smem<16>();
    if ((s = make_plans(ctx)) != ISM_OK) {
        ism_destroy(ctx);
        return s;
    }
    if (cudaDeviceSynchronize() != cudaSuccess) {
        ism_destroy(ctx);
        return ISM_ERR_CUDA;
    }
    *out = ctx;
    return ISM_OK;
}

extern "C" ism_status ism_get_options(const ism_ctx *ctx, ism_options *opt)
{
    if (!ctx || !opt) return ISM_ERR_ARG;
    *opt = ctx->opt;
    return ISM_OK;
}

extern "C" ism_status ism_set_options(ism_ctx *ctx, const ism_options *o)
{
    if (!ctx || !o) return ISM_ERR_ARG;
    if (o->nu < 1 || o->nu > 256) return ISM_ERR_ARG;
    if (o->sweeps_per_pass < 1 || o->sweeps_per_pass > SMAXK || o->nu % o->sweeps_per_pass) return ISM_ERR_ARG;
    if (o->kind < ISM_COARSE_ISM || o->kind > ISM_COARSE_ACMV) return ISM_ERR_ARG;
    if (o->kind == ISM_COARSE_ACMV && ctx->prec != ISM_FP64) return ISM_ERR_ARG;
    if (o->max_outer < 1 || o->inner_max < 1 || o->check_every < 1 || o->check_every > 4096) return ISM_ERR_ARG;
    if (o->use_graphs < 0 || o->use_graphs > 2) return ISM_ERR_ARG;
    if (o->coarse_tc < 0 || o->coarse_tc > 2) return ISM_ERR_ARG;
    if (o->cycle < 0 || o->cycle > 1) return ISM_ERR_ARG;
    if (o->cycle == 1 && (ctx->prec != ISM_FP64 || o->kind != ISM_COARSE_ISM)) return ISM_ERR_ARG;
    // the four-colour coarse Gauss-Seidel needs an even coarse count along a periodic axis
    if (o->cycle == 1 && (((ctx->bcmask & ISM_PER_X) && (ctx->ncx & 1)) || ((ctx->bcmask & ISM_PER_Y) && (ctx->ncy & 1))))
        return ISM_ERR_ARG;
    if (!(o->accom_tol_c > 0.0) || o->accom_max_coarse < 1) return ISM_ERR_ARG;
    if (o->stream < 0 || o->stream > 1) return ISM_ERR_ARG;
    if (o->fault_test < 0 || o->fault_test > 1) return ISM_ERR_ARG;
    if (o->tile_rows != 128 && o->tile_rows != 256) return ISM_ERR_ARG;
    if (o->packed < 0 || o->packed > 2) return ISM_ERR_ARG;
    if (!(o->inner_tol > 0.0 && o->inner_tol < 1.0) || !(o->floor_mult >= 0.0)) return ISM_ERR_ARG;
    // a narrower last coarse cell: the ISM and ACM operators; the accommodative
    // cycle with walls only (its coarse coefficients come from the 1-D W, T)
    if (ctx->ragged && (o->kind == ISM_COARSE_GMG || o->kind == ISM_COARSE_ACMV)) return ISM_ERR_ARG;
    if (ctx->ragged && o->cycle == 1 && (ctx->bcmask & (ISM_PER_X | ISM_PER_Y))) return ISM_ERR_ARG;
    const int kind_changed = o->kind != ctx->opt.kind;
    EigenHost E;
    if (kind_changed && build_eigen(ctx, o->kind, E) != ISM_OK) return ISM_ERR_ARG;
    cudaStreamSynchronize(ctx->ws);
    if (o->kind == ISM_COARSE_ACMV && !ctx->lvl_r[1]) {
        // levels 1 .. L-1 of the V-cycle (level l: (nx >> l) x (ny >> l))
        for (int l = 1; (1 << l) < ctx->m; ++l) {
            const size_t b = (size_t)(ctx->nx >> l) * (ctx->ny >> l) * 8;
            if (cudaMalloc((void **)&ctx->lvl_r[l], b) != cudaSuccess ||
                cudaMalloc((void **)&ctx->lvl_e[l], b) != cudaSuccess) {
                cudaGetLastError();
                return ISM_ERR_NOMEM;
            }
        }
    }
    if (o->cycle == 1 && ctx->ragged && !ctx->ac_tri) {
        const int ncx = ctx->ncx, ncy = ctx->ncy;
        std::vector<double> t(6 * (size_t)(ncx + ncy));
        if (!ism_axis_tridiag(ctx->nx, ctx->m, ctx->bc[0], ctx->bc[1], ISM_COARSE_ISM, t.data(), t.data() + 3 * ncx) ||
            !ism_axis_tridiag(ctx->ny, ctx->m, ctx->bc[2], ctx->bc[3], ISM_COARSE_ISM, t.data() + 6 * ncx,
                              t.data() + 6 * ncx + 3 * ncy))
            return ISM_ERR_ARG;
        if (cudaMalloc((void **)&ctx->ac_tri, t.size() * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            ctx->ac_tri = nullptr;
            return ISM_ERR_NOMEM;
        }
        ISM_CUDA_TRY(cudaMemcpy(ctx->ac_tri, t.data(), t.size() * sizeof(double), cudaMemcpyHostToDevice));
    }
    ctx->opt = *o;
    ctx->opt_gen++;
    free_graphs(ctx);
    if (kind_changed) return upload_coarse(ctx, E);
    return ISM_OK;
}

ism_status ism_enter(ism_ctx *ctx)
{
    ISM_CUDA_TRY(cudaEventRecord(ctx->ev_in, ctx->user_stream));
    ISM_CUDA_TRY(cudaStreamWaitEvent(ctx->ws, ctx->ev_in, 0));
    return ISM_OK;
}

ism_status ism_leave(ism_ctx *ctx)
{
    ISM_CUDA_TRY(cudaEventRecord(ctx->ev_out, ctx->ws));
    ISM_CUDA_TRY(cudaStreamWaitEvent(ctx->user_stream, ctx->ev_out, 0));
    return ISM_OK;
}

// ================================================================ host: launch helpers

static inline dim3 row_grid(int nx, int ny, int threads) { return dim3((nx + threads - 1) / threads, ny); }

// e_c = A_c^+ r_c.  FUSED (single precision inside the cycle): r_c is read as
// the sum of the 4 partial block sums and the x-interpolated rows G are made.
template <typename T, bool FUSED>
static ism_status launch_coarse(ism_ctx *ctx, const T *rc, T *ec, T *Tm, const int *skip)
{
    const T *Qx, *QxT, *Qy, *QyT, *Minv;
    if (sizeof(T) == 8) {
        Qx = (const T *)ctx->Qx64; QxT = (const T *)ctx->QxT64;
        Qy = (const T *)ctx->Qy64; QyT = (const T *)ctx->QyT64; Minv = (const T *)ctx->Minv64;
    } else {
        Qx = (const T *)ctx->Qx32; QxT = (const T *)ctx->QxT32;
        Qy = (const T *)ctx->Qy32; QyT = (const T *)ctx->QyT32; Minv = (const T *)ctx->Minv32;
    }
    const int th = 256;
    const int JS = ctx->ncx >= th ? 1 : th / ctx->ncx;
    const size_t sm = (size_t)(JS + 2) * ctx->ncx * sizeof(T);
    k_coarse1<T, FUSED><<<ctx->ncy, th, sm, ctx->ws>>>(rc, QyT, Qx, Minv, Tm, ctx->ncx, ctx->ncy, skip);
    ISM_LAUNCH_CHECK(ctx);
    k_coarse2<T, FUSED><<<ctx->ncy, th, sm, ctx->ws>>>(Tm, Qy, QxT, ec, ctx->ncx, ctx->ncy, skip,
                                                       (T *)(FUSED ? (void *)ctx->rcpart : nullptr));
    ISM_LAUNCH_CHECK(ctx);
    return ISM_OK;
}

// Streaming restriction for one m: strips of 128 columns and chunks of rows
// (multiples of m) sized to fill the resident warps once.  Returns the number
// of CTAs, or 0 when that exceeds the norm-partial slots.
template <typename T, int M>
static int launch_restrict_stream(ism_ctx *ctx, const T *p, const T *b, T *rc, const int *skip, int ctl_mode,
                                  unsigned long long cond)
{
    using S = RestrictShape<T>;
    static int slots = 0;                        // resident warps on the device
    if (!slots) {
        int dev = 0, sms = 152, per_sm = 1;
        if (cudaGetDevice(&dev) == cudaSuccess)
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_restrict_stream<T, M>, 32 * RR_NW, S::smem) !=
                cudaSuccess || per_sm < 1)
            per_sm = 1;
        cudaGetLastError();
        slots = sms * per_sm * RR_NW;
    }
    const int nstrip = (ctx->nx + SRW - 1) / SRW;
    const int nchunk = std::max(1, slots / nstrip);
    int chunk_h = (ctx->ny + nchunk - 1) / nchunk;
    chunk_h = ((chunk_h + M - 1) / M) * M;       // whole coarse rows
    const int ntask = nstrip * ((ctx->ny + chunk_h - 1) / chunk_h);
    const int grid = (ntask + RR_NW - 1) / RR_NW;
    if (grid > ctx->max_blocks) return 0;
    k_restrict_stream<T, M><<<grid, 32 * RR_NW, S::smem, ctx->ws>>>(
        p, b, rc, ctx->partials, ctx->nx, ctx->ny, ctx->ncx, ctx->bcmask, nstrip, chunk_h, ntask, skip, ctx->st,
        ctl_mode, cond);
    return grid;
}

// Residual, restriction and norm partials.  Rows of whole 16-byte groups
// (nx % 4 == 0; along a periodic x axis whole 128-column strips): the
// streaming pass (ism_restrict_stream.cuh); otherwise one CTA per coarse
// cell.  *nblk: the number of CTAs, i.e. of norm partials.
template <typename T>
static ism_status launch_resid(ism_ctx *ctx, const T *p, const T *b, T *rc, const int *skip,
                               int ctl_mode = -1, unsigned long long cond = 0, int *nblk = nullptr)
{
    if (ctx->nx % 4 == 0 && (!(ctx->bcmask & ISM_PER_X) || ctx->nx % SRW == 0)) {
        int grid = 0;
        if (ctx->m == 8) grid = launch_restrict_stream<T, 8>(ctx, p, b, rc, skip, ctl_mode, cond);
        else if (ctx->m == 16) grid = launch_restrict_stream<T, 16>(ctx, p, b, rc, skip, ctl_mode, cond);
        else if (ctx->m == 32) grid = launch_restrict_stream<T, 32>(ctx, p, b, rc, skip, ctl_mode, cond);
        if (grid > 0) {
            ISM_LAUNCH_CHECK(ctx);
            if (nblk) *nblk = grid;
            return ISM_OK;
        }
    }
    const int th = std::min(256, ctx->m * ctx->m);
    k_resid<T><<<dim3(ctx->ncx, ctx->ncy), th, 0, ctx->ws>>>(p, b, rc, ctx->partials, ctx->nx,
                                                                ctx->ny, ctx->m, ctx->bcmask, skip,
                                                                ctx->st, ctl_mode, cond);
    ISM_LAUNCH_CHECK(ctx);
    if (nblk) *nblk = ctx->ncx * ctx->ncy;
    return ISM_OK;
}

static ism_status launch_ctl(ism_ctx *ctx, IsmState *st, int nblk, int nq, int mode,
                             unsigned long long cond = 0)
{
    k_ctl<<<1, 256, 0, ctx->ws>>>(st, ctx->partials, nblk, nq, mode, cond);
    ISM_LAUNCH_CHECK(ctx);
    return ISM_OK;
}

template <typename T>
static ism_status launch_sweeps(ism_ctx *ctx, T *p, const T *b, int sweeps, const int *skip)
{
    const int hx = (ctx->nx + 1) / 2;
    const dim3 g = row_grid(hx, ctx->ny, 128);
    for (int s = 0; s < sweeps; ++s)
        for (int col = 0; col < 2; ++col) {
            k_rbgs_colour<T><<<g, 128, 0, ctx->ws>>>(p, b, ctx->nx, ctx->ny, ctx->bcmask, col, skip);
            ISM_LAUNCH_CHECK(ctx);
        }
    return ISM_OK;
}

// Tile grid of a pass and its split into an interior rectangle (regions
// strictly inside the domain) and the list of edge tiles.
using SweepPlan = ism_ctx::SweepPlan;

static SweepPlan &sweep_plan(ism_ctx *ctx, int K, bool resid)
{
    return ctx->plans[ctx->opt.tile_rows == 256 ? 1 : 0][K][resid ? 1 : 0];
}

static ism_status make_plans(ism_ctx *ctx)
{
    for (int shape = 0; shape < 2; ++shape)
    for (int K = 0; K <= SMAXK; ++K)
        for (int r = 0; r < 2; ++r) {
            SweepPlan &P = ctx->plans[shape][K][r];
            const int nw = shape ? 16 : 8, rh = nw * SRR;
            const int tw = sweep_tile_w(K, r), th = sweep_tile_h(K, r, nw);
            const int Hc = sweep_halo_cols(K, r), H = sweep_halo(K, r);
            P.gx = (ctx->nx + tw - 1) / tw;
            P.gy = (ctx->ny + th - 1) / th;
            // interior: region [bx*tw - Hc, +SRW) inside [1, nx-2], same in y
            auto lo = [](int t, int h) { int b = 0; while (b * t - h < 1) ++b; return b; };
            P.ix0 = lo(tw, Hc);
            P.iy0 = lo(th, H);
            P.ix1 = P.ix0; while (P.ix1 < P.gx && P.ix1 * tw - Hc + SRW <= ctx->nx - 1) ++P.ix1;
            P.iy1 = P.iy0; while (P.iy1 < P.gy && P.iy1 * th - H + rh <= ctx->ny - 1) ++P.iy1;
            if (P.ix1 <= P.ix0 || P.iy1 <= P.iy0) { P.ix1 = P.ix0; P.iy1 = P.iy0; }
            std::vector<int2> e;
            for (int by = 0; by < P.gy; ++by)
                for (int bx = 0; bx < P.gx; ++bx)
                    if (!(bx >= P.ix0 && bx < P.ix1 && by >= P.iy0 && by < P.iy1)) e.push_back(make_int2(bx, by));
            P.nedge = (int)e.size();
            if (cudaMalloc((void **)&P.edge, e.size() * sizeof(int2)) != cudaSuccess) {
                cudaGetLastError();
                return ISM_ERR_NOMEM;
            }
            ISM_CUDA_TRY(cudaMemcpy(P.edge, e.data(), e.size() * sizeof(int2), cudaMemcpyHostToDevice));
        }
    return ISM_OK;
}

// Streaming multiprocessors of the current device (read once).
static int ism_sm_count()
{
    static int sms = 0;
    if (!sms) {
        int dev = 0, n = 152;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
            sms = n;
        else
            sms = 152;
        cudaGetLastError();
    }
    return sms;
}

// Interior and edge launches of one pass run concurrently: the edge launch
// goes to a forked stream joined back before the next kernel.
template <int NW, bool PR, bool RE>
static ism_status launch_sweep_pair(ism_ctx *ctx, const SweepArgs &a, const SweepPlan &P)
{
    const size_t sm = sweep_smem_bytes(NW);
    const bool both = P.ix1 > P.ix0 && P.nedge > 0;
    const dim3 gin(P.ix1 - P.ix0, P.iy1 - P.iy0);
    // packed pair updates in the interior launch: option packed 1, or 2
    // (automatic) when the launch runs at least four waves of resident CTAs
    const bool pk = ctx->opt.packed == 1 ||
                    (ctx->opt.packed == 2 && (long long)gin.x * gin.y >= 4LL * (16 / NW) * ism_sm_count());
    auto interior = [&]() {
        if (pk) k_sweep32<NW, PR, RE, false, true><<<gin, 32 * NW, sm, ctx->ws>>>(a);
        else k_sweep32<NW, PR, RE, false, false><<<gin, 32 * NW, sm, ctx->ws>>>(a);
    };
    if (both) {
        ISM_CUDA_TRY(cudaEventRecord(ctx->ev_fork, ctx->ws));
        ISM_CUDA_TRY(cudaStreamWaitEvent(ctx->ws2, ctx->ev_fork, 0));
        k_sweep32<NW, PR, RE, true><<<P.nedge, 32 * NW, sm, ctx->ws2>>>(a);
        interior();
        ISM_CUDA_TRY(cudaEventRecord(ctx->ev_join, ctx->ws2));
        ISM_CUDA_TRY(cudaStreamWaitEvent(ctx->ws, ctx->ev_join, 0));
    } else if (P.ix1 > P.ix0) {
        interior();
    } else {
        k_sweep32<NW, PR, RE, true><<<P.nedge, 32 * NW, sm, ctx->ws>>>(a);
    }
    return ISM_OK;
}

template <bool PR, bool RE>
static ism_status launch_sweep_pair(ism_ctx *ctx, const SweepArgs &a, const SweepPlan &P)
{
    return ctx->opt.tile_rows == 256 ? launch_sweep_pair<16, PR, RE>(ctx, a, P) : launch_sweep_pair<8, PR, RE>(ctx, a, P);
}

// Streaming pass (ism_stream32.cuh): strips of 128 columns, chunks of rows
// sized so that the tasks fill the resident warps of the GPU once (every
// warp then runs the same number of steps).
template <int K>
static ism_status launch_stream(ism_ctx *ctx, const SweepArgs &a)
{
    using S = StreamShape<K>;
    static int slots = 0;                        // resident warps on the device
    if (!slots) {
        int dev = 0, sms = 152, per_sm = 4;
        if (cudaGetDevice(&dev) == cudaSuccess)
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_stream32<K>, 32 * ST_NW, S::smem) != cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
        cudaGetLastError();
        slots = sms * per_sm * ST_NW;
    }
    const int nstrip = (ctx->nx + S::VW - 1) / S::VW;
    const int nchunk = std::max(1, slots / nstrip);
    int chunk_h = std::max(16 * K, (ctx->ny + nchunk - 1) / nchunk);
    chunk_h += chunk_h & 1;                      // even: every chunk starts on an even row
    const int ntask = nstrip * ((ctx->ny + chunk_h - 1) / chunk_h);
    k_stream32<K><<<(ntask + ST_NW - 1) / ST_NW, 32 * ST_NW, S::smem, ctx->ws>>>(a, nstrip, chunk_h, ntask);
    ctx->launches += 1;
    return cudaGetLastError() == cudaSuccess ? ISM_OK : ISM_ERR_CUDA;
}

static ism_status launch_sweep32(ism_ctx *ctx, SweepArgs a, bool prolong, bool resid)
{
    if (ctx->opt.stream && !prolong && !resid) {
        if (a.K == 1) return launch_stream<1>(ctx, a);
        if (a.K == 2) return launch_stream<2>(ctx, a);
        if (a.K == 4) return launch_stream<4>(ctx, a);
    }
    const SweepPlan &P = sweep_plan(ctx, a.K, resid);
    a.H = sweep_halo(a.K, resid);
    a.Hc = sweep_halo_cols(a.K, resid);
    a.TW = sweep_tile_w(a.K, resid);
    a.TH = sweep_tile_h(a.K, resid, ctx->opt.tile_rows == 256 ? 16 : 8);
    a.gx = P.gx; a.gy = P.gy; a.ix0 = P.ix0; a.iy0 = P.iy0; a.edge_tiles = P.edge;
    a.pf_ahead = (ctx->opt.tile_rows == 256 ? 1 : 2) * ism_sm_count();   // one wave of resident CTAs ahead
    a.pgx = P.ix1 - P.ix0;
    a.pn = a.pgx * (P.iy1 - P.iy0);
    if (!resid) a.ctl_mode = -1;
    ism_status st;
    if (prolong && resid) st = launch_sweep_pair<true, true>(ctx, a, P);
    else if (prolong) st = launch_sweep_pair<true, false>(ctx, a, P);
    else if (resid) st = launch_sweep_pair<false, true>(ctx, a, P);
    else st = launch_sweep_pair<false, false>(ctx, a, P);
    if (st != ISM_OK) return st;
    ctx->launches += (P.ix1 > P.ix0) + (P.nedge > 0);
    if (cudaGetLastError() != cudaSuccess) return ISM_ERR_CUDA;
    return ISM_OK;
}

#define TRY(x)                                                                   \
    do {                                                                         \
        ism_status _s = (x);                                                     \
        if (_s != ISM_OK) return _s;                                             \
    } while (0)

// ================================================================ host: cycles

// One FP64 cycle; every kernel returns at once when st->done is set.  cond:
// while-node handle that the residual's control sets (0 outside such a node).
// Residual, its 2 x 2 block sums (level 1 of the V-cycle) and the control.
static ism_status launch_resid2(ism_ctx *ctx, int ctl_mode, unsigned long long cond)
{
    const int ncx = ctx->nx / 2, ncy = ctx->ny / 2;
    k_resid2<double><<<row_grid(ncx, ncy, 128), 128, 0, ctx->ws>>>(
        ctx->p64[0], ctx->b64, ctx->lvl_r[1], ctx->partials, ctx->nx, ctx->ny, ctx->bcmask, &ctx->st->done,
        ctx->st, ctl_mode, cond);
    ISM_LAUNCH_CHECK(ctx);
    return ISM_OK;
}

// One cycle of the deep additive-correction V-cycle (FP64, see ISM_COARSE_ACMV).
static ism_status acmv_cycle(ism_ctx *ctx, unsigned long long cond)
{
    const int *skip = &ctx->st->done;
    int L = 0;
    while ((1 << L) < ctx->m) ++L;
    // down: r_{l+1} = R_2 r_l (r_1 comes from the previous residual), r_L -> rc64
    for (int l = 1; l < L; ++l) {
        const int nxl = ctx->nx >> l, nyl = ctx->ny >> l;
        double *out = (l + 1 < L) ? ctx->lvl_r[l + 1] : ctx->rc64;
        k_restrict2<double><<<row_grid(nxl / 2, nyl / 2, 128), 128, 0, ctx->ws>>>(ctx->lvl_r[l], out, nxl, nyl, skip);
        ISM_LAUNCH_CHECK(ctx);
    }
    // coarsest: A_L = m x five-point, exact
    TRY((launch_coarse<double, false>(ctx, ctx->rc64, ctx->ec64, ctx->T64, skip)));
    // up: e_l = P_2 e_{l+1}, one sweep on (2^l five-point) e_l = r_l
    for (int l = L - 1; l >= 1; --l) {
        const int nxl = ctx->nx >> l, nyl = ctx->ny >> l;
        const double *ec = (l + 1 < L) ? ctx->lvl_e[l + 1] : ctx->ec64;
        k_inject2<double><<<row_grid(nxl, nyl, 128), 128, 0, ctx->ws>>>(ctx->lvl_e[l], ec, nxl, nyl, skip);
        ISM_LAUNCH_CHECK(ctx);
        const dim3 g = row_grid((nxl + 1) / 2, nyl, 128);
        for (int col = 0; col < 2; ++col) {
            k_rbgs_colour<double><<<g, 128, 0, ctx->ws>>>(ctx->lvl_e[l], ctx->lvl_r[l], nxl, nyl, ctx->bcmask, col,
                                                           skip, 1.0 / (double)(1 << l));
            ISM_LAUNCH_CHECK(ctx);
        }
    }
    // p = p - mean + P_2 e_1, nu sweeps, residual (next r_1) with the control
    k_prolong<double><<<row_grid(ctx->nx, ctx->ny, 128), 128, 0, ctx->ws>>>(
        ctx->p64[0], ctx->lvl_e[1], ctx->nx, ctx->ny, 2, ctx->nx / 2, ctx->ny / 2, ctx->bcmask, ISM_COARSE_ACM,
        ctx->st, ctx->singular, skip);
    ISM_LAUNCH_CHECK(ctx);
    TRY(launch_sweeps<double>(ctx, ctx->p64[0], ctx->b64, ctx->opt.nu, skip));
    return launch_resid2(ctx, CTL_FP64_AFTER, cond);
}

static ism_status fp64_cycle(ism_ctx *ctx, unsigned long long cond = 0)
{
    if (ctx->opt.kind == ISM_COARSE_ACMV) return acmv_cycle(ctx, cond);
    const int *skip = &ctx->st->done;
    TRY((launch_coarse<double, false>(ctx, ctx->rc64, ctx->ec64, ctx->T64, skip)));
    if (ctx->opt.kind == ISM_COARSE_ACM) {
        k_prolong<double><<<row_grid(ctx->nx, ctx->ny, 128), 128, 0, ctx->ws>>>(
            ctx->p64[0], ctx->ec64, ctx->nx, ctx->ny, ctx->m, ctx->ncx, ctx->ncy, ctx->bcmask,
            ctx->opt.kind, ctx->st, ctx->singular, skip);
        ISM_LAUNCH_CHECK(ctx);
    } else {
        // bilinear (ISM, GMG): separable form, x first into G, then y per fine row
        k_prolong_x<double><<<dim3((ctx->nx + 127) / 128, ctx->ncy), 128, 0, ctx->ws>>>(
            ctx->ec64, ctx->G64, ctx->nx, ctx->m, ctx->ncx, ctx->ncy, ctx->bcmask, skip);
        ISM_LAUNCH_CHECK(ctx);
        k_prolong_y<double><<<dim3((ctx->nx + 1023) / 1024, ctx->ny), 256, 0, ctx->ws>>>(
            ctx->p64[0], ctx->G64, ctx->nx, ctx->ny, ctx->m, ctx->ncy, ctx->bcmask, ctx->st, ctx->singular, skip);
        ISM_LAUNCH_CHECK(ctx);
    }
    TRY(launch_sweeps<double>(ctx, ctx->p64[0], ctx->b64, ctx->opt.nu, skip));
    return launch_resid<double>(ctx, ctx->p64[0], ctx->b64, ctx->rc64, skip, CTL_FP64_AFTER, cond);
}

static SweepArgs inner_args(ism_ctx *ctx, IsmState *st, float *e0, float *e1, const float *b,
                            const int *skip, const int *curp)
{
    SweepArgs a;
    a.e0 = e0; a.e1 = e1; a.b = b; a.E = ctx->ec32; a.rcpart = ctx->rcpart;
    a.partials = ctx->partials; a.st = st; a.skip = skip; a.curp = curp;
    a.nx = ctx->nx; a.ny = ctx->ny; a.m = ctx->m; a.ncx = ctx->ncx; a.ncy = ctx->ncy;
    a.lm = ctx->m == 8 ? 3 : ctx->m == 16 ? 4 : 5;
    a.bcmask = ctx->bcmask; a.kind = ctx->opt.kind; a.K = ctx->opt.sweeps_per_pass;
    a.q = 0; a.use_mean = ctx->singular; a.ctl_mode = -1; a.pf_ahead = 0;
    a.pgx = a.pn = 0;
    a.H = a.Hc = a.TW = a.TH = 0;
    a.cond = 0;
    return a;
}

// One single-precision inner cycle; kernels return at once when st->inner_done:
// coarse solve (from the partial block sums of the previous pass), then nu/K
// fused passes (the first adds the prolongation, the last computes the
// residual and its restriction), then the control kernel.
static ism_status inner_cycle(ism_ctx *ctx, unsigned long long cond = 0)
{
    const int *skip = &ctx->st->inner_done;
    if (ctx->opt.coarse_tc && ism_coarse_tc_supported(ctx))
        TRY(ism_launch_coarse_tc(ctx, ctx->rcpart, true, ctx->ec32, ctx->rcpart, skip));
    else
        TRY((launch_coarse<float, true>(ctx, ctx->rcpart, ctx->ec32, ctx->T32, skip)));
    const int npass = ctx->opt.nu / ctx->opt.sweeps_per_pass;
    SweepArgs a = inner_args(ctx, ctx->st, ctx->e32[0], ctx->e32[1], ctx->r32, skip, &ctx->st->cur);
    a.ctl_mode = CTL_INNER;
    a.cond = cond;
    for (int q = 0; q < npass; ++q) {
        a.q = q;
        TRY(launch_sweep32(ctx, a, q == 0, q == npass - 1));
    }
    return ISM_OK;
}

// Run chunks of `check_every` cycles (as a CUDA graph when enabled) until the
// flag at `flag_off` in the state becomes nonzero.
static ism_status run_chunks(ism_ctx *ctx, bool inner, int max_chunks)
{
    const int C = ctx->opt.check_every;
    cudaGraphExec_t *gx = inner ? &ctx->g_inner : &ctx->g_fp64;
    int *glen = inner ? &ctx->g_inner_len : &ctx->g_fp64_len;
    for (int it = 0; it < max_chunks; ++it) {
        if (ctx->opt.use_graphs >= 1) {
            if (!*gx) {
                cudaGraph_t g;
                const long long l0 = ctx->launches;
                ISM_CUDA_TRY(cudaStreamBeginCapture(ctx->ws, cudaStreamCaptureModeThreadLocal));
                ism_status s = ISM_OK;
                for (int c = 0; c < C && s == ISM_OK; ++c) s = inner ? inner_cycle(ctx) : fp64_cycle(ctx);
                cudaError_t e = cudaStreamEndCapture(ctx->ws, &g);
                if (s != ISM_OK || e != cudaSuccess) return s != ISM_OK ? s : ISM_ERR_CUDA;
                e = cudaGraphInstantiate(gx, g, 0);
                cudaGraphDestroy(g);
                if (e != cudaSuccess) { *gx = nullptr; return ISM_ERR_CUDA; }
                *glen = (int)(ctx->launches - l0);
                ctx->launches = l0;
            }
            ISM_CUDA_TRY(cudaGraphLaunch(*gx, ctx->ws));
            ctx->launches += *glen;
        } else {
            for (int c = 0; c < C; ++c) TRY(inner ? inner_cycle(ctx) : fp64_cycle(ctx));
        }
        ISM_CUDA_TRY(cudaMemcpyAsync(ctx->st_host, ctx->st, offsetof(IsmState, hist),
                                     cudaMemcpyDeviceToHost, ctx->ws));
        ISM_CUDA_TRY(cudaStreamSynchronize(ctx->ws));
        if (inner ? (ctx->st_host->inner_done || ctx->st_host->done) : ctx->st_host->done) return ISM_OK;
    }
    return ISM_OK;
}

// ================================================================ host: solve

static void init_state(ism_ctx *ctx, IsmState *h, double tol, int max_cycles)
{
    memset(h, 0, offsetof(IsmState, hist));
    h->max_cycles = max_cycles;
    h->max_outer = ctx->opt.max_outer;
    h->inner_max = ctx->opt.inner_max;
    h->npass = ctx->opt.nu / ctx->opt.sweeps_per_pass;
    h->tol = tol;
    h->inner_tol = ctx->opt.inner_tol;
    h->floor_mult = ctx->opt.floor_mult;
    h->inv_n = 1.0 / (double)ctx->n;
}

ism_status ism_prepare_rhs(ism_ctx *ctx, const double *rhs)
{
    const int G = 4 * 152;
    k_rhs_stats<<<G, 256, 0, ctx->ws>>>(rhs, nullptr, ctx->n, ctx->st, 0, 0, ctx->partials);
    ISM_LAUNCH_CHECK(ctx);
    TRY(launch_ctl(ctx, ctx->st, G, 2, CTL_RHS_MEAN));
    k_rhs_stats<<<G, 256, 0, ctx->ws>>>(rhs, ctx->b64, ctx->n, ctx->st, 1, ctx->singular, ctx->partials);
    ISM_LAUNCH_CHECK(ctx);
    return launch_ctl(ctx, ctx->st, G, 1, CTL_RHS_NORM);
}

static ism_status read_state(ism_ctx *ctx)
{
    ISM_CUDA_TRY(cudaMemcpyAsync(ctx->st_host, ctx->st, offsetof(IsmState, hist),
                                 cudaMemcpyDeviceToHost, ctx->ws));
    ISM_CUDA_TRY(cudaStreamSynchronize(ctx->ws));
    return ISM_OK;
}

// ---------------------------------------------------------------- device-side loops
//
// use_graphs = 2: the whole iteration is one CUDA graph.  A while node
// repeats the cycle; its condition is set by the control point fused into the
// last kernel of the cycle (cudaGraphSetConditional), so a solve needs one
// graph launch and one host synchronisation.  The mixed path nests the
// single-precision cycle loop inside the refinement loop.

template <typename F>
static ism_status capture_into(ism_ctx *ctx, cudaGraph_t g, const cudaGraphNode_t *deps, size_t ndeps,
                               F fn, cudaGraphNode_t *last)
{
    ISM_CUDA_TRY(cudaStreamBeginCaptureToGraph(ctx->ws, g, deps, nullptr, ndeps,
                                               cudaStreamCaptureModeThreadLocal));
    ism_status s = fn();
    if (s == ISM_OK && last) {
        cudaStreamCaptureStatus cs;
        const cudaGraphNode_t *d = nullptr;
        size_t nd = 0;
        if (cudaStreamGetCaptureInfo(ctx->ws, &cs, nullptr, nullptr, &d, nullptr, &nd) != cudaSuccess || nd != 1)
            s = ISM_ERR_CUDA;
        else
            *last = d[0];
    }
    cudaGraph_t out = nullptr;
    const cudaError_t e = cudaStreamEndCapture(ctx->ws, &out);
    if (s != ISM_OK) return s;
    return e == cudaSuccess ? ISM_OK : ISM_ERR_CUDA;
}

static inline ism_status ISM_CUDA_OK(cudaError_t e) { return e == cudaSuccess ? ISM_OK : ISM_ERR_CUDA; }

static ism_status add_while_handle(cudaGraph_t g, const cudaGraphNode_t *deps, size_t ndeps,
                                   cudaGraphConditionalHandle h, cudaGraphNode_t *node, cudaGraph_t *body)
{
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    ISM_CUDA_TRY(cudaGraphAddNode(node, g, deps, nullptr, ndeps, &p));
    *body = p.conditional.phGraph_out[0];
    return ISM_OK;
}

static ism_status add_while(cudaGraph_t g, const cudaGraphNode_t *deps, size_t ndeps,
                            cudaGraphConditionalHandle *h, cudaGraphNode_t *node, cudaGraph_t *body)
{
    ISM_CUDA_TRY(cudaGraphConditionalHandleCreate(h, g, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = *h;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    ISM_CUDA_TRY(cudaGraphAddNode(node, g, deps, nullptr, ndeps, &p));
    *body = p.conditional.phGraph_out[0];
    return ISM_OK;
}

// First step of an inner solve: e = 0 and the restriction of its residual r
// (a pass with no sweeps).
static ism_status inner_init(ism_ctx *ctx)
{
    k_zero<<<4 * 152, 256, 0, ctx->ws>>>(ctx->e32[0], ctx->n);
    ISM_LAUNCH_CHECK(ctx);
    k_zero<<<64, 256, 0, ctx->ws>>>(ctx->rcpart, (long long)ctx->ncx * ctx->ncy * 4);
    ISM_LAUNCH_CHECK(ctx);
    SweepArgs a = inner_args(ctx, ctx->st, ctx->e32[0], ctx->e32[1], ctx->r32, nullptr, nullptr);
    a.K = 0;
    return launch_sweep32(ctx, a, false, true);
}

static ism_status refine_update(ism_ctx *ctx, unsigned long long cond)
{
    k_refine_add<<<4 * 152, 256, 0, ctx->ws>>>(ctx->p64[0], ctx->p64[1], ctx->e32[0], ctx->e32[1], ctx->n / 4,
                                               ctx->st);
    ISM_LAUNCH_CHECK(ctx);
    const dim3 rg = refine_grid(ctx->nx, ctx->ny);
    k_refine_resid<<<rg, RF_THREADS, 0, ctx->ws>>>(ctx->p64[0], ctx->p64[1], ctx->b64, ctx->r32, ctx->partials,
                                                   ctx->nx, ctx->ny, ctx->bcmask, ctx->st, 1);
    ISM_LAUNCH_CHECK(ctx);
    return launch_ctl(ctx, ctx->st, rg.x * rg.y, 2, CTL_OUTER_AFTER, cond);
}

static ism_status build_cond_fp64(ism_ctx *ctx)
{
    cudaGraph_t g;
    ISM_CUDA_TRY(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle h;
    cudaGraphNode_t n;
    cudaGraph_t body;
    const long long l0 = ctx->launches;
    ism_status s = add_while(g, nullptr, 0, &h, &n, &body);
    if (s == ISM_OK) s = capture_into(ctx, body, nullptr, 0, [&]() { return fp64_cycle(ctx, h); }, nullptr);
    if (s == ISM_OK && cudaGraphInstantiate(&ctx->gc_fp64, g, 0) != cudaSuccess) s = ISM_ERR_CUDA;
    cudaGraphDestroy(g);
    ctx->g_fp64_len = (int)(ctx->launches - l0);   // launches per cycle
    ctx->launches = l0;
    if (s != ISM_OK) { cudaGetLastError(); ctx->gc_fp64 = nullptr; }
    return s;
}

static ism_status build_cond_mixed(ism_ctx *ctx)
{
    cudaGraph_t g;
    ISM_CUDA_TRY(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle ho, hi;
    cudaGraphNode_t no, ni, last;
    cudaGraph_t bo, bi;
    const long long l0 = ctx->launches;
    ism_status s = add_while(g, nullptr, 0, &ho, &no, &bo);
    // outer body: inner init (which arms the inner loop), then the inner loop,
    // then the FP64 update + control.  The inner handle lives on the outer
    // body, so it exists before the capture that arms it.
    if (s == ISM_OK) s = ISM_CUDA_OK(cudaGraphConditionalHandleCreate(&hi, bo, 1, cudaGraphCondAssignDefault));
    if (s == ISM_OK)
        s = capture_into(ctx, bo, nullptr, 0, [&]() {
            ism_status r = inner_init(ctx);
            if (r != ISM_OK) return r;
            k_arm_condition<<<1, 1, 0, ctx->ws>>>(hi);
            ISM_LAUNCH_CHECK(ctx);
            return ISM_OK;
        }, &last);
    if (s == ISM_OK) s = add_while_handle(bo, &last, 1, hi, &ni, &bi);
    const long long l1 = ctx->launches;
    if (s == ISM_OK) s = capture_into(ctx, bi, nullptr, 0, [&]() { return inner_cycle(ctx, hi); }, nullptr);
    const long long l2 = ctx->launches;
    if (s == ISM_OK) s = capture_into(ctx, bo, &ni, 1, [&]() { return refine_update(ctx, ho); }, nullptr);
    if (s == ISM_OK && cudaGraphInstantiate(&ctx->gc_mixed, g, 0) != cudaSuccess) s = ISM_ERR_CUDA;
    cudaGraphDestroy(g);
    ctx->g_inner_len = (int)(l2 - l1);                          // launches per inner cycle
    ctx->g_fp64_len = (int)((ctx->launches - l0) - (l2 - l1));  // launches per refinement iteration
    ctx->launches = l0;
    if (s != ISM_OK) { cudaGetLastError(); ctx->gc_mixed = nullptr; }
    return s;
}

static ism_status solve_fp64(ism_ctx *ctx)
{
    if (ctx->opt.kind == ISM_COARSE_ACMV) TRY(launch_resid2(ctx, CTL_FP64_INIT, 0));
    else TRY(launch_resid<double>(ctx, ctx->p64[0], ctx->b64, ctx->rc64, nullptr, CTL_FP64_INIT));
    TRY(read_state(ctx));
    if (!ctx->st_host->done) {
        if (ctx->opt.use_graphs == 2) {
            if (!ctx->gc_fp64) TRY(build_cond_fp64(ctx));
            const int c0 = ctx->st_host->cycles;
            ISM_CUDA_TRY(cudaGraphLaunch(ctx->gc_fp64, ctx->ws));
            TRY(read_state(ctx));
            ctx->launches += (long long)(ctx->st_host->cycles - c0 + 1) * ctx->g_fp64_len;
        } else {
            const int C = ctx->opt.check_every;
            TRY(run_chunks(ctx, false, ctx->st_host->max_cycles / C + 2));
        }
    }
    k_finalize<<<4 * 152, 256, 0, ctx->ws>>>(ctx->p64[0], nullptr, ctx->p64[0], ctx->n, ctx->st, ctx->singular);
    ISM_LAUNCH_CHECK(ctx);
    return read_state(ctx);
}

static ism_status solve_mixed(ism_ctx *ctx)
{
    const dim3 rg = refine_grid(ctx->nx, ctx->ny);
    const int nrb = rg.x * rg.y;
    k_refine_resid<<<rg, RF_THREADS, 0, ctx->ws>>>(ctx->p64[0], ctx->p64[1], ctx->b64, ctx->r32, ctx->partials,
                                                   ctx->nx, ctx->ny, ctx->bcmask, ctx->st, 0);
    ISM_LAUNCH_CHECK(ctx);
    TRY(launch_ctl(ctx, ctx->st, nrb, 2, CTL_OUTER_INIT));
    TRY(read_state(ctx));
    if (!ctx->st_host->done && ctx->opt.use_graphs == 2) {
        if (!ctx->gc_mixed) TRY(build_cond_mixed(ctx));
        ISM_CUDA_TRY(cudaGraphLaunch(ctx->gc_mixed, ctx->ws));
        TRY(read_state(ctx));
        ctx->launches += (long long)ctx->st_host->cycles * ctx->g_inner_len +
                         (long long)ctx->st_host->outer * ctx->g_fp64_len;
    } else {
        const int C = ctx->opt.check_every;
        while (!ctx->st_host->done) {
            TRY(inner_init(ctx));
            const int max_chunks = std::min(ctx->opt.inner_max, ctx->st_host->max_cycles) / C + 2;
            TRY(run_chunks(ctx, true, max_chunks));
            TRY(refine_update(ctx, 0));
            TRY(read_state(ctx));
        }
    }
    k_finalize<<<4 * 152, 256, 0, ctx->ws>>>(ctx->p64[0], ctx->p64[1], ctx->p64[0], ctx->n, ctx->st, ctx->singular);
    ISM_LAUNCH_CHECK(ctx);
    return read_state(ctx);
}

ism_status ism_solve_internal(ism_ctx *ctx, double tol, int max_cycles, bool record_rhs)
{
    // keep rhs-preparation results (bnorm, zero_rhs, status) and reset the rest
    TRY(read_state(ctx));
    IsmState h = *ctx->st_host;
    const double bn = h.bnorm;
    if (record_rhs) {
        ctx->last_rhs_sum = h.rhs_sum;
        ctx->last_rhs_l1 = h.rhs_l1;
    }
    const int zr = h.zero_rhs, stt = h.status, dn = h.done;
    init_state(ctx, &h, tol, max_cycles);
    h.bnorm = bn;
    h.zero_rhs = zr;
    h.status = stt;
    h.done = dn;
    ISM_CUDA_TRY(cudaMemcpyAsync(ctx->st, &h, offsetof(IsmState, hist), cudaMemcpyHostToDevice, ctx->ws));
    if (dn) {                      // right-hand side already rejected (non-finite)
        ctx->last_cycles = ctx->last_outer = 0;
        ctx->last_relres = NAN;
        ctx->last_status = stt;
        ctx->last_nhist = 0;
        return (ism_status)stt;
    }
    if (ctx->opt.cycle == 1) return ism_solve_accommodative(ctx, tol, max_cycles);
    ism_status s = ctx->prec == ISM_FP64 ? solve_fp64(ctx) : solve_mixed(ctx);
    if (s != ISM_OK) return s;
    const IsmState *hs = ctx->st_host;
    if (hs->tc_fail) {            // a tensor-core coarse solve gave up waiting: the result is void
        ctx->last_status = ISM_ERR_CUDA;
        return ISM_ERR_CUDA;
    }
    ctx->last_cycles = hs->cycles;
    ctx->last_outer = hs->outer;
    ctx->last_relres = hs->relres;
    ctx->last_status = hs->status;
    ctx->last_nhist = std::min(ISM_HMAX, (ctx->prec == ISM_FP64 ? hs->cycles : hs->outer) + 1);
    return (ism_status)hs->status;
}

extern "C" ism_status ism_solve(ism_ctx *ctx, const double *rhs, double *p, double tol,
                                int max_cycles, int *cycles_out, double *relres_out)
{
    if (!ctx || !rhs || !p || !(tol > 0.0) || max_cycles < 0) return ISM_ERR_ARG;
    TRY(ism_enter(ctx));
    // reset the state, then prepare the rhs
    IsmState h;
    memset(&h, 0, offsetof(IsmState, hist));
    h.inv_n = 1.0 / (double)ctx->n;
    ISM_CUDA_TRY(cudaMemcpyAsync(ctx->st, &h, offsetof(IsmState, hist), cudaMemcpyHostToDevice, ctx->ws));
    TRY(ism_prepare_rhs(ctx, rhs));
    ISM_CUDA_TRY(cudaMemcpyAsync(ctx->p64[0], p, (size_t)ctx->n * 8, cudaMemcpyDeviceToDevice, ctx->ws));
    ism_status s = ism_solve_internal(ctx, tol, max_cycles);
    if (s == ISM_OK || s == ISM_ERR_NOT_CONVERGED || s == ISM_ERR_NONFINITE) {
        ISM_CUDA_TRY(cudaMemcpyAsync(p, ctx->p64[0], (size_t)ctx->n * 8, cudaMemcpyDeviceToDevice, ctx->ws));
    }
    ism_status s2 = ism_leave(ctx);
    ISM_CUDA_TRY(cudaStreamSynchronize(ctx->ws));
    if (cycles_out) *cycles_out = ctx->last_cycles;
    if (relres_out) *relres_out = ctx->last_relres;
    return s != ISM_OK ? s : s2;
}

extern "C" int ism_last_history(const ism_ctx *ctx, double *hist, int cap)
{
    if (!ctx || !hist || cap <= 0) return 0;
    const int n = std::min(cap, ctx->last_nhist);
    if (cudaMemcpy(hist, ctx->st->hist, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
        return 0;
    return n;
}

extern "C" ism_status ism_last_rhs(const ism_ctx *ctx, double *mean_removed, int *incompatible)
{
    if (!ctx) return ISM_ERR_ARG;
    const double sum = ctx->singular ? ctx->last_rhs_sum : 0.0;
    if (mean_removed) *mean_removed = sum / (double)ctx->n;
    if (incompatible) *incompatible = ctx->singular && fabs(sum) > 1e-12 * ctx->last_rhs_l1;
    return ISM_OK;
}

extern "C" ism_status ism_last_counts(const ism_ctx *ctx, int *outer, int *cycles, long long *launches)
{
    if (!ctx) return ISM_ERR_ARG;
    if (outer) *outer = ctx->last_outer;
    if (cycles) *cycles = ctx->last_cycles;
    if (launches) *launches = ctx->launches;
    return ISM_OK;
}

// ================================================================ kernel-level entry points

extern "C" ism_status ism_smooth(ism_ctx *ctx, void *p, const void *b, int sweeps)
{
    if (!ctx || !p || !b || sweeps < 0) return ISM_ERR_ARG;
    if (sweeps == 0) return ISM_OK;
    TRY(ism_enter(ctx));
    if (ctx->prec == ISM_FP64) {
        TRY(launch_sweeps<double>(ctx, (double *)p, (const double *)b, sweeps, nullptr));
    } else {
        // fused passes of up to K sweeps, ping-pong between p and e32[1]
        float *buf[2] = {(float *)p, ctx->e32[1]};
        SweepArgs a = inner_args(ctx, ctx->st_k, buf[0], buf[1], (const float *)b, nullptr, nullptr);
        a.use_mean = 0;
        int cur = 0, left = sweeps;
        while (left > 0) {
            a.K = std::min(left, SMAXK);
            a.q = cur;
            TRY(launch_sweep32(ctx, a, false, false));
            cur ^= 1;
            left -= a.K;
        }
        if (cur) ISM_CUDA_TRY(cudaMemcpyAsync(p, buf[1], (size_t)ctx->n * 4, cudaMemcpyDeviceToDevice, ctx->ws));
    }
    return ism_leave(ctx);
}

extern "C" ism_status ism_residual_restrict(ism_ctx *ctx, const void *p, const void *b, void *rc,
                                            double *norms)
{
    if (!ctx || !p || !b || !rc) return ISM_ERR_ARG;
    TRY(ism_enter(ctx));
    int nb = 0;
    if (ctx->prec == ISM_FP64)
        TRY(launch_resid<double>(ctx, (const double *)p, (const double *)b, (double *)rc, nullptr, -1, 0, &nb));
    else
        TRY(launch_resid<float>(ctx, (const float *)p, (const float *)b, (float *)rc, nullptr, -1, 0, &nb));
    if (norms) {
        std::vector<double> part((size_t)3 * nb);
        ISM_CUDA_TRY(cudaMemcpyAsync(part.data(), ctx->partials, part.size() * 8, cudaMemcpyDeviceToHost, ctx->ws));
        ISM_CUDA_TRY(cudaStreamSynchronize(ctx->ws));
        double r2 = 0, ps = 0;
        for (int k = 0; k < nb; ++k) { r2 += part[k]; ps += part[nb + k]; }
        norms[0] = sqrt(r2);
        norms[1] = ps;
    }
    return ism_leave(ctx);
}

extern "C" ism_status ism_residual_norms(ism_ctx *ctx, const double *rhs, const double *p, double *l2,
                                         double *maxabs)
{
    if (!ctx || !rhs || !p || (!l2 && !maxabs)) return ISM_ERR_ARG;
    TRY(ism_enter(ctx));
    const dim3 g = row_grid(ctx->nx, ctx->ny, 256);
    k_resnorms<<<g, 256, 0, ctx->ws>>>(p, rhs, ctx->partials, ctx->nx, ctx->ny, ctx->bcmask);
    ISM_LAUNCH_CHECK(ctx);
    const int nb = (int)(g.x * g.y);
    std::vector<double> part((size_t)2 * nb);
    ISM_CUDA_TRY(cudaMemcpyAsync(part.data(), ctx->partials, part.size() * 8, cudaMemcpyDeviceToHost, ctx->ws));
    ISM_CUDA_TRY(cudaStreamSynchronize(ctx->ws));
    double r2 = 0.0, rm = 0.0;
    for (int k = 0; k < nb; ++k) {
        r2 += part[k];
        rm = std::max(rm, part[(size_t)nb + k]);
    }
    if (l2) *l2 = sqrt(r2);
    if (maxabs) *maxabs = rm;
    return ism_leave(ctx);
}

extern "C" ism_status ism_coarse_solve(ism_ctx *ctx, const void *rc, void *ec)
{
    if (!ctx || !rc || !ec) return ISM_ERR_ARG;
    TRY(ism_enter(ctx));
    if (ctx->prec == ISM_FP64) TRY((launch_coarse<double, false>(ctx, (const double *)rc, (double *)ec, ctx->T64, nullptr)));
    else if (ctx->opt.coarse_tc && ism_coarse_tc_supported(ctx))
        TRY(ism_launch_coarse_tc(ctx, (const float *)rc, false, (float *)ec, nullptr, nullptr));
    else TRY((launch_coarse<float, false>(ctx, (const float *)rc, (float *)ec, ctx->T32, nullptr)));
    return ism_leave(ctx);
}

extern "C" ism_status ism_prolong_add(ism_ctx *ctx, const void *ec, void *p)
{
    if (!ctx || !ec || !p) return ISM_ERR_ARG;
    TRY(ism_enter(ctx));
    const dim3 g = row_grid(ctx->nx, ctx->ny, 128);
    if (ctx->prec == ISM_FP64)
        k_prolong<double><<<g, 128, 0, ctx->ws>>>((double *)p, (const double *)ec, ctx->nx, ctx->ny, ctx->m,
                                                  ctx->ncx, ctx->ncy, ctx->bcmask, ctx->opt.kind, nullptr, 0, nullptr);
    else
        k_prolong<float><<<g, 128, 0, ctx->ws>>>((float *)p, (const float *)ec, ctx->nx, ctx->ny, ctx->m,
                                                 ctx->ncx, ctx->ncy, ctx->bcmask, ctx->opt.kind, nullptr, 0, nullptr);
    ISM_LAUNCH_CHECK(ctx);
    return ism_leave(ctx);
}

// Device time of `reps` launches of pass(r), r = 0 .. reps-1, as the solver
// runs them: the launches are captured into one CUDA graph on the work
// stream (no host launch gaps between kernels, as inside the solve graphs),
// the graph is replayed once to warm up and once between two CUDA events on
// the work stream.
template <typename F>
static ism_status time_graph(ism_ctx *ctx, int reps, F pass, double *us_per_pass)
{
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t gx = nullptr;
    ism_status st = ISM_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = ISM_ERR_CUDA;
    if (st == ISM_OK && cudaStreamBeginCapture(ctx->ws, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        st = ISM_ERR_CUDA;
    if (st == ISM_OK) {
        for (int r = 0; r < reps && st == ISM_OK; ++r) st = pass(r);
        // always end the capture, also after a failed launch
        if (cudaStreamEndCapture(ctx->ws, &g) != cudaSuccess && st == ISM_OK) st = ISM_ERR_CUDA;
    }
    if (st == ISM_OK && cudaGraphInstantiate(&gx, g, 0) != cudaSuccess) st = ISM_ERR_CUDA;
    if (st == ISM_OK && cudaGraphLaunch(gx, ctx->ws) != cudaSuccess) st = ISM_ERR_CUDA;      // warm-up
    if (st == ISM_OK && (cudaEventRecord(e0, ctx->ws) != cudaSuccess || cudaGraphLaunch(gx, ctx->ws) != cudaSuccess ||
                         cudaEventRecord(e1, ctx->ws) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess))
        st = ISM_ERR_CUDA;
    if (st == ISM_OK) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) st = ISM_ERR_CUDA;
        else *us_per_pass = 1000.0 * ms / reps;
    }
    if (gx) cudaGraphExecDestroy(gx);
    if (g) cudaGraphDestroy(g);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st != ISM_OK) cudaGetLastError();
    return st;
}

extern "C" ism_status ism_time_restrict(ism_ctx *ctx, const void *p, const void *b, void *rc, int reps,
                                        double *us_per_pass)
{
    if (!ctx || !p || !b || !rc || reps < 1 || !us_per_pass) return ISM_ERR_ARG;
    auto pass = [&](int) -> ism_status {
        if (ctx->prec == ISM_FP64) return launch_resid<double>(ctx, (const double *)p, (const double *)b, (double *)rc, nullptr);
        return launch_resid<float>(ctx, (const float *)p, (const float *)b, (float *)rc, nullptr);
    };
    TRY(ism_enter(ctx));
    ism_status st = time_graph(ctx, reps, pass, us_per_pass);
    ism_status s2 = ism_leave(ctx);
    ISM_CUDA_TRY(cudaStreamSynchronize(ctx->ws));
    return st != ISM_OK ? st : s2;
}

extern "C" ism_status ism_time_pass(ism_ctx *ctx, void *p, const void *b, int sweeps, int reps,
                                    double *us_per_pass)
{
    if (!ctx || !p || !b || sweeps < 1 || reps < 1 || !us_per_pass) return ISM_ERR_ARG;
    if (ctx->prec == ISM_MIXED && sweeps > SMAXK) return ISM_ERR_ARG;
    // an even number of single-precision passes: the ping-pong ends in p
    if (ctx->prec == ISM_MIXED) reps += reps & 1;
    auto pass = [&](int r) -> ism_status {
        if (ctx->prec == ISM_FP64) return launch_sweeps<double>(ctx, (double *)p, (const double *)b, sweeps, nullptr);
        SweepArgs a = inner_args(ctx, ctx->st_k, (float *)p, ctx->e32[1], (const float *)b, nullptr, nullptr);
        a.use_mean = 0;
        a.K = sweeps;
        a.q = r & 1;
        return launch_sweep32(ctx, a, false, false);
    };
    TRY(ism_enter(ctx));
    ism_status st = time_graph(ctx, reps, pass, us_per_pass);
    ism_status s2 = ism_leave(ctx);
    ISM_CUDA_TRY(cudaStreamSynchronize(ctx->ws));
    return st != ISM_OK ? st : s2;
}

extern "C" ism_status ism_time_coarse(ism_ctx *ctx, const void *rc, void *ec, int reps, double *us_per_solve)
{
    if (!ctx || !rc || !ec || reps < 1 || !us_per_solve) return ISM_ERR_ARG;
    auto solve = [&](int) -> ism_status {
        if (ctx->prec == ISM_FP64)
            return launch_coarse<double, false>(ctx, (const double *)rc, (double *)ec, ctx->T64, nullptr);
        if (ctx->opt.coarse_tc && ism_coarse_tc_supported(ctx))
            return ism_launch_coarse_tc(ctx, (const float *)rc, false, (float *)ec, nullptr, nullptr);
        return launch_coarse<float, false>(ctx, (const float *)rc, (float *)ec, ctx->T32, nullptr);
    };
    TRY(ism_enter(ctx));
    ism_status st = time_graph(ctx, reps, solve, us_per_solve);
    ism_status s2 = ism_leave(ctx);
    ISM_CUDA_TRY(cudaStreamSynchronize(ctx->ws));
    return st != ISM_OK ? st : s2;
}

// ================================================================ autotuner

extern "C" ism_status ism_autotune(ism_ctx *ctx, const double *rhs, double tol, int max_cycles,
                                   ism_options *best)
{
    return ism_autotune_from(ctx, rhs, nullptr, tol, max_cycles, best);
}

extern "C" ism_status ism_autotune_from(ism_ctx *ctx, const double *rhs, const double *p0, double tol,
                                        int max_cycles, ism_options *best)
{
    if (!ctx || !rhs || !(tol > 0.0) || max_cycles < 1) return ISM_ERR_ARG;
    // a cycle costs a fixed part (coarse solve, fused prolongation and residual,
    // control) plus one part per pass, and the total sweeps of a solve are
    // nearly independent of nu: larger nu amortises the fixed part.  Mixed
    // candidates {nu, sweeps per pass, stream}: the streaming middle passes
    // (stream = 1, 4 sweeps per pass) win on grids larger than L2.
    // (K = 6, whose 104 x 104 valid tile wastes fewer cells than the 96 x 96
    // of K = 8, measured slower per sweep on 8192 x 4096 and 2048^2 grids and
    // is not offered.)
    static const int cand_mixed[][3] = {{8, 4, 0},   {8, 8, 0},   {16, 8, 0},  {24, 8, 0}, {32, 8, 0},
                                        {48, 8, 0},  {64, 8, 0},  {96, 8, 0},  {128, 8, 0}, {192, 8, 0},
                                        {256, 8, 0}, {16, 4, 0},  {32, 4, 1},  {64, 4, 1}, {128, 4, 1}};
    static const int cand_fp64[][3] = {{8, 4, 0}, {16, 4, 0}, {32, 4, 0}, {48, 4, 0}, {64, 4, 0}, {96, 4, 0},
                                       {128, 4, 0}};
    // then, for the five fastest mixed candidates, the inner stopping factor
    // of the refinement (it interacts with nu: a longer cycle reaches a
    // tighter inner tolerance in fewer cycles, and candidates that tie at the
    // default factor can differ by 20% at another); for the winner the other
    // height of the fused pass's tiled region (tile shape), and last the other
    // coarse engines (CUDA cores, the single-CTA tensor-core kernel, the tiled
    // split-TF32 chain: TF32 error costs cycles on some grids, and the chain's
    // four launches cost time on small ones)
    static const double inner_tols[] = {1e-4, 1e-2};
    const int (*cand)[3] = ctx->prec == ISM_MIXED ? cand_mixed : cand_fp64;
    const int ncand = ctx->prec == ISM_MIXED ? (int)(sizeof(cand_mixed) / sizeof(cand_mixed[0]))
                                             : (int)(sizeof(cand_fp64) / sizeof(cand_fp64[0]));
    // the engine coarse_tc = k selects (0 CUDA cores, 1 single CTA, 2 chain)
    auto engine = [&](int k) {
        if (k == 0 || !ism_coarse_tc_supported(ctx)) return 0;
        return (k == 1 && ism_coarse_tc_small(ctx)) ? 1 : 2;
    };
    const ism_options saved = ctx->opt;
    double *p = nullptr;
    if (cudaMalloc((void **)&p, (size_t)ctx->n * 8) != cudaSuccess) { cudaGetLastError(); return ISM_ERR_NOMEM; }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    ism_status st = ISM_OK;
    // time of a complete solve under `o` (the first run builds the graph and
    // is not counted), 1e30 if it does not converge
    auto time_opt = [&](const ism_options &o) -> float {
        if ((st = ism_set_options(ctx, &o)) != ISM_OK) return 1e30f;
        float ms = 1e30f;
        for (int rep = 0; rep < 2; ++rep) {
            if (p0) cudaMemcpyAsync(p, p0, (size_t)ctx->n * 8, cudaMemcpyDeviceToDevice, ctx->user_stream);
            else cudaMemsetAsync(p, 0, (size_t)ctx->n * 8, ctx->user_stream);
            cudaEventRecord(e0, ctx->user_stream);
            int cyc = 0;
            double rel = 0.0;
            const ism_status s = ism_solve(ctx, rhs, p, tol, max_cycles, &cyc, &rel);
            cudaEventRecord(e1, ctx->user_stream);
            cudaEventSynchronize(e1);
            if (s != ISM_OK) return 1e30f;
            cudaEventElapsedTime(&ms, e0, e1);
        }
        return ms;
    };
    std::vector<std::pair<float, ism_options>> first;
    for (int c = 0; c < ncand && st == ISM_OK; ++c) {
        ism_options o = saved;
        o.nu = cand[c][0];
        o.sweeps_per_pass = cand[c][1];
        o.stream = cand[c][2];
        first.push_back({time_opt(o), o});
    }
    std::stable_sort(first.begin(), first.end(),
                     [](const std::pair<float, ism_options> &x, const std::pair<float, ism_options> &y) {
                         return x.first < y.first;
                     });
    float best_ms = first.empty() ? 1e30f : first[0].first;
    ism_options win = first.empty() ? saved : first[0].second;
    if (ctx->prec == ISM_MIXED && st == ISM_OK) {
        auto consider = [&](const ism_options &o) {
            const float ms = time_opt(o);
            if (ms < best_ms) { best_ms = ms; win = o; }
        };
        const int top = std::min<int>(5, (int)first.size());
        for (int k = 0; k < top && st == ISM_OK; ++k)
            for (double it : inner_tols) {
                if (first[k].first >= 1e29f || st != ISM_OK) continue;
                ism_options o = first[k].second;
                o.inner_tol = it;
                consider(o);
            }
        if (st == ISM_OK) {
            ism_options o = win;
            o.tile_rows = win.tile_rows == 256 ? 128 : 256;
            consider(o);
        }
        // scalar or packed pair updates in the interior tiles, explicitly
        const ism_options w1 = win;
        for (int pk = 0; pk <= 1 && st == ISM_OK; ++pk) {
            ism_options o = w1;
            o.packed = pk;
            consider(o);
        }
        const ism_options w0 = win;
        for (int d = 1; d <= 2 && st == ISM_OK; ++d) {
            ism_options o = w0;
            o.coarse_tc = (w0.coarse_tc + d) % 3;
            if (engine(o.coarse_tc) == engine(w0.coarse_tc)) continue;                 // the same engine
            if (d == 2 && engine(o.coarse_tc) == engine((w0.coarse_tc + 1) % 3)) continue;
            consider(o);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(p);
    if (st != ISM_OK) { ism_set_options(ctx, &saved); return st; }
    if (best_ms >= 1e29f) { ism_set_options(ctx, &saved); return ISM_ERR_NOT_CONVERGED; }
    st = ism_set_options(ctx, &win);
    if (best) *best = win;
    return st;
}
