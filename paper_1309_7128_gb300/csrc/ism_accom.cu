// ism_accom.cu -- the paper's accommodative strategy for one pressure solve
// (Sec. 4.3.1), FP64: iterate on the coarse grid first, prolongate when the
// coarse residual is small enough, then iterate on the fine grid until the
// fine criterion holds (one coarse-then-fine pass).
//
//   r = b - A_f p; r_c = R r (m x m block sums)
//   e_c = 0; four-colour Gauss-Seidel on the nine-point ISM equations
//        A_c e_c = r_c until max |r_c - A_c e_c| <= tol_c
//   p += P e_c (bilinear, Eq. 5), mean removed when every face is Neumann
//   red-black sweeps on A_f p = b until max |b - A_f p| <= tol
//
// The coarse iteration runs in one CTA (the coarse grid is small); its sums
// are rounded at every step (no contraction) in the neighbour order of the
// oracle.  A_c comes from its closed form (Sec. 3.3, Eq. 5-7):
// A_c = 1/4 (S_y x S_x) - 4 I with S = tridiag(1, 2, 1), end diagonal 3 at
// a Neumann end and 1 at a Dirichlet-0 end, circulant on a periodic axis
// (whose neighbours then wrap; such an axis has an even number >= 4 of
// coarse cells, so the nine neighbours are distinct and the four colours
// independent).  When the grid is not a multiple of m (a narrower last
// coarse cell, walls only) A_c = W_y x T_x + T_y x W_x with the tridiagonal
// 1-D operators W = R1 P1 and T = R1 T1 P1 of each axis (ism_pencil.cu),
// passed in as `tri`.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "ism_kernels.cuh"

// defined in ism_core.cu
__global__ void k_ctl(IsmState *st, const double *partials, int nblk, int nq, int mode,
                      unsigned long long cond);
__global__ void k_rhs_stats(const double *__restrict__ x, double *__restrict__ y, long long n,
                            const IsmState *st, int mode, int sub_mean, double *partials);
__global__ void k_finalize(const double *in, const double *in_alt, double *out, long long n,
                           const IsmState *st, int sub_mean);

namespace {

constexpr int AC_THREADS = 1024;

// S[I][I + d] for |d| <= 1 (d != 0: a neighbour that exists)
__device__ __forceinline__ double s_entry(int I, int d, int n, int lo_dir, int hi_dir, bool periodic)
{
    if (d != 0) return 1.0;
    if (periodic) return 2.0;
    if (n == 1) return (lo_dir ? 1.0 : 3.0) + (hi_dir ? 1.0 : 3.0) - 2.0;
    if (I == 0) return lo_dir ? 1.0 : 3.0;
    if (I == n - 1) return hi_dir ? 1.0 : 3.0;
    return 2.0;
}

// coefficient of e[J + dJ][I + dI] (wrapped on a periodic axis) in row (I, J) of A_c
__device__ __forceinline__ double ac_coef(int I, int J, int dI, int dJ, int ncx, int ncy, int bcmask,
                                          const double *tri)
{
    if (tri) {   // W_x, T_x (3 ncx each), W_y, T_y (3 ncy each): row k as (k-1, k, k+1)
        const double *Wx = tri, *Tx = tri + 3 * ncx, *Wy = tri + 6 * ncx, *Ty = Wy + 3 * ncy;
        return __dadd_rn(__dmul_rn(Wy[3 * J + 1 + dJ], Tx[3 * I + 1 + dI]),
                         __dmul_rn(Ty[3 * J + 1 + dJ], Wx[3 * I + 1 + dI]));
    }
    const double sx = s_entry(I, dI, ncx, bcmask & 1, bcmask & 2, (bcmask & ISM_PER_X) != 0);
    const double sy = s_entry(J, dJ, ncy, bcmask & 4, bcmask & 8, (bcmask & ISM_PER_Y) != 0);
    double a = __dmul_rn(0.25, __dmul_rn(sx, sy));
    if (dI == 0 && dJ == 0) a = __dadd_rn(a, -4.0);
    return a;
}

// row sum over the nine neighbours (dJ = -1..1, dI = -1..1), optionally
// without the centre
__device__ __forceinline__ double row_sum(const double *e, int I, int J, int ncx, int ncy, int bcmask,
                                          bool centre, const double *tri)
{
    double s = 0.0;
    for (int dJ = -1; dJ <= 1; ++dJ)
        for (int dI = -1; dI <= 1; ++dI) {
            int K = J + dJ, L = I + dI;
            if (bcmask & ISM_PER_Y) K = K < 0 ? K + ncy : (K >= ncy ? K - ncy : K);
            if (bcmask & ISM_PER_X) L = L < 0 ? L + ncx : (L >= ncx ? L - ncx : L);
            if ((!centre && dI == 0 && dJ == 0) || K < 0 || K >= ncy || L < 0 || L >= ncx) continue;
            s = __dadd_rn(s, __dmul_rn(ac_coef(I, J, dI, dJ, ncx, ncy, bcmask, tri), e[(size_t)K * ncx + L]));
        }
    return s;
}

// One CTA: e = 0, then Gauss-Seidel iterations until the criterion or the
// cap; the iteration count goes to st->outer.  SMEM: the iterate and the
// right-hand side live in dynamic shared memory during the iteration (coarse
// grids up to AC_SMEM_MAX cells), e is written back at the end.
constexpr int AC_SMEM_MAX = 12800;             // 2 x 8 B x 12800 = 200 KB

template <bool SMEM>
__global__ void __launch_bounds__(AC_THREADS, 1)
k_coarse_gs4(const double *__restrict__ r_g, double *__restrict__ e_g, int ncx, int ncy, int bcmask, double tol,
             int cap, IsmState *st, const double *__restrict__ tri)
{
    if (st->done) return;
    extern __shared__ double ac_sm[];
    __shared__ double red[32];
    __shared__ int stop;
    const int t = threadIdx.x, nc = ncx * ncy;
    double *e = SMEM ? ac_sm : e_g;
    const double *r = r_g;
    if (SMEM) {
        double *rs = ac_sm + nc;
        for (int k = t; k < nc; k += AC_THREADS) rs[k] = r_g[k];
        r = rs;
    }
    for (int k = t; k < nc; k += AC_THREADS) e[k] = 0.0;
    __syncthreads();
    int it = 0;
    for (;;) {
        double mx = 0.0;
        for (int k = t; k < nc; k += AC_THREADS) {
            const int I = k % ncx, J = k / ncx;
            const double d = fabs(__dadd_rn(r[k], -row_sum(e, I, J, ncx, ncy, bcmask, true, tri)));
            mx = fmax(mx, d);
        }
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(FULLMASK, mx, o));
        if ((t & 31) == 0) red[t >> 5] = mx;
        __syncthreads();
        if (t == 0) {
            double m2 = 0.0;
            for (int w = 0; w < AC_THREADS / 32; ++w) m2 = fmax(m2, red[w]);
            stop = (m2 <= tol || it >= cap);
        }
        __syncthreads();
        if (stop) break;
        for (int colour = 0; colour < 4; ++colour) {
            const int I0 = colour & 1, J0 = colour >> 1;
            const int hx = (ncx - I0 + 1) / 2, hy = (ncy - J0 + 1) / 2;
            for (int k = t; k < hx * hy; k += AC_THREADS) {
                const int I = I0 + 2 * (k % hx), J = J0 + 2 * (k / hx);
                const double s = row_sum(e, I, J, ncx, ncy, bcmask, false, tri);
                e[(size_t)J * ncx + I] =
                    __ddiv_rn(__dadd_rn(r[(size_t)J * ncx + I], -s), ac_coef(I, J, 0, 0, ncx, ncy, bcmask, tri));
            }
            __syncthreads();
        }
        ++it;
    }
    if (SMEM)
        for (int k = t; k < nc; k += AC_THREADS) e_g[k] = e[k];
    if (t == 0) st->outer = it;
}

// max |b - A_f p| per block, then (last block) the fine criterion: counts a
// sweep unless `initial`, sets done / status.
__global__ void k_resmax(const double *__restrict__ p, const double *__restrict__ b, double *partials, int nx,
                         int ny, int bcmask, IsmState *st, double tol, int cap, int initial)
{
    if (st->done) return;
    __shared__ double red[32];
    __shared__ int am_last;
    double mx = 0.0;
    const long long n = (long long)nx * ny;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(k % nx), j = (int)(k / nx);
        const double s = nb_sum<double>([&](long long q) -> double { return p[q]; }, k, i, j, nx, ny, bcmask);
        const double r = b[k] - (s - (double)diag_count(i, j, nx, ny, bcmask) * p[k]);
        mx = fmax(mx, fabs(r));
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(FULLMASK, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m2 = 0.0;
        for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) m2 = fmax(m2, red[w]);
        partials[blockIdx.x] = m2;
        __threadfence();
        am_last = (atomicAdd(&st->ticket, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!am_last || threadIdx.x != 0) return;
    __threadfence();
    double m2 = 0.0;
    for (int k = 0; k < (int)gridDim.x; ++k) m2 = fmax(m2, __ldcg(partials + k));
    st->ticket = 0;
    if (!initial) st->cycles++;
    st->relres = m2;
    if (!isfinite(m2)) { st->status = ISM_ERR_NONFINITE; st->done = 1; }
    else if (m2 <= tol) { st->status = ISM_OK; st->done = 1; }
    else if (!initial && st->cycles >= cap) { st->status = ISM_ERR_NOT_CONVERGED; st->done = 1; }
}

}  // namespace

#define TRY(x)                                                                   \
    do {                                                                         \
        ism_status _s = (x);                                                     \
        if (_s != ISM_OK) return _s;                                             \
    } while (0)

// p -= mean(p) (all faces Neumann): sums, mean into st->mean, subtraction
static ism_status remove_mean(ism_ctx *ctx, double *p)
{
    const int G = 4 * 152;
    k_rhs_stats<<<G, 256, 0, ctx->ws>>>(p, nullptr, ctx->n, ctx->st, 0, 0, ctx->partials);
    ISM_LAUNCH_CHECK(ctx);
    k_ctl<<<1, 256, 0, ctx->ws>>>(ctx->st, ctx->partials, G, 1, 0 /* mean */, 0);
    ISM_LAUNCH_CHECK(ctx);
    k_finalize<<<G, 256, 0, ctx->ws>>>(p, nullptr, p, ctx->n, ctx->st, 1);
    ISM_LAUNCH_CHECK(ctx);
    return ISM_OK;
}

// Solve with cycle = 1 on the internal buffers (b64 prepared, p64[0] the
// initial guess); ism_solve_internal's contract.
ism_status ism_solve_accommodative(ism_ctx *ctx, double tol, int max_sweeps)
{
    const int G = 2 * 152, T = 256;
    IsmState h;
    ISM_CUDA_TRY(cudaMemcpyAsync(&h, ctx->st, offsetof(IsmState, hist), cudaMemcpyDeviceToHost, ctx->ws));
    ISM_CUDA_TRY(cudaStreamSynchronize(ctx->ws));
    if (!h.done) {
        // initial guess: mean removed (all Neumann), its criterion
        if (ctx->singular) TRY(remove_mean(ctx, ctx->p64[0]));
        k_resmax<<<G, T, 0, ctx->ws>>>(ctx->p64[0], ctx->b64, ctx->partials, ctx->nx, ctx->ny, ctx->bcmask, ctx->st,
                                       tol, max_sweeps, 1);
        ISM_LAUNCH_CHECK(ctx);
        // restriction, coarse iteration, bilinear correction
        const int th = std::min(256, ctx->m * ctx->m);
        k_resid<double><<<dim3(ctx->ncx, ctx->ncy), th, 0, ctx->ws>>>(ctx->p64[0], ctx->b64, ctx->rc64, ctx->partials,
                                                                     ctx->nx, ctx->ny, ctx->m, ctx->bcmask,
                                                                     &ctx->st->done);
        ISM_LAUNCH_CHECK(ctx);
        const int nc = ctx->ncx * ctx->ncy;
        const double *tri = ctx->ragged ? ctx->ac_tri : nullptr;
        if (nc <= AC_SMEM_MAX) {
            const size_t smb = 2 * sizeof(double) * (size_t)nc;
            static bool attr = false;
            if (!attr) {
                cudaFuncSetAttribute(k_coarse_gs4<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(2 * sizeof(double) * AC_SMEM_MAX));
                attr = true;
            }
            k_coarse_gs4<true><<<1, AC_THREADS, smb, ctx->ws>>>(ctx->rc64, ctx->ec64, ctx->ncx, ctx->ncy, ctx->bcmask,
                                                                ctx->opt.accom_tol_c, ctx->opt.accom_max_coarse,
                                                                ctx->st, tri);
        } else {
            k_coarse_gs4<false><<<1, AC_THREADS, 0, ctx->ws>>>(ctx->rc64, ctx->ec64, ctx->ncx, ctx->ncy, ctx->bcmask,
                                                               ctx->opt.accom_tol_c, ctx->opt.accom_max_coarse,
                                                               ctx->st, tri);
        }
        ISM_LAUNCH_CHECK(ctx);
        k_prolong<double><<<dim3((ctx->nx + 127) / 128, ctx->ny), 128, 0, ctx->ws>>>(
            ctx->p64[0], ctx->ec64, ctx->nx, ctx->ny, ctx->m, ctx->ncx, ctx->ncy, ctx->bcmask, ISM_COARSE_ISM,
            ctx->st, 0, &ctx->st->done);
        ISM_LAUNCH_CHECK(ctx);
        if (ctx->singular) TRY(remove_mean(ctx, ctx->p64[0]));
        // fine sweeps in chunks, the criterion after every sweep
        const int hx = (ctx->nx + 1) / 2;
        const dim3 gs((hx + 127) / 128, ctx->ny);
        const int C = ctx->opt.check_every;
        for (;;) {
            for (int c = 0; c < C; ++c) {
                for (int col = 0; col < 2; ++col) {
                    k_rbgs_colour<double><<<gs, 128, 0, ctx->ws>>>(ctx->p64[0], ctx->b64, ctx->nx, ctx->ny,
                                                                   ctx->bcmask, col, &ctx->st->done);
                    ISM_LAUNCH_CHECK(ctx);
                }
                k_resmax<<<G, T, 0, ctx->ws>>>(ctx->p64[0], ctx->b64, ctx->partials, ctx->nx, ctx->ny, ctx->bcmask,
                                               ctx->st, tol, max_sweeps, 0);
                ISM_LAUNCH_CHECK(ctx);
            }
            ISM_CUDA_TRY(cudaMemcpyAsync(&h, ctx->st, offsetof(IsmState, hist), cudaMemcpyDeviceToHost, ctx->ws));
            ISM_CUDA_TRY(cudaStreamSynchronize(ctx->ws));
            if (h.done) break;
        }
    }
    // mean removal of the result (all Neumann); zeros for a zero right-hand side
    if (ctx->singular) TRY(remove_mean(ctx, ctx->p64[0]));
    else {
        k_finalize<<<4 * 152, 256, 0, ctx->ws>>>(ctx->p64[0], nullptr, ctx->p64[0], ctx->n, ctx->st, 0);
        ISM_LAUNCH_CHECK(ctx);
    }
    ISM_CUDA_TRY(cudaMemcpyAsync(&h, ctx->st, offsetof(IsmState, hist), cudaMemcpyDeviceToHost, ctx->ws));
    ISM_CUDA_TRY(cudaStreamSynchronize(ctx->ws));
    ctx->last_cycles = h.cycles;
    ctx->last_outer = h.outer;
    ctx->last_relres = h.relres;
    ctx->last_status = h.status;
    ctx->last_nhist = 0;
    return (ism_status)h.status;
}
