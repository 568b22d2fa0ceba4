// ism_tune.cu -- choices the paper made by hand, made by timing here:
// the coarsening factor of a context (16h or 32h, Sec. 4.1 and 4.3.1 tune the
// tile size by hand) and the sweeps per cycle of a batched ensemble.
#include <math.h>

#include <algorithm>
#include <chrono>
#include <vector>

#include "ism_kernels.cuh"

namespace {

// Test right-hand side for timing: a few smooth modes plus a small
// deterministic hash component, so that both the smooth and the rough parts
// of the spectrum are present (the solver removes the mean when needed).
__global__ void k_tune_rhs(double *b, int nx, int ny)
{
    const int j = blockIdx.y, i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nx) return;
    const double x = (i + 0.5) / nx, y = (j + 0.5) / ny, pi = 3.141592653589793;
    const unsigned hsh = ((unsigned)i * 73856093u) ^ ((unsigned)j * 19349663u);
    b[(size_t)j * nx + i] = cos(3.0 * pi * x) * cos(2.0 * pi * y) + 0.5 * sin(5.0 * pi * x + 1.0) * cos(7.0 * pi * y) +
                            0.05 * ((double)(hsh & 1023u) / 1024.0 - 0.5);
}

double time_solve(ism_ctx *ctx, const double *b, double *p, double tol)
{
    double best = 1e30;
    for (int rep = 0; rep < 2; ++rep) {           // the first solve also builds the graph
        if (cudaMemsetAsync(p, 0, (size_t)ctx->n * 8, ctx->user_stream) != cudaSuccess) return 1e30;
        if (cudaStreamSynchronize(ctx->user_stream) != cudaSuccess) return 1e30;
        const auto t0 = std::chrono::steady_clock::now();
        int cyc = 0;
        double rr = 0.0;
        const ism_status s = ism_solve(ctx, b, p, tol, 100000, &cyc, &rr);
        const auto t1 = std::chrono::steady_clock::now();
        if (s != ISM_OK) return 1e30;
        if (rep) best = std::chrono::duration<double>(t1 - t0).count();
    }
    return best;
}

}  // namespace

extern "C" ism_status ism_setup(int nx, int ny, double h, const int bc[4], int coarsen, ism_precision prec,
                                void *stream, ism_ctx **out)
{
    if (coarsen != 0) return ism_setup_fixed(nx, ny, h, bc, coarsen, prec, stream, out);
    // the argument checks of ism_setup_fixed that do not depend on m, first
    if (!out || !bc || nx <= 0 || ny <= 0 || !(h > 0.0) || !isfinite(h)) return ISM_ERR_ARG;
    if ((long long)nx * ny > (1LL << 31) || nx > (1 << 20) || ny > (1 << 20)) return ISM_ERR_ARG;
    const int mask = ism_bc_mask(bc);
    if (mask < 0) return ISM_ERR_ARG;
    if (prec != ISM_FP64 && prec != ISM_MIXED) return ISM_ERR_ARG;
    std::vector<int> cand;
    const int minx = (mask & ISM_PER_X) ? 4 : 2, miny = (mask & ISM_PER_Y) ? 4 : 2;
    for (int m : {16, 32})
        if (nx % m == 0 && ny % m == 0 && nx / m >= minx && ny / m >= miny && nx / m <= 1024 && ny / m <= 1024)
            cand.push_back(m);
    if (cand.empty()) return ISM_ERR_ARG;
    if (cand.size() == 1) return ism_setup_fixed(nx, ny, h, bc, cand[0], prec, stream, out);
    double *b = nullptr, *p = nullptr;
    const size_t bytes = (size_t)nx * ny * 8;
    if (cudaMalloc((void **)&b, bytes) != cudaSuccess || cudaMalloc((void **)&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        if (b) cudaFree(b);
        return ISM_ERR_NOMEM;
    }
    k_tune_rhs<<<dim3((nx + 127) / 128, ny), 128, 0, (cudaStream_t)stream>>>(b, nx, ny);
    ism_status st = cudaGetLastError() == cudaSuccess ? ISM_OK : ISM_ERR_CUDA;
    ism_ctx *best = nullptr;
    double best_t = 1e30;
    for (size_t k = 0; k < cand.size() && st == ISM_OK; ++k) {
        ism_ctx *c = nullptr;
        st = ism_setup_fixed(nx, ny, h, bc, cand[k], prec, stream, &c);
        if (st != ISM_OK) break;
        const double t = time_solve(c, b, p, 1e-8);
        if (t < best_t) {
            if (best) ism_destroy(best);
            best = c;
            best_t = t;
        } else {
            ism_destroy(c);
        }
    }
    cudaFree(b);
    cudaFree(p);
    if (st != ISM_OK) {
        if (best) ism_destroy(best);
        return st;
    }
    if (!best) return ISM_ERR_NOT_CONVERGED;
    *out = best;
    return ISM_OK;
}

extern "C" int ism_coarsening(const ism_ctx *ctx) { return ctx ? ctx->m : 0; }

extern "C" ism_status ism_autotune_batched(int n, ism_ctx *const *ctxs, const double *const *rhs,
                                           double *const *p, double tol, int *nu_out)
{
    if (n < 1 || !ctxs || !rhs || !p || !(tol > 0.0)) return ISM_ERR_ARG;
    // (nu, coarse engine: 1 the tensor cores, single-CTA kernel where every
    // coarse grid allows it; 2 the tiled split-TF32 chain; 0 the CUDA cores)
    static const int cand[][2] = {{16, 1}, {32, 1}, {64, 1}, {128, 1}, {16, 2}, {32, 2},
                                  {64, 2}, {128, 2}, {16, 0}, {32, 0}, {64, 0}, {128, 0}};
    std::vector<ism_options> saved(n);
    for (int d = 0; d < n; ++d) {
        if (!ctxs[d] || !rhs[d] || !p[d]) return ISM_ERR_ARG;
        ism_get_options(ctxs[d], &saved[d]);
    }
    int best_nu = -1, best_tc = 0;
    double best_t = 1e30;
    ism_status st = ISM_OK;
    for (const auto &cd : cand) {
        const int nu = cd[0], tcflag = cd[1];
        for (int d = 0; d < n && st == ISM_OK; ++d) {
            ism_options o = saved[d];
            o.nu = nu;
            o.sweeps_per_pass = 8;
            o.coarse_tc = tcflag;
            st = ism_set_options(ctxs[d], &o);
        }
        if (st != ISM_OK) break;
        double t = 1e30;
        for (int rep = 0; rep < 2 && st == ISM_OK; ++rep) {     // the first call builds the graph
            for (int d = 0; d < n; ++d)
                if (cudaMemsetAsync(p[d], 0, (size_t)ctxs[d]->n * 8, ctxs[0]->user_stream) != cudaSuccess)
                    st = ISM_ERR_CUDA;
            if (cudaStreamSynchronize(ctxs[0]->user_stream) != cudaSuccess) st = ISM_ERR_CUDA;
            if (st != ISM_OK) break;
            const auto t0 = std::chrono::steady_clock::now();
            const ism_status s = ism_solve_batched(n, ctxs, rhs, p, tol, 200000, nullptr, nullptr);
            const auto t1 = std::chrono::steady_clock::now();
            if (s == ISM_ERR_ARG || s == ISM_ERR_CUDA || s == ISM_ERR_NOMEM) st = s;
            else if (s == ISM_OK && rep) t = std::chrono::duration<double>(t1 - t0).count();
        }
        if (st == ISM_OK && t < best_t) {
            best_t = t;
            best_nu = nu;
            best_tc = tcflag;
        }
    }
    if (st == ISM_OK && best_nu < 0) st = ISM_ERR_NOT_CONVERGED;
    for (int d = 0; d < n; ++d) {
        ism_options o = saved[d];
        if (st == ISM_OK) {
            o.nu = best_nu;
            o.sweeps_per_pass = 8;
            o.coarse_tc = best_tc;
        }
        ism_set_options(ctxs[d], &o);
    }
    if (st == ISM_OK && nu_out) *nu_out = best_nu;
    return st;
}
