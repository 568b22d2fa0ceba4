// ism_adjoint.cu -- hand-written adjoint of the projection step (proj_step).
//
// Forward (ism_proj.cu, Sec. 2.2-2.3, Eq. 3-4):
//   v*  = Pred(v, p)                       predictor (nonlinear in v, linear in p)
//   b   = (h/dt) D v*                      divergence, mean removed when all-Neumann
//   dp  = Pi A_f^+ Pi b                    ISM solve (Pi: mean removal)
//   v'  = v* - (dt/h) G dp                 on the faces the projection corrects
//   p'  = p + dp
// Given the adjoints (v-bar', p-bar') of the outputs, the adjoints of the
// inputs are, in reverse order:
//   dp-bar = p-bar' - (dt/h) G^T v-bar'    (transposed correction)
//   b-bar  = Pi A_f^+ Pi dp-bar            (A_f is symmetric: the same ISM solve)
//   v*-bar = v-bar' + (h/dt) D^T b-bar     (transposed divergence)
//   (v-bar, p-bar) = J_Pred(v, p)^T v*-bar,  p-bar += p-bar'
// The predictor's Jacobian is evaluated at the input velocities (the step is
// linear in p), so the adjoint needs only the step's input u and v.  Every transpose is written in gather form
// (each input entry sums the terms of all outputs that read it), so results
// are deterministic.  Entries of u* / v* that the predictor prescribes
// (walls, inlet) do not depend on the inputs and carry no adjoint.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "ism_kernels.cuh"

struct AdjArgs {
    int nx, ny;
    float ih, dt, nu;
    int vbc[4];
    float wall_u[4];
    float conv_u;
};

// d(ghost)/d(inner) of a tangential ghost value (see tangential_ghost)
__device__ __forceinline__ float dghost(int kind)
{
    return (kind == ISM_VEL_NOSLIP || kind == ISM_VEL_INFLOW) ? -1.0f : 1.0f;
}
__device__ __forceinline__ float ghostv(int kind, float wall, float inner)
{
    switch (kind) {
    case ISM_VEL_NOSLIP: return 2.0f * wall - inner;
    case ISM_VEL_INFLOW: return -inner;
    default: return inner;
    }
}

#define UA(i, j) u[(size_t)(j) * (nx + 1) + (i)]
#define VA(i, j) v[(size_t)(j) * nx + (i)]

// ---------------------------------------------------------------- 1. transposed correction
// dp-bar = p-bar' + (dt/h) (sum over corrected faces of +-u-bar'), in double.
__global__ void k_adj_correct(const float *__restrict__ gu, const float *__restrict__ gv,
                              const float *__restrict__ gp, double *__restrict__ dpbar, int nx, int ny,
                              double s, int outflow_e)
{
    const int j = blockIdx.y, i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nx) return;
    const float *u = gu, *v = gv;
    double acc = gp[(size_t)j * nx + i];
    if (i >= 1) acc -= s * (double)UA(i, j);                    // cell is R of its west face
    if (i + 1 <= nx - 1) acc += s * (double)UA(i + 1, j);      // cell is L of its east face
    if (i == nx - 1 && outflow_e) acc += 2.0 * s * (double)UA(nx, j);
    if (j >= 1) acc -= s * (double)VA(i, j);
    if (j + 1 <= ny - 1) acc += s * (double)VA(i, j + 1);
    dpbar[(size_t)j * nx + i] = acc;
}

// ---------------------------------------------------------------- 3. transposed divergence
// u*-bar = u-bar' + (h/dt)(b-bar of the cell west of the face - b-bar of the cell east)
__global__ void k_adj_div_u(const float *__restrict__ gu, const double *__restrict__ bbar,
                            float *__restrict__ gus, int nx, int ny, double c)
{
    const int j = blockIdx.y, i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > nx) return;
    double acc = gu[(size_t)j * (nx + 1) + i];
    if (i >= 1) acc += c * bbar[(size_t)j * nx + i - 1];
    if (i <= nx - 1) acc -= c * bbar[(size_t)j * nx + i];
    gus[(size_t)j * (nx + 1) + i] = (float)acc;
}

__global__ void k_adj_div_v(const float *__restrict__ gv, const double *__restrict__ bbar,
                            float *__restrict__ gvs, int nx, int ny, double c)
{
    const int j = blockIdx.y, i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nx) return;
    double acc = gv[(size_t)j * nx + i];
    if (j >= 1) acc += c * bbar[(size_t)(j - 1) * nx + i];
    if (j <= ny - 1) acc -= c * bbar[(size_t)j * nx + i];
    gvs[(size_t)j * nx + i] = (float)acc;
}

// ---------------------------------------------------------------- 4. transposed predictor
// Output u-face (i, j) is "free" (depends on inputs) when 1 <= i <= nx-1, or
// i == nx with a convective outflow; output v-face when 1 <= j <= ny-1.
__device__ __forceinline__ bool ufree(int i, int nx, const AdjArgs &a)
{
    return (i >= 1 && i <= nx - 1) || (i == nx && a.vbc[1] == ISM_VEL_OUTFLOW);
}

// transverse averages and ghost-aware neighbours at output faces
__device__ __forceinline__ float vbar_at(const float *v, int i, int j, int nx)
{
    return 0.25f * (VA(i - 1, j) + VA(i, j) + VA(i - 1, j + 1) + VA(i, j + 1));
}
__device__ __forceinline__ float ubar_at(const float *u, int i, int j, int nx)
{
    return 0.25f * (UA(i, j - 1) + UA(i + 1, j - 1) + UA(i, j) + UA(i + 1, j));
}

// u-bar_g for input u-face g = (i, j), and the contribution of u-faces to p-bar
__global__ void k_adj_pred_u(const float *__restrict__ u, const float *__restrict__ v,
                             const float *__restrict__ gus, const float *__restrict__ gvs,
                             float *__restrict__ gu_out, AdjArgs a)
{
    const int nx = a.nx, ny = a.ny;
    const int j = blockIdx.y, i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > nx) return;
    const float ih = a.ih, dt = a.dt, nu = a.nu, h2 = ih * ih, hh = 0.5f * ih;
    auto UB = [&](int ii, int jj) -> float { return gus[(size_t)jj * (nx + 1) + ii]; };
    auto VB = [&](int ii, int jj) -> float { return gvs[(size_t)jj * nx + ii]; };
    double acc = 0.0;
    // (a) own output face
    if (i >= 1 && i <= nx - 1) {
        const float dS = (j > 0) ? 0.0f : dghost(a.vbc[2]);
        const float dN = (j < ny - 1) ? 0.0f : dghost(a.vbc[3]);
        const float vb = vbar_at(v, i, j, nx);
        const float d = 1.0f + dt * (-(UA(i + 1, j) - UA(i - 1, j)) * hh - vb * (dN - dS) * hh +
                                     nu * (dN + dS - 4.0f) * h2);
        acc += (double)UB(i, j) * d;
    } else if (i == nx && a.vbc[1] == ISM_VEL_OUTFLOW) {
        acc += (double)UB(i, j) * (1.0f - dt * a.conv_u * ih);
    }
    // (b) g is uw of output face (i+1, j)
    if (i + 1 <= nx - 1) acc += (double)UB(i + 1, j) * dt * (UA(i + 1, j) * hh + nu * h2);
    else if (i + 1 == nx && a.vbc[1] == ISM_VEL_OUTFLOW) acc += (double)UB(nx, j) * dt * a.conv_u * ih;
    // (c) g is ue of output face (i-1, j)
    if (i - 1 >= 1 && i - 1 <= nx - 1) acc += (double)UB(i - 1, j) * dt * (-UA(i - 1, j) * hh + nu * h2);
    // (d) g is usx of output face (i, j+1); (e) g is unx of output face (i, j-1)
    if (i >= 1 && i <= nx - 1) {
        if (j + 1 <= ny - 1) acc += (double)UB(i, j + 1) * dt * (vbar_at(v, i, j + 1, nx) * hh + nu * h2);
        if (j - 1 >= 0) acc += (double)UB(i, j - 1) * dt * (-vbar_at(v, i, j - 1, nx) * hh + nu * h2);
    }
    // (f) g enters ubar of output v-faces (i, j), (i-1, j), (i, j+1), (i-1, j+1)
    const int fi[4] = {i, i - 1, i, i - 1}, fj[4] = {j, j, j + 1, j + 1};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int ii = fi[k], jj = fj[k];
        if (ii < 0 || ii > nx - 1 || jj < 1 || jj > ny - 1) continue;
        const float vc = VA(ii, jj);
        const float vw = (ii > 0) ? VA(ii - 1, jj) : ghostv(a.vbc[0], a.wall_u[0], vc);
        const float ve = (ii < nx - 1) ? VA(ii + 1, jj) : ghostv(a.vbc[1], a.wall_u[1], vc);
        acc += (double)VB(ii, jj) * dt * (-0.25f * (ve - vw) * hh);
    }
    gu_out[(size_t)j * (nx + 1) + i] = (float)acc;
}

// v-bar_g for input v-face g = (i, j)
__global__ void k_adj_pred_v(const float *__restrict__ u, const float *__restrict__ v,
                             const float *__restrict__ gus, const float *__restrict__ gvs,
                             float *__restrict__ gv_out, AdjArgs a)
{
    const int nx = a.nx, ny = a.ny;
    const int j = blockIdx.y, i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nx) return;
    const float ih = a.ih, dt = a.dt, nu = a.nu, h2 = ih * ih, hh = 0.5f * ih;
    auto UB = [&](int ii, int jj) -> float { return gus[(size_t)jj * (nx + 1) + ii]; };
    auto VB = [&](int ii, int jj) -> float { return gvs[(size_t)jj * nx + ii]; };
    double acc = 0.0;
    // (a) own output face
    if (j >= 1 && j <= ny - 1) {
        const float dW = (i > 0) ? 0.0f : dghost(a.vbc[0]);
        const float dE = (i < nx - 1) ? 0.0f : dghost(a.vbc[1]);
        const float ub = ubar_at(u, i, j, nx);
        const float d = 1.0f + dt * (-ub * (dE - dW) * hh - (VA(i, j + 1) - VA(i, j - 1)) * hh +
                                     nu * (dE + dW - 4.0f) * h2);
        acc += (double)VB(i, j) * d;
    }
    // (b) g is vsy of output face (i, j+1); (c) g is vny of output face (i, j-1)
    if (j + 1 >= 1 && j + 1 <= ny - 1) acc += (double)VB(i, j + 1) * dt * (VA(i, j + 1) * hh + nu * h2);
    if (j - 1 >= 1 && j - 1 <= ny - 1) acc += (double)VB(i, j - 1) * dt * (-VA(i, j - 1) * hh + nu * h2);
    // (d) g is vw of output face (i+1, j); (e) g is ve of output face (i-1, j)
    if (j >= 1 && j <= ny - 1) {
        if (i + 1 <= nx - 1) acc += (double)VB(i + 1, j) * dt * (ubar_at(u, i + 1, j, nx) * hh + nu * h2);
        if (i - 1 >= 0) acc += (double)VB(i - 1, j) * dt * (-ubar_at(u, i - 1, j, nx) * hh + nu * h2);
    }
    // (f) g enters vbar of output u-faces (i, j), (i+1, j), (i, j-1), (i+1, j-1)
    const int fi[4] = {i, i + 1, i, i + 1}, fj[4] = {j, j, j - 1, j - 1};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int ii = fi[k], jj = fj[k];
        if (ii < 1 || ii > nx - 1 || jj < 0 || jj > ny - 1) continue;
        const float uc = UA(ii, jj);
        const float usx = (jj > 0) ? UA(ii, jj - 1) : ghostv(a.vbc[2], a.wall_u[2], uc);
        const float unx = (jj < ny - 1) ? UA(ii, jj + 1) : ghostv(a.vbc[3], a.wall_u[3], uc);
        acc += (double)UB(ii, jj) * dt * (-0.25f * (unx - usx) * hh);
    }
    gv_out[(size_t)j * nx + i] = (float)acc;
}

// p-bar = p-bar' + (pressure-gradient terms of the predictor)^T v*-bar
__global__ void k_adj_pred_p(const float *__restrict__ gus, const float *__restrict__ gvs,
                             float *__restrict__ gp, AdjArgs a)
{
    const int nx = a.nx, ny = a.ny;
    const int j = blockIdx.y, i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nx) return;
    const double c = (double)a.dt * (double)a.ih;
    double acc = gp[(size_t)j * nx + i];
    if (i >= 1) acc -= c * gus[(size_t)j * (nx + 1) + i];
    if (i + 1 <= nx - 1) acc += c * gus[(size_t)j * (nx + 1) + i + 1];
    if (i == nx - 1 && a.vbc[1] == ISM_VEL_OUTFLOW) acc += 2.0 * c * gus[(size_t)j * (nx + 1) + nx];
    if (j >= 1) acc -= c * gvs[(size_t)j * nx + i];
    if (j + 1 <= ny - 1) acc += c * gvs[(size_t)(j + 1) * nx + i];
    gp[(size_t)j * nx + i] = (float)acc;
}

#undef UA
#undef VA

// ---------------------------------------------------------------- enstrophy loss
// Vorticity at the interior grid nodes (1 <= i <= nx-1, 1 <= j <= ny-1):
//   w_ij = (v[j][i] - v[j][i-1]) / h - (u[j][i] - u[j-1][i]) / h,
// loss E = 1/2 sum w_ij^2 h^2 (boundary nodes, whose vorticity involves the
// wall velocity, are left out).
__device__ __forceinline__ double node_w(const float *u, const float *v, int i, int j, int nx,
                                         double ih)
{
    return ((double)v[(size_t)j * nx + i] - (double)v[(size_t)j * nx + i - 1] -
            (double)u[(size_t)j * (nx + 1) + i] + (double)u[(size_t)(j - 1) * (nx + 1) + i]) * ih;
}

__global__ void k_enstrophy(const float *__restrict__ u, const float *__restrict__ v, int nx, int ny,
                            double h, double *partials)
{
    const long long nn = (long long)(nx - 1) * (ny - 1);
    const double ih = 1.0 / h;
    double acc = 0.0;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < nn;
         k += (long long)gridDim.x * blockDim.x) {
        const int i = 1 + (int)(k % (nx - 1)), j = 1 + (int)(k / (nx - 1));
        const double w = node_w(u, v, i, j, nx, ih);
        acc += w * w;
    }
    double q[1] = {0.5 * h * h * acc};
    block_partials<1>(q, partials, gridDim.x, blockIdx.x);
}

// one warp sums the block partials in a fixed order
__global__ void k_sum_partials(const double *__restrict__ partials, int nblk, double *out)
{
    double t = 0.0;
    for (int k = threadIdx.x; k < nblk; k += 32) t += partials[k];
    t = warp_sum(t);
    if (threadIdx.x == 0) *out = t;
}

// dE/du[j][i] = h (w_{i,j+1} - w_{i,j}),  dE/dv[j][i] = h (w_{i,j} - w_{i+1,j}),
// each node term present only for interior nodes.
__global__ void k_enstrophy_grad_u(const float *__restrict__ u, const float *__restrict__ v,
                                   float *__restrict__ gu, int nx, int ny, double h)
{
    const int j = blockIdx.y, i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > nx) return;
    const double ih = 1.0 / h;
    double g = 0.0;
    if (i >= 1 && i <= nx - 1) {
        if (j + 1 <= ny - 1) g += node_w(u, v, i, j + 1, nx, ih);
        if (j >= 1) g -= node_w(u, v, i, j, nx, ih);
    }
    gu[(size_t)j * (nx + 1) + i] = (float)(h * g);
}

__global__ void k_enstrophy_grad_v(const float *__restrict__ u, const float *__restrict__ v,
                                   float *__restrict__ gv, int nx, int ny, double h)
{
    const int j = blockIdx.y, i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nx) return;
    const double ih = 1.0 / h;
    double g = 0.0;
    if (j >= 1 && j <= ny - 1) {
        if (i >= 1) g += node_w(u, v, i, j, nx, ih);
        if (i + 1 <= nx - 1) g -= node_w(u, v, i + 1, j, nx, ih);
    }
    gv[(size_t)j * nx + i] = (float)(h * g);
}

// ---------------------------------------------------------------- host

#define TRY(x)                                                                   \
    do {                                                                         \
        ism_status _s = (x);                                                     \
        if (_s != ISM_OK) return _s;                                             \
    } while (0)

extern "C" ism_status proj_step_adjoint(ism_ctx *ctx, const float *u, const float *v, double dt,
                                        double nu, float *gu, float *gv, float *gp)
{
    if (!ctx || !u || !v || !gu || !gv || !gp || !(dt > 0.0) || !(nu >= 0.0) || !isfinite(dt) ||
        !isfinite(nu))
        return ISM_ERR_ARG;
    if (!ctx->flow_set) return ISM_ERR_ARG;
    // the transposed step is written for walls, inflow and outflow faces
    for (int f = 0; f < 4; ++f)
        if (ctx->vel_bc[f] == ISM_VEL_PERIODIC) return ISM_ERR_ARG;
    TRY(ism_proj_buffers(ctx));
    TRY(ism_enter(ctx));
    const int nx = ctx->nx, ny = ctx->ny, T = 128;
    const double s = dt / ctx->h;
    const int outflow = ctx->vel_bc[1] == ISM_VEL_OUTFLOW;
    // 1. dp-bar (double) into the right-hand-side buffer of the adjoint solve;
    //    the forward increment ctx->dp (warm start) is left untouched
    k_adj_correct<<<dim3((nx + T - 1) / T, ny), T, 0, ctx->ws>>>(gu, gv, gp, ctx->b64, nx, ny, s, outflow);
    ISM_LAUNCH_CHECK(ctx);
    // 2. b-bar = Pi A^+ Pi dp-bar with the ISM solve (the operator is symmetric)
    IsmState h0;
    memset(&h0, 0, offsetof(IsmState, hist));
    h0.inv_n = 1.0 / (double)ctx->n;
    ISM_CUDA_TRY(cudaMemcpyAsync(ctx->st, &h0, offsetof(IsmState, hist), cudaMemcpyHostToDevice, ctx->ws));
    TRY(ism_prepare_rhs(ctx, ctx->b64));
    ISM_CUDA_TRY(cudaMemsetAsync(ctx->p64[0], 0, (size_t)ctx->n * 8, ctx->ws));
    ism_status st = ism_solve_internal(ctx, ctx->proj_tol, ctx->proj_max_cycles, false);
    if (st != ISM_OK && st != ISM_ERR_NOT_CONVERGED) {
        ism_leave(ctx);
        return st;
    }
    // 3. u*-bar, v*-bar (in the predicted-velocity buffers)
    const double c = ctx->h / dt;
    k_adj_div_u<<<dim3((nx + 1 + T - 1) / T, ny), T, 0, ctx->ws>>>(gu, ctx->p64[0], ctx->us, nx, ny, c);
    ISM_LAUNCH_CHECK(ctx);
    k_adj_div_v<<<dim3((nx + T - 1) / T, ny + 1), T, 0, ctx->ws>>>(gv, ctx->p64[0], ctx->vs, nx, ny, c);
    ISM_LAUNCH_CHECK(ctx);
    // 4. predictor transpose: u-bar, v-bar overwrite gu, gv; p-bar accumulates into gp
    AdjArgs a;
    a.nx = nx; a.ny = ny;
    a.ih = (float)(1.0 / ctx->h);
    a.dt = (float)dt;
    a.nu = (float)nu;
    for (int k = 0; k < 4; ++k) { a.vbc[k] = ctx->vel_bc[k]; a.wall_u[k] = (float)ctx->wall_u[k]; }
    a.conv_u = (float)ctx->conv_u;
    k_adj_pred_u<<<dim3((nx + 1 + T - 1) / T, ny), T, 0, ctx->ws>>>(u, v, ctx->us, ctx->vs, gu, a);
    ISM_LAUNCH_CHECK(ctx);
    k_adj_pred_v<<<dim3((nx + T - 1) / T, ny + 1), T, 0, ctx->ws>>>(u, v, ctx->us, ctx->vs, gv, a);
    ISM_LAUNCH_CHECK(ctx);
    k_adj_pred_p<<<dim3((nx + T - 1) / T, ny), T, 0, ctx->ws>>>(ctx->us, ctx->vs, gp, a);
    ISM_LAUNCH_CHECK(ctx);
    TRY(ism_leave(ctx));
    return st;
}

static ism_status ensure_scal(ism_ctx *ctx)
{
    if (ctx->scal) return ISM_OK;
    if (cudaMalloc((void **)&ctx->scal, 8 * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return ISM_ERR_NOMEM;
    }
    return ISM_OK;
}

// Loss into ctx->scal[slot] (device), gradient into (gu, gv) when given.
static ism_status enstrophy_launch(ism_ctx *ctx, const float *u, const float *v, int slot, float *gu,
                                   float *gv)
{
    const int nx = ctx->nx, ny = ctx->ny, T = 128, G = 4 * 152;
    if (nx >= 2 && ny >= 2) {
        k_enstrophy<<<G, 256, 0, ctx->ws>>>(u, v, nx, ny, ctx->h, ctx->partials);
        ISM_LAUNCH_CHECK(ctx);
        k_sum_partials<<<1, 32, 0, ctx->ws>>>(ctx->partials, G, ctx->scal + slot);
        ISM_LAUNCH_CHECK(ctx);
    } else {
        ISM_CUDA_TRY(cudaMemsetAsync(ctx->scal + slot, 0, sizeof(double), ctx->ws));
    }
    if (gu) {
        k_enstrophy_grad_u<<<dim3((nx + 1 + T - 1) / T, ny), T, 0, ctx->ws>>>(u, v, gu, nx, ny, ctx->h);
        ISM_LAUNCH_CHECK(ctx);
    }
    if (gv) {
        k_enstrophy_grad_v<<<dim3((nx + T - 1) / T, ny + 1), T, 0, ctx->ws>>>(u, v, gv, nx, ny, ctx->h);
        ISM_LAUNCH_CHECK(ctx);
    }
    return ISM_OK;
}

extern "C" ism_status ism_enstrophy(ism_ctx *ctx, const float *u, const float *v, double *value,
                                    float *gu, float *gv)
{
    if (!ctx || !u || !v || (!value && !gu && !gv)) return ISM_ERR_ARG;
    TRY(ensure_scal(ctx));
    TRY(ism_enter(ctx));
    TRY(enstrophy_launch(ctx, u, v, 0, gu, gv));
    if (value) ISM_CUDA_TRY(cudaMemcpyAsync(ctx->st_host, ctx->scal, sizeof(double), cudaMemcpyDeviceToHost, ctx->ws));
    TRY(ism_leave(ctx));
    if (value) {
        ISM_CUDA_TRY(cudaStreamSynchronize(ctx->ws));
        memcpy(value, ctx->st_host, sizeof(double));
    }
    return ISM_OK;
}

// ---------------------------------------------------------------- checkpointed rollout
//
// Forward: S steps of proj_step from (u0, v0, p0), keeping the state before
// every `every`-th step (u, v, p and, for warm-started solves, the previous
// increment dp).  Loss: enstrophy of the final velocity.  Reverse: for each
// segment, last first, the forward steps are replayed from its checkpoint
// (bit-identical: same inputs, same deterministic kernels) keeping each
// step's input velocities, then the adjoint steps run backwards through the
// segment.  Memory: (S/every + 1) checkpoints + `every` segment states.

namespace {
struct RollLayout {
    size_t nu, nv, np;         // elements per field
    size_t ck_bytes, seg_bytes, total;
    int nck;
};
}

static RollLayout roll_layout(const ism_ctx *ctx, int steps, int every)
{
    RollLayout L;
    L.nu = (size_t)(ctx->nx + 1) * ctx->ny;
    L.nv = (size_t)ctx->nx * (ctx->ny + 1);
    L.np = (size_t)ctx->nx * ctx->ny;
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    L.ck_bytes = up(L.nu * 4) + up(L.nv * 4) + up(L.np * 4) + up(L.np * 8);
    L.seg_bytes = up(L.nu * 4) + up(L.nv * 4);
    L.nck = (steps + every - 1) / every;
    // working state (one checkpoint-sized slot) + checkpoints + segment states
    L.total = L.ck_bytes * (size_t)(L.nck + 1) + L.seg_bytes * (size_t)every;
    return L;
}

struct CkPtr { float *u, *v, *p; double *dp; };

static CkPtr ck_slot(const ism_ctx *ctx, const RollLayout &L, int k)
{
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    char *b = (char *)ctx->roll + L.ck_bytes * (size_t)k;
    CkPtr c;
    c.u = (float *)b;
    c.v = (float *)(b + up(L.nu * 4));
    c.p = (float *)(b + up(L.nu * 4) + up(L.nv * 4));
    c.dp = (double *)(b + up(L.nu * 4) + up(L.nv * 4) + up(L.np * 4));
    return c;
}

static void seg_slot(const ism_ctx *ctx, const RollLayout &L, int k, float **u, float **v)
{
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    char *b = (char *)ctx->roll + L.ck_bytes * (size_t)(L.nck + 1) + L.seg_bytes * (size_t)k;
    *u = (float *)b;
    *v = (float *)(b + up(L.nu * 4));
}

static ism_status copy_state(ism_ctx *ctx, const RollLayout &L, const CkPtr &dst, const float *u,
                             const float *v, const float *p, const double *dp)
{
    ISM_CUDA_TRY(cudaMemcpyAsync(dst.u, u, L.nu * 4, cudaMemcpyDeviceToDevice, ctx->ws));
    ISM_CUDA_TRY(cudaMemcpyAsync(dst.v, v, L.nv * 4, cudaMemcpyDeviceToDevice, ctx->ws));
    ISM_CUDA_TRY(cudaMemcpyAsync(dst.p, p, L.np * 4, cudaMemcpyDeviceToDevice, ctx->ws));
    if (dp && dst.dp) ISM_CUDA_TRY(cudaMemcpyAsync(dst.dp, dp, L.np * 8, cudaMemcpyDeviceToDevice, ctx->ws));
    return ISM_OK;
}

static ism_status worst(ism_status a, ism_status b) { return a != ISM_OK ? a : b; }

extern "C" ism_status proj_rollout_grad(ism_ctx *ctx, const float *u0, const float *v0, const float *p0,
                                        double dt, double nu, int steps, int every, double *loss,
                                        float *gu, float *gv, float *gp)
{
    if (!ctx || !u0 || !v0 || !p0 || steps < 0 || every < 1 || !(dt > 0.0) || !(nu >= 0.0))
        return ISM_ERR_ARG;
    const bool grad = gu || gv || gp;
    if (grad && !(gu && gv && gp)) return ISM_ERR_ARG;
    if (!ctx->flow_set) return ISM_ERR_ARG;
    if (steps == 0) every = 1;
    TRY(ism_proj_buffers(ctx));
    TRY(ensure_scal(ctx));
    const RollLayout L = roll_layout(ctx, steps, every);
    if (L.total > ctx->roll_bytes) {
        if (ctx->ws) cudaStreamSynchronize(ctx->ws);
        if (ctx->roll) cudaFree(ctx->roll);
        ctx->roll = nullptr;
        ctx->roll_bytes = 0;
        if (cudaMalloc(&ctx->roll, L.total) != cudaSuccess) {
            cudaGetLastError();
            return ISM_ERR_NOMEM;
        }
        ctx->roll_bytes = L.total;
    }
    // ordering against the caller's stream: ism_enter/leave around the whole
    // call; proj_step / proj_step_adjoint re-enter, which only adds event waits
    TRY(ism_enter(ctx));
    const CkPtr cur = ck_slot(ctx, L, L.nck);      // working state
    TRY(copy_state(ctx, L, cur, u0, v0, p0, nullptr));
    ISM_CUDA_TRY(cudaMemsetAsync(ctx->dp, 0, L.np * 8, ctx->ws));
    ism_status agg = ISM_OK;
    for (int s = 0; s < steps; ++s) {
        if (grad && s % every == 0) TRY(copy_state(ctx, L, ck_slot(ctx, L, s / every), cur.u, cur.v, cur.p, ctx->dp));
        const ism_status st = proj_step(ctx, cur.u, cur.v, cur.p, dt, nu);
        if (st != ISM_OK && st != ISM_ERR_NOT_CONVERGED) return st;
        agg = worst(agg, st);
    }
    TRY(enstrophy_launch(ctx, cur.u, cur.v, 0, grad ? gu : nullptr, grad ? gv : nullptr));
    if (grad) ISM_CUDA_TRY(cudaMemsetAsync(gp, 0, L.np * 4, ctx->ws));
    // read the loss now: the solves of the reverse sweep reuse the pinned buffer
    double loss_h = 0.0;
    if (loss) {
        ISM_CUDA_TRY(cudaMemcpyAsync(ctx->st_host, ctx->scal, sizeof(double), cudaMemcpyDeviceToHost, ctx->ws));
        ISM_CUDA_TRY(cudaStreamSynchronize(ctx->ws));
        memcpy(&loss_h, ctx->st_host, sizeof(double));
    }
    if (grad) {
        for (int seg = L.nck - 1; seg >= 0; --seg) {
            const int s0 = seg * every, s1 = std::min(steps, s0 + every);
            const CkPtr ck = ck_slot(ctx, L, seg);
            TRY(copy_state(ctx, L, cur, ck.u, ck.v, ck.p, nullptr));
            ISM_CUDA_TRY(cudaMemcpyAsync(ctx->dp, ck.dp, L.np * 8, cudaMemcpyDeviceToDevice, ctx->ws));
            for (int s = s0; s < s1; ++s) {
                float *su, *sv;
                seg_slot(ctx, L, s - s0, &su, &sv);
                ISM_CUDA_TRY(cudaMemcpyAsync(su, cur.u, L.nu * 4, cudaMemcpyDeviceToDevice, ctx->ws));
                ISM_CUDA_TRY(cudaMemcpyAsync(sv, cur.v, L.nv * 4, cudaMemcpyDeviceToDevice, ctx->ws));
                if (s + 1 < s1) {      // the segment's last output is not needed
                    const ism_status st = proj_step(ctx, cur.u, cur.v, cur.p, dt, nu);
                    if (st != ISM_OK && st != ISM_ERR_NOT_CONVERGED) return st;
                }
            }
            for (int s = s1 - 1; s >= s0; --s) {
                float *su, *sv;
                seg_slot(ctx, L, s - s0, &su, &sv);
                const ism_status st = proj_step_adjoint(ctx, su, sv, dt, nu, gu, gv, gp);
                if (st != ISM_OK && st != ISM_ERR_NOT_CONVERGED) return st;
                agg = worst(agg, st);
            }
        }
    }
    TRY(ism_leave(ctx));
    ISM_CUDA_TRY(cudaStreamSynchronize(ctx->ws));
    if (loss) *loss = loss_h;
    return agg;
}
