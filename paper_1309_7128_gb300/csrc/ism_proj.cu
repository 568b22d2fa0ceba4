// ism_proj.cu -- projection time step around the ISM pressure solve.
//
// Goda incremental pressure correction (Sec. 2.2, Eq. 3-4) on the staggered
// MAC grid (Sec. 2.3), physical signs:
//   v* = v^n + dt [ -(v.grad) v + nu lap v - grad p^n ]   (forward Euler)
//   A_f dp = h (u_e - u_w + v_n - v_s)* / dt               (flux units)
//   v^{n+1} = v* - dt grad dp,   p^{n+1} = p^n + dp.
// Second-order central differences in advective form; the transverse
// velocity at a face is the average of the four nearest faces.  Velocities
// and pressure are single precision; the divergence and the correction are
// evaluated in double around the FP64 pressure increment.
#include <math.h>
#include <string.h>

#include "ism_kernels.cuh"

struct FlowArgs {
    int nx, ny;
    float ih, dt, nu;     // 1/h
    int vbc[4];
    float wall_u[4];
    const float *u_in;
    float conv_u;
};

// Ghost value of a tangential velocity beyond a face.
__device__ __forceinline__ float tangential_ghost(int kind, float wall, float inner)
{
    switch (kind) {
    case ISM_VEL_NOSLIP: return 2.0f * wall - inner;   // mean of inner and ghost = wall speed
    case ISM_VEL_INFLOW: return -inner;                // no tangential velocity at the inlet
    default: return inner;                             // free slip / outflow: zero gradient
    }
}

#define UA(i, j) u[(size_t)(j) * (nx + 1) + (i)]
#define VA(i, j) v[(size_t)(j) * nx + (i)]
#define PA(i, j) p[(size_t)(j) * nx + (i)]

__device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// x-face predictor; grid (ceil((nx+1)/128), ny).  Along a periodic x axis
// face 0 is computed like an interior face (its west neighbours wrap) and
// face nx, the same face, repeats that computation.
__global__ void k_predict_u(const float *__restrict__ u, const float *__restrict__ v,
                            const float *__restrict__ p, float *__restrict__ us, FlowArgs f)
{
    const int nx = f.nx, ny = f.ny;
    const int j = blockIdx.y, io = blockIdx.x * blockDim.x + threadIdx.x;
    if (io > nx) return;
    const bool px = f.vbc[0] == ISM_VEL_PERIODIC, py = f.vbc[2] == ISM_VEL_PERIODIC;
    const int i = (px && io == nx) ? 0 : io;
    const float uc = UA(i, j);
    float out;
    if (i == 0 && !px) {
        out = (f.vbc[0] == ISM_VEL_INFLOW) ? f.u_in[j] : 0.0f;
    } else if (i == nx && !px) {
        if (f.vbc[1] == ISM_VEL_OUTFLOW) {
            const float pin = PA(nx - 1, j);
            const float gp = (-pin - pin) * f.ih;                 // ghost -p: Dirichlet 0
            out = uc + f.dt * (-f.conv_u * (uc - UA(nx - 1, j)) * f.ih - gp);
        } else {
            out = 0.0f;
        }
    } else {
        const int im = wrapi(i - 1, nx), ip = px ? wrapi(i + 1, nx) : i + 1, jp = py ? wrapi(j + 1, ny) : j + 1;
        const float uw = UA(im, j), ue = UA(ip, j);
        const float usx = (j > 0) ? UA(i, j - 1) : (py ? UA(i, ny - 1) : tangential_ghost(f.vbc[2], f.wall_u[2], uc));
        const float unx = (j < ny - 1) ? UA(i, j + 1) : (py ? UA(i, 0) : tangential_ghost(f.vbc[3], f.wall_u[3], uc));
        const float vbar = 0.25f * (VA(im, j) + VA(i, j) + VA(im, jp) + VA(i, jp));
        const float adv = uc * (ue - uw) * (0.5f * f.ih) + vbar * (unx - usx) * (0.5f * f.ih);
        const float lap = (ue + uw + unx + usx - 4.0f * uc) * (f.ih * f.ih);
        const float gp = (PA(i, j) - PA(im, j)) * f.ih;
        out = uc + f.dt * (-adv + f.nu * lap - gp);
    }
    us[(size_t)j * (nx + 1) + io] = out;
}

// y-face predictor; grid (ceil(nx/128), ny+1).  South and north faces are
// walls, or along a periodic y axis face 0 is computed like an interior face
// and face ny repeats it.
__global__ void k_predict_v(const float *__restrict__ u, const float *__restrict__ v,
                            const float *__restrict__ p, float *__restrict__ vs, FlowArgs f)
{
    const int nx = f.nx, ny = f.ny;
    const int jo = blockIdx.y, i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nx) return;
    const bool px = f.vbc[0] == ISM_VEL_PERIODIC, py = f.vbc[2] == ISM_VEL_PERIODIC;
    const int j = (py && jo == ny) ? 0 : jo;
    float out = 0.0f;
    if (py || (j > 0 && j < ny)) {
        const int jm = wrapi(j - 1, ny), jp = py ? wrapi(j + 1, ny) : j + 1, ip = px ? wrapi(i + 1, nx) : i + 1;
        const float vc = VA(i, j);
        const float vsy = VA(i, jm), vny = VA(i, jp);
        const float vw = (i > 0) ? VA(i - 1, j) : (px ? VA(nx - 1, j) : tangential_ghost(f.vbc[0], f.wall_u[0], vc));
        const float ve = (i < nx - 1) ? VA(i + 1, j) : (px ? VA(0, j) : tangential_ghost(f.vbc[1], f.wall_u[1], vc));
        const float ubar = 0.25f * (UA(i, jm) + UA(ip, jm) + UA(i, j) + UA(ip, j));
        const float adv = ubar * (ve - vw) * (0.5f * f.ih) + vc * (vny - vsy) * (0.5f * f.ih);
        const float lap = (ve + vw + vny + vsy - 4.0f * vc) * (f.ih * f.ih);
        const float gp = (PA(i, j) - PA(i, jm)) * f.ih;
        out = vc + f.dt * (-adv + f.nu * lap - gp);
    }
    vs[(size_t)jo * nx + i] = out;
}

// b = h (u_e - u_w + v_n - v_s) / dt in double; partial sums of b and |b|.  h_dt =
// h / dt is formed once on the host: a double division per cell costs about
// ten operations of this GPU's slow FP64 pipe.
__global__ void k_divergence(const float *__restrict__ u, const float *__restrict__ v,
                             double *__restrict__ b, int nx, int ny, double h_dt, double *partials)
{
    const int j = blockIdx.y, i = blockIdx.x * blockDim.x + threadIdx.x;
    double s = 0.0, sa = 0.0;
    if (i < nx) {
        const double du = (double)UA(i + 1, j) - (double)UA(i, j);
        const double dv = (double)VA(i, j + 1) - (double)VA(i, j);
        const double val = h_dt * (du + dv);
        b[(size_t)j * nx + i] = val;
        s = val;
        sa = fabs(val);
    }
    double v2[2] = {s, sa};
    block_partials<2>(v2, partials, gridDim.x * gridDim.y, blockIdx.y * gridDim.x + blockIdx.x);
}

// v = v* - (dt/h) grad dp on the faces whose normal velocity is free
// (interior faces and the outflow face with its Dirichlet-0 ghost); p += dp.
__global__ void k_correct_u(float *__restrict__ u, const float *__restrict__ us,
                            const double *__restrict__ dp, int nx, int ny, double s, int outflow_e, int px)
{
    const int j = blockIdx.y, i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > nx) return;
    const size_t k = (size_t)j * (nx + 1) + i;
    double val = us[k];
    if (i > 0 && i < nx) val -= s * (dp[(size_t)j * nx + i] - dp[(size_t)j * nx + i - 1]);
    else if (px) val -= s * (dp[(size_t)j * nx] - dp[(size_t)j * nx + nx - 1]);   // faces 0 and nx: the same face
    else if (i == nx && outflow_e) {
        const double pin = dp[(size_t)j * nx + nx - 1];
        val -= s * (-pin - pin);
    }
    u[k] = (float)val;
}

__global__ void k_correct_v(float *__restrict__ v, const float *__restrict__ vs,
                            const double *__restrict__ dp, float *__restrict__ p, int nx, int ny,
                            double s, int py)
{
    const int j = blockIdx.y, i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nx) return;
    const size_t k = (size_t)j * nx + i;
    double val = vs[k];
    if (j > 0 && j < ny) val -= s * (dp[k] - dp[k - nx]);
    else if (py) val -= s * (dp[i] - dp[(size_t)(ny - 1) * nx + i]);         // faces 0 and ny: the same face
    v[k] = (float)val;
    if (j < ny) p[k] = (float)((double)p[k] + dp[k]);
}

#undef UA
#undef VA
#undef PA

// ------------------------------------------------------------------ host

#define TRY(x)                                                                   \
    do {                                                                         \
        ism_status _s = (x);                                                     \
        if (_s != ISM_OK) return _s;                                             \
    } while (0)

extern "C" ism_status ism_set_flow(ism_ctx *ctx, const int vel_bc[4], const double wall_u[4],
                                   const float *u_in, double conv_u)
{
    if (!ctx || !vel_bc || !wall_u) return ISM_ERR_ARG;
    for (int f = 0; f < 4; ++f) {
        if (vel_bc[f] < ISM_VEL_NOSLIP || vel_bc[f] > ISM_VEL_PERIODIC) return ISM_ERR_ARG;
        if (vel_bc[f] == ISM_VEL_INFLOW && f != 0) return ISM_ERR_ARG;
        if (vel_bc[f] == ISM_VEL_OUTFLOW && f != 1) return ISM_ERR_ARG;
        // pressure: Dirichlet-0 exactly on outflow faces, periodic exactly on
        // periodic faces (ism_setup pairs periodic faces), Neumann elsewhere
        if ((vel_bc[f] == ISM_VEL_OUTFLOW) != (ctx->bc[f] == ISM_BC_DIRICHLET0)) return ISM_ERR_ARG;
        if ((vel_bc[f] == ISM_VEL_PERIODIC) != (ctx->bc[f] == ISM_BC_PERIODIC)) return ISM_ERR_ARG;
        if (!isfinite(wall_u[f])) return ISM_ERR_ARG;
    }
    if (vel_bc[0] == ISM_VEL_INFLOW && !u_in) return ISM_ERR_ARG;
    if (vel_bc[1] == ISM_VEL_OUTFLOW && !(conv_u > 0.0)) return ISM_ERR_ARG;
    memcpy(ctx->vel_bc, vel_bc, sizeof(ctx->vel_bc));
    memcpy(ctx->wall_u, wall_u, sizeof(ctx->wall_u));
    ctx->u_in = u_in;
    ctx->conv_u = conv_u;
    ctx->flow_set = 1;
    return ISM_OK;
}

extern "C" ism_status ism_proj_tol(ism_ctx *ctx, double tol, int max_cycles, int warm_start)
{
    if (!ctx || !(tol > 0.0) || max_cycles < 0) return ISM_ERR_ARG;
    ctx->proj_tol = tol;
    ctx->proj_max_cycles = max_cycles;
    ctx->proj_warm = warm_start != 0;
    return ISM_OK;
}

extern "C" const double *ism_last_dp(const ism_ctx *ctx) { return ctx ? ctx->dp : nullptr; }

extern "C" const double *ism_last_b(const ism_ctx *ctx) { return ctx ? ctx->b64 : nullptr; }

ism_status ism_proj_buffers(ism_ctx *ctx);

extern "C" ism_status ism_set_warm_start(ism_ctx *ctx, const double *dp0)
{
    if (!ctx || !dp0) return ISM_ERR_ARG;
    TRY(ism_proj_buffers(ctx));
    TRY(ism_enter(ctx));
    ISM_CUDA_TRY(cudaMemcpyAsync(ctx->dp, dp0, (size_t)ctx->n * 8, cudaMemcpyDeviceToDevice, ctx->ws));
    return ism_leave(ctx);
}

ism_status ism_proj_buffers(ism_ctx *ctx)
{
    if (ctx->us) return ISM_OK;
    const size_t nx = ctx->nx, ny = ctx->ny;
    if (cudaMalloc((void **)&ctx->us, (nx + 1) * ny * sizeof(float)) != cudaSuccess ||
        cudaMalloc((void **)&ctx->vs, nx * (ny + 1) * sizeof(float)) != cudaSuccess ||
        cudaMalloc((void **)&ctx->dp, nx * ny * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return ISM_ERR_NOMEM;
    }
    if (cudaMemset(ctx->dp, 0, nx * ny * sizeof(double)) != cudaSuccess) return ISM_ERR_CUDA;
    return ISM_OK;
}

// defined in ism_core.cu
__global__ void k_ctl(IsmState *st, const double *partials, int nblk, int nq, int mode,
                      unsigned long long cond);
__global__ void k_rhs_stats(const double *__restrict__ x, double *__restrict__ y, long long n,
                            const IsmState *st, int mode, int sub_mean, double *partials);

extern "C" ism_status proj_step(ism_ctx *ctx, float *u, float *v, float *p, double dt, double nu)
{
    if (!ctx || !u || !v || !p || !(dt > 0.0) || !(nu >= 0.0) || !isfinite(dt) || !isfinite(nu))
        return ISM_ERR_ARG;
    if (!ctx->flow_set) return ISM_ERR_ARG;
    TRY(ism_proj_buffers(ctx));
    TRY(ism_enter(ctx));
    const int nx = ctx->nx, ny = ctx->ny;
    FlowArgs f;
    f.nx = nx; f.ny = ny;
    f.ih = (float)(1.0 / ctx->h);
    f.dt = (float)dt;
    f.nu = (float)nu;
    for (int k = 0; k < 4; ++k) { f.vbc[k] = ctx->vel_bc[k]; f.wall_u[k] = (float)ctx->wall_u[k]; }
    f.u_in = ctx->u_in;
    f.conv_u = (float)ctx->conv_u;
    const int T = 128;
    k_predict_u<<<dim3((nx + 1 + T - 1) / T, ny), T, 0, ctx->ws>>>(u, v, p, ctx->us, f);
    ISM_LAUNCH_CHECK(ctx);
    k_predict_v<<<dim3((nx + T - 1) / T, ny + 1), T, 0, ctx->ws>>>(u, v, p, ctx->vs, f);
    ISM_LAUNCH_CHECK(ctx);

    // right-hand side: reset the state, divergence -> b64, mean removal, ||b||
    IsmState h0;
    memset(&h0, 0, offsetof(IsmState, hist));
    h0.inv_n = 1.0 / (double)ctx->n;
    ISM_CUDA_TRY(cudaMemcpyAsync(ctx->st, &h0, offsetof(IsmState, hist), cudaMemcpyHostToDevice, ctx->ws));
    const dim3 dg((nx + 255) / 256, ny);
    k_divergence<<<dg, 256, 0, ctx->ws>>>(ctx->us, ctx->vs, ctx->b64, nx, ny, ctx->h / dt, ctx->partials);
    ISM_LAUNCH_CHECK(ctx);
    k_ctl<<<1, 256, 0, ctx->ws>>>(ctx->st, ctx->partials, dg.x * dg.y, 2, 0 /*CTL_RHS_MEAN*/, 0);
    ISM_LAUNCH_CHECK(ctx);
    k_rhs_stats<<<4 * 152, 256, 0, ctx->ws>>>(ctx->b64, ctx->b64, ctx->n, ctx->st, 1, ctx->singular, ctx->partials);
    ISM_LAUNCH_CHECK(ctx);
    k_ctl<<<1, 256, 0, ctx->ws>>>(ctx->st, ctx->partials, 4 * 152, 1, 1 /*CTL_RHS_NORM*/, 0);
    ISM_LAUNCH_CHECK(ctx);

    // initial guess: previous increment (warm start) or zero
    if (ctx->proj_warm)
        ISM_CUDA_TRY(cudaMemcpyAsync(ctx->p64[0], ctx->dp, (size_t)ctx->n * 8, cudaMemcpyDeviceToDevice, ctx->ws));
    else
        ISM_CUDA_TRY(cudaMemsetAsync(ctx->p64[0], 0, (size_t)ctx->n * 8, ctx->ws));
    ism_status s = ism_solve_internal(ctx, ctx->proj_tol, ctx->proj_max_cycles);
    if (s != ISM_OK && s != ISM_ERR_NOT_CONVERGED) {
        ism_leave(ctx);
        return s;
    }
    ISM_CUDA_TRY(cudaMemcpyAsync(ctx->dp, ctx->p64[0], (size_t)ctx->n * 8, cudaMemcpyDeviceToDevice, ctx->ws));
    const double sc = dt / ctx->h;
    k_correct_u<<<dim3((nx + 1 + T - 1) / T, ny), T, 0, ctx->ws>>>(u, ctx->us, ctx->dp, nx, ny, sc,
                                                                   ctx->vel_bc[1] == ISM_VEL_OUTFLOW,
                                                                   ctx->vel_bc[0] == ISM_VEL_PERIODIC);
    ISM_LAUNCH_CHECK(ctx);
    k_correct_v<<<dim3((nx + T - 1) / T, ny + 1), T, 0, ctx->ws>>>(v, ctx->vs, ctx->dp, p, nx, ny, sc,
                                                                   ctx->vel_bc[2] == ISM_VEL_PERIODIC);
    ISM_LAUNCH_CHECK(ctx);
    TRY(ism_leave(ctx));
    return s;
}
