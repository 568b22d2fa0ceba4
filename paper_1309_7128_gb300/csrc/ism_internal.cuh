// ism_internal.cuh -- shared declarations of the ISM library (not installed).
//
// Layout of everything the library owns on the device, the control block
// that the kernels use to decide convergence without host round trips, and
// the launch helpers shared by the solver, the projection step and the
// batched ensemble.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/ism.h"

#define ISM_HMAX 4096          // residual-history entries kept on the device
#define ISM_NQ 4               // partial sums per CTA (q-major)

// Device control block.  Written by the one-CTA control kernels, read by
// every cycle kernel (which returns at once when its phase is finished).
struct IsmState {
    int done;          // FP64 path / outer refinement finished
    int status;        // ism_status of the finished solve
    int cycles;        // FP64: coarse corrections; mixed: single-precision cycles (all outer iterations)
    int outer;         // mixed: refinement iterations applied
    int inner_done;    // mixed: current inner solve finished
    int inner_cycles;  // mixed: cycles in the current inner solve
    int cur;           // mixed: which ping-pong buffer holds the inner iterate
    int zero_rhs;      // ||b|| == 0: the solution is p = 0
    int max_cycles, max_outer, inner_max, npass;
    double tol, inner_tol, floor_mult, inv_n;
    double bnorm;      // ||b - mean(b)||_2
    double relres;     // latest relative residual (FP64 measure)
    double mean;       // mean to subtract from the iterate (all-Neumann), FP64 path / outer p
    double mean_e;     // mixed: mean of the inner iterate
    double r32norm;    // mixed: ||r|| of the current inner right-hand side
    double rin, enorm; // mixed: latest inner residual and iterate norms
    double rhs_sum;    // sum of the right-hand side as given (before the mean is removed)
    double rhs_l1;     // its L1 norm (0 where the preparation does not form it: batched)
    int c64;           // mixed: which FP64 buffer holds the outer iterate
    int skip_init;     // batched: 0 while a new inner solve still needs its first restriction
    int tc_fail;       // a tensor-core coarse solve gave up waiting for its MMAs
    unsigned int ticket; // CTAs finished in the current fused-control kernel
    double hist[ISM_HMAX];
};

struct ism_ctx {
    int nx, ny, m, ncx, ncy;
    long long n;               // nx * ny
    double h;
    int bc[4];
    int bcmask;                // ism_bc_mask(bc)
    int singular;              // no Dirichlet-0 face (A_f 1 = 0)
    int ragged;                // m does not divide nx or ny: the last coarse cell is narrower
    int prec;
    ism_options opt;
    unsigned long long opt_gen;  // incremented by every ism_set_options (batched plans are keyed on it)
    cudaStream_t user_stream;  // ordering stream given by the caller
    cudaStream_t ws;           // private work stream (graph capture needs a non-legacy stream)
    cudaStream_t ws2;          // forked stream for concurrent launches within a step
    cudaEvent_t ev_in, ev_out, ev_fork, ev_join;

    // coarse level: separable eigenbases of A_c = (Qy x Qx) diag(mu) (Qy x Qx)^T
    double *Qx64, *QxT64, *Qy64, *QyT64, *Minv64;
    float *Qx32, *QxT32, *Qy32, *QyT32, *Minv32;

    // work buffers
    double *b64;               // right-hand side with the mean removed
    double *p64[2];            // FP64 iterate (ping-pong for the mixed refinement update)
    float *e32[2];             // mixed: single-precision inner iterate (ping-pong)
    float *r32;                // mixed: inner right-hand side
    double *rc64, *ec64, *T64; // coarse residual, correction, intermediate
    double *G64;               // FP64: coarse rows interpolated along x (ncy x nx), separable prolongation
    float *rc32, *ec32, *T32;
    float *rcpart;             // 4 partial block sums per coarse cell (fused restriction)
    double *lvl_r[6], *lvl_e[6];   // deep V-cycle (ISM_COARSE_ACMV): residual / correction of levels 1..L-1
    void *tc_block;            // tensor-core coarse solve: constant operand tiles (TF32), or NULL
    size_t tc_bytes;
    void *tct_block;           // tiled tensor-core coarse solve: chunked operand tiles and intermediates, or NULL
    size_t tct_bytes;
    double *partials;          // ISM_NQ * max_blocks
    int max_blocks;
    IsmState *st;              // device control block
    IsmState *st_k;            // device control block for kernel-level entry points
    double *ac_tri;            // cycle 1 on a grid not a multiple of m: W_x, T_x, W_y, T_y (3 per coarse row)
    IsmState *st_host;         // pinned host copy (selected fields are read back)

    // tile plans of the fused sweep pass, per (region height 128 | 256, sweeps K, residual fused)
    struct SweepPlan { int gx, gy, ix0, ix1, iy0, iy1, nedge; int2 *edge; } plans[2][9][2];

    // CUDA graphs of a chunk of cycles
    cudaGraphExec_t g_fp64, g_inner;       // chunks of cycles (use_graphs = 1)
    cudaGraphExec_t gc_fp64, gc_mixed;     // whole solve with device-side loops (use_graphs = 2)
    int g_fp64_len, g_inner_len;

    // last solve
    int last_cycles, last_outer, last_status, last_nhist;
    double last_rhs_sum, last_rhs_l1;   // right-hand side of the last ism_solve / proj_step
    double last_relres;
    long long launches;
    unsigned long long uid;    // unique per context (batched plan cache key)
    void *batch;               // cached batched-solve plan (ism_batched.cu), owned

    // projection step
    int vel_bc[4];
    double wall_u[4];
    const float *u_in;
    double conv_u;
    int flow_set;
    float *us, *vs;            // predicted velocities
    double *dp;                // pressure increment
    double proj_tol;
    int proj_max_cycles, proj_warm;

    // adjoint rollout (ism_adjoint.cu): checkpoints, segment states, adjoint state
    void *roll;                // one allocation, grown on demand
    size_t roll_bytes;
    double *scal;              // device scalars (loss)
};

// ------------------------------------------------------------------ helpers

#define ISM_CUDA_TRY(call)                                                    \
    do {                                                                      \
        cudaError_t _e = (call);                                              \
        if (_e != cudaSuccess) return ISM_ERR_CUDA;                           \
    } while (0)

#define ISM_LAUNCH_CHECK(ctx)                                                 \
    do {                                                                      \
        (ctx)->launches++;                                                    \
        if (cudaGetLastError() != cudaSuccess) return ISM_ERR_CUDA;           \
    } while (0)

// ism_setup for a given coarsening factor (8, 16, 32); ism_setup adds the
// autotuned choice (coarsen = 0, ism_tune.cu).
// Face mask of the kernels: bit f (W, E, S, N = 0..3) set when face f is
// Dirichlet-0; ISM_PER_X / ISM_PER_Y when the x / y axis is periodic (face
// type ISM_BC_PERIODIC on both of its faces).  -1 for an invalid bc.
constexpr int ISM_PER_X = 16, ISM_PER_Y = 32;
inline int ism_bc_mask(const int bc[4])
{
    int mask = 0;
    for (int f = 0; f < 4; ++f) {
        if (bc[f] != ISM_BC_NEUMANN && bc[f] != ISM_BC_DIRICHLET0 && bc[f] != ISM_BC_PERIODIC) return -1;
        if (bc[f] == ISM_BC_DIRICHLET0) mask |= 1 << f;
    }
    if ((bc[0] == ISM_BC_PERIODIC) != (bc[1] == ISM_BC_PERIODIC)) return -1;
    if ((bc[2] == ISM_BC_PERIODIC) != (bc[3] == ISM_BC_PERIODIC)) return -1;
    if (bc[0] == ISM_BC_PERIODIC) mask |= ISM_PER_X;
    if (bc[2] == ISM_BC_PERIODIC) mask |= ISM_PER_Y;
    return mask;
}

// 1-D factor of the coarse operator along one axis (ism_pencil.cu):
// T V = W V diag(lam), L = (W V)^-1, V and L row-major n x n, lam ascending.
struct IsmAxisFactor {
    std::vector<double> V, L, lam;
};
// The factor of an axis of n fine cells (the last coarse cell narrower when
// m does not divide n), computed numerically; lo, hi: ism_bc of its ends
// (not periodic); kind: ism_coarse_kind (ISM or ACM).  false when a
// numerical check fails.
bool ism_axis_factor(int n, int m, int lo, int hi, int kind, IsmAxisFactor &F);
// The tridiagonal W = R1 P1 and T = R1 T1 P1 of such an axis, row k as
// (A[k][k-1], A[k][k], A[k][k+1]) at 3k .. 3k+2 of W3, T3 (host, 3 nc each).
bool ism_axis_tridiag(int n, int m, int lo, int hi, int kind, double *W3, double *T3);

ism_status ism_setup_fixed(int nx, int ny, double h, const int bc[4], int coarsen, ism_precision prec,
                           void *stream, ism_ctx **out);

// Order ctx->ws after the caller's stream, and the caller's stream after ws.
ism_status ism_enter(ism_ctx *ctx);
ism_status ism_leave(ism_ctx *ctx);

// Solve on internal buffers: b64 holds the right-hand side (mean removed),
// p64[0] the initial guess; on return p64[0] holds the solution.
// record_rhs: keep the right-hand side's sums for ism_last_rhs (the caller's
// own solves, ism_solve and proj_step; not the adjoint's internal solve).
ism_status ism_solve_internal(ism_ctx *ctx, double tol, int max_cycles, bool record_rhs = true);
// The accommodative strategy (cycle = 1, ism_accom.cu) on the same buffers.
ism_status ism_solve_accommodative(ism_ctx *ctx, double tol, int max_sweeps);
// Copy user rhs into b64 (removing the mean when singular) and compute ||b||.
ism_status ism_prepare_rhs(ism_ctx *ctx, const double *rhs);

// Projection-step kernels (ism_proj.cu) need the residual solver above.
// Allocate the predicted-velocity and increment buffers on first use.
ism_status ism_proj_buffers(ism_ctx *ctx);

// Tensor-core coarse solve of the single-precision cycle (ism_coarse_tc.cu):
// rc -> ec (ncy x ncx); from_parts: rc holds 4 partial block sums per coarse
// cell; rcpart (or NULL) is cleared afterwards.
// ism_coarse_tc_supported: either kernel applies (coarse grids up to
// 256 x 256); ism_coarse_tc_small: the single-CTA kernel (up to 64 x 64),
// the only one of the batched ensemble.
bool ism_coarse_tc_supported(const ism_ctx *ctx);
bool ism_coarse_tc_small(const ism_ctx *ctx);
void ism_coarse_tc_prepare();   // kernel attributes (called by ism_setup, outside any capture)
// Lay out the constant operands of E = Qy [(QyT R Qx) . Minv] QxT as TF32
// tiles on the device.
ism_status ism_coarse_tc_upload(ism_ctx *ctx, const std::vector<double> &Qx, const std::vector<double> &QxT,
                                const std::vector<double> &Qy, const std::vector<double> &QyT,
                                const std::vector<double> &Minv);
ism_status ism_launch_coarse_tc(ism_ctx *ctx, const float *rc, bool from_parts, float *ec, float *rcpart,
                                const int *skip);
// The tiled chain of ism_coarse_tct.cu: four launches of a 128 x 32-block
// tcgen05 GEMM over chunked K-major TF32 tiles (coarse grids up to 256 x 256).
bool ism_coarse_tct_fits(int ncx, int ncy);
void ism_coarse_tct_prepare();
ism_status ism_coarse_tct_upload(ism_ctx *ctx, const std::vector<double> &Qx, const std::vector<double> &QxT,
                                 const std::vector<double> &Qy, const std::vector<double> &QyT);
ism_status ism_launch_coarse_tct(ism_ctx *ctx, const float *rc, bool from_parts, float *ec, float *rcpart,
                                 const int *skip);
// Batched ensemble: one device block (owned by the caller, cudaFree) holding
// the four products' per-problem arguments and the list of every problem's
// CTAs (*nwork entries), and the shared memory of each product's launch;
// problems outside an inner solve skip.
ism_status ism_coarse_tct_batch_table(ism_ctx *const *ctxs, int n, void **table, int *nwork, size_t smem[4]);
ism_status ism_launch_coarse_tct_batch(cudaStream_t s, const void *table, int n, int nwork, const size_t smem[4]);
// Batched ensemble: a device table of per-problem arguments (owned by the
// caller, cudaFree) and the shared memory the launch needs; one CTA per
// problem, problems outside an inner solve skip.
ism_status ism_coarse_tc_batch_table(ism_ctx *const *ctxs, int n, void **table, size_t *smem);
ism_status ism_launch_coarse_tc_batch(cudaStream_t s, const void *table, int n, size_t smem);
