/*
 * ism.h -- C ABI of the GB300 interpolated stencil multigrid (ISM) library.
 *
 * Method: Tegze & Toth, "A GPU cluster optimized multigrid scheme for
 * computing unsteady incompressible fluid flow".  The library solves the
 * cell-centred pressure Poisson equation of a projection time step (Sec. 2.2,
 * Eq. 4) with a two-level multigrid: red-black Gauss-Seidel smoothing on the
 * fine grid (Sec. 3.1), aggregating restriction over m x m blocks with
 * m = 16 or 32 (Sec. 3.2-3.4, Fig. 2b), an exact solve on the interpolated
 * nine-point coarse stencil (Sec. 3.3, Eq. 5-7) and bilinear prolongation
 * with correction (Eq. 5).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Fields are row-major: cell (i, j), i along x (fastest), j along y, at
 * element j*nx + i.  Face order for boundary arrays is west, east, south,
 * north.  The fine operator is the finite-volume five-point flux sum
 *     (A_f p)_c = sum over faces (p_neighbour - p_c),
 * where a Neumann face contributes 0 and a Dirichlet-0 face -2 p_c; the
 * equation solved is A_f p = b ("flux units": b is h^2 times the usual
 * Laplacian right-hand side).
 *
 * Pointers: arrays documented "device" are CUDA device pointers (or managed
 * memory) owned by the caller; the library never frees them.  Arrays
 * documented "host" are ordinary host memory.  The library owns all of its
 * workspaces; they live until ism_destroy.
 *
 * Streams: every call is ordered on the stream given to ism_setup.  Calls
 * that return numbers on the host (cycles, residuals) synchronise that
 * stream before returning.  A context must not be used from two host threads
 * at once.
 *
 * Errors: every entry point returns an ism_status.  ISM_ERR_ARG leaves all
 * caller arrays untouched.  ISM_ERR_NOT_CONVERGED leaves the last iterate in
 * the output array and the reached residual in the *_out arguments.  No entry
 * point aborts the process or traps on the device; device-side limits
 * (iteration caps) end in a status code.
 */
#ifndef ISM_H
#define ISM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ISM_OK = 0,
    ISM_ERR_ARG = 1,            /* invalid argument; nothing was written */
    ISM_ERR_NOT_CONVERGED = 2,  /* cycle or refinement cap reached before tol */
    ISM_ERR_NONFINITE = 3,      /* NaN or Inf met in the right-hand side or iterate */
    ISM_ERR_CUDA = 4,           /* a CUDA runtime call failed */
    ISM_ERR_NOMEM = 5           /* device or host allocation failed */
} ism_status;

/* Pressure face types.  ISM_BC_PERIODIC is given on both faces of an axis
 * (west and east, or south and north): the neighbour across the face is the
 * cell at the other end of the row / column, and the bilinear correction
 * interpolates across it between the last and the first coarse centre.  The
 * paper's cases have walls only; periodic axes extend the same operators. */
typedef enum { ISM_BC_NEUMANN = 0, ISM_BC_DIRICHLET0 = 1, ISM_BC_PERIODIC = 2 } ism_bc;

typedef enum {
    ISM_FP64 = 0,   /* every step in IEEE double */
    ISM_MIXED = 1   /* FP64 iterative refinement around single-precision cycles */
} ism_precision;

typedef enum {
    ISM_COARSE_ISM = 0,   /* interpolated nine-point coarse stencil, bilinear correction (Sec. 3.3) */
    ISM_COARSE_ACM = 1,   /* summed five-point coarse equations, constant correction (Sec. 3.2) */
    ISM_COARSE_GMG = 2,   /* five-point operator re-discretised on the coarse grid, bilinear
                             correction (the comparator of Sec. 4.3.2) */
    ISM_COARSE_ACMV = 3   /* additive correction as a deep V-cycle (Sec. 3.2, the paper's ACM
                             comparator): 2 x 2 agglomeration levels down to the coarsening factor,
                             piecewise-constant corrections, one red-black sweep per intermediate
                             level, exact solve at the coarsest; FP64 contexts only */
} ism_coarse_kind;

/* Velocity boundary kinds of the projection step, per face. */
typedef enum {
    ISM_VEL_NOSLIP = 0,    /* wall; tangential velocity wall_u[face] */
    ISM_VEL_FREESLIP = 1,  /* wall; zero tangential stress */
    ISM_VEL_INFLOW = 2,    /* west face only: u = inflow profile */
    ISM_VEL_OUTFLOW = 3,   /* east face only: convective outflow, pressure Dirichlet 0 */
    ISM_VEL_PERIODIC = 4   /* both faces of an axis (the pressure faces periodic too): the
                              neighbour across the face is at the other end; the last face of
                              the axis (u[., nx] or v[ny, .]) is the first face again and the
                              step keeps the two equal */
} ism_vel_bc;

/* Solver options (ism_get_options fills the defaults). */
typedef struct {
    int nu;               /* post-smoothing red-black sweeps per cycle (default 8 FP64, 64 mixed) */
    int sweeps_per_pass;  /* single precision: sweeps fused into one pass over memory (1..8,
                             nu % it == 0; default 4 FP64 (unused), 8 mixed) */
    int kind;             /* ism_coarse_kind (default ISM_COARSE_ISM) */
    int max_outer;        /* mixed: refinement iterations cap (default 50) */
    int inner_max;        /* mixed: single-precision cycles per refinement iteration cap (default 10000) */
    double inner_tol;     /* mixed: inner stop when ||r_in|| <= inner_tol ||r|| ... (default 1e-3) */
    double floor_mult;    /* ... or ||r_in|| <= floor_mult 2^-23 ||e|| (rounding floor, default 4) */
    int check_every;      /* use_graphs 0/1: cycles launched between host reads of the flags (default 16) */
    int use_graphs;       /* 0: plain launches; 1: CUDA graphs of check_every cycles; 2 (default):
                             the whole solve as one graph with device-side while loops */
    int coarse_tc;        /* mixed: 1 (default) runs the single-precision coarse solve on the tensor
                             cores (tcgen05, FP32 accumulation) when ncx, ncy <= 256: up to 64 x 64
                             one CTA runs the whole product chain with TF32 operands, above that
                             four launches of a tiled GEMM (128 x 32 blocks) do, in split TF32
                             (operands as hi + lo TF32 parts, about FP32 accuracy); 2 takes the
                             tiled launches on every coarse grid up to 256 x 256; 0 runs it on the
                             CUDA cores in FP32, as do 1 and 2 above 256.  The batched ensemble
                             picks its engine from the same setting (see ism_solve_batched).
                             Ignored by the FP64 path. */
    int cycle;            /* 0 (default): the correction-scheme cycle above.  1: the paper's
                             accommodative strategy (Sec. 4.3.1), FP64 contexts with the ISM coarse
                             operator only: Gauss-Seidel on the coarse equations until max |r_c| <=
                             accom_tol_c, bilinear correction, red-black sweeps on the fine grid until
                             max |r| <= tol (ism_solve's tol is then an absolute maximum norm and
                             max_cycles caps the fine sweeps).  A periodic axis then needs an even
                             number of coarse cells; a grid that is not a multiple of coarsen takes
                             it with walls only (its coarse coefficients are those of
                             A_c = W_y x T_x + T_y x W_x, see ism_setup). */
    double accom_tol_c;   /* cycle 1: coarse criterion (absolute maximum norm, default 1e-5) */
    int accom_max_coarse; /* cycle 1: cap on coarse Gauss-Seidel iterations (default 100000) */
    int stream;           /* single precision: 1 runs the passes that carry neither the correction
                             nor the residual (the middle passes of a cycle, ism_smooth) through the
                             streaming pass (one warp per 128-column strip marching down the rows,
                             the sweeps pipelined as a wavefront) when sweeps_per_pass is 1, 2 or 4;
                             0 (default): register-tiled passes only.  For grids larger than L2. */
    int fault_test;       /* failure-detection test only; 0 (default) in normal use.  1: every
                             tensor-core coarse solve (coarse_tc) first waits for an mbarrier phase
                             that nothing completes, under the same time limit as its real waits
                             (about 0.2 s); the wait runs out, the kernel records the failure, lets
                             its bulk copies finish, frees its tensor memory and returns, and the
                             solve stops with ISM_ERR_CUDA.  The CUDA context stays usable. */
    int tile_rows;        /* single precision: height of the register-tiled region of the fused pass,
                             128 (default: 8 warps, two CTAs per SM) or 256 (16 warps, one CTA per
                             SM; less halo overlap, 1.52x instead of 1.78x the cells at 8 sweeps);
                             ism_autotune tries both.  The batched solve uses 128. */
    int packed;           /* single precision: 1 updates the two same-colour cells of a row of the
                             fused pass's interior tiles with packed FP32 pair instructions (fewer
                             instructions, longer latency; results bit-identical); 0 with scalar
                             ones; 2 (default) packed when a pass runs at least four waves of
                             resident CTAs.  ism_autotune tries 0 and 1.  The batched solve uses
                             scalar updates. */
} ism_options;

typedef struct ism_ctx ism_ctx;

/* Human-readable name of a status code (static string). */
const char *ism_status_str(ism_status s);

/* ism_setup -- validate the problem and build the coarse level.
 * Sec. 3.3-3.4 and Sec. 4 (problem statement: grid, boundary conditions,
 * tile/coarsening size).
 *   nx, ny   fine cells, each >= `coarsen`, nx*ny <= 2^31.  When coarsen
 *            does not divide nx (ny), the last coarse column (row) is
 *            narrower (Sec. 3.3: padding, interpolation rectangles of
 *            different sizes; the coarse centre sits at the middle of its
 *            cell); such grids take the ISM and ACM coarse operators, the
 *            correction-scheme cycle and, with walls only, the accommodative
 *            cycle 1 (ism_set_options rejects GMG and the deep ACM V-cycle
 *            there) and ISM_MIXED needs nx % 4 == 0.
 *   h        cell size (used by proj_step only; > 0).
 *   bc       host, 4 ints (ism_bc) for the west, east, south, north faces;
 *            ISM_BC_PERIODIC on both faces of an axis or on neither, and
 *            then that axis a multiple of coarsen with at least 4 coarse
 *            cells.  A_f is singular
 *            (constants) when no face is Dirichlet-0: the solve then works
 *            on the mean-free subspace.
 *   coarsen  m in {8, 16, 32}: coarse cells are m x m blocks of fine cells;
 *            0: the library picks 16 or 32 (those dividing nx and ny with at
 *            least 2 coarse cells per direction) by timing two solves of an
 *            internal test right-hand side to 1e-8 with each (synchronises;
 *            about four solves of setup time).  ism_coarsening reports m.
 *   prec     ism_precision.
 *   stream   cudaStream_t to order all work on (NULL = legacy default stream).
 *   out      host; receives the new context.
 * Builds the coarse operator A_c = R A_f P in FP64 on the host (closed form
 * of the face-flux sums of Eq. 6-7), its separable eigenbases (with a
 * narrower last coarse cell: A_c = W_y x T_x + T_y x W_x and the 1-D pencils
 * T V = W V diag(lam), computed and checked numerically; ISM_ERR_ARG if a
 * check fails), and allocates all workspaces.  Returns ISM_ERR_ARG, ISM_ERR_NOMEM or ISM_ERR_CUDA on
 * failure (*out untouched). */
ism_status ism_setup(int nx, int ny, double h, const int bc[4], int coarsen,
                     ism_precision prec, void *stream, ism_ctx **out);

void ism_destroy(ism_ctx *ctx);

ism_status ism_get_options(const ism_ctx *ctx, ism_options *opt);
/* Replace the options; invalid values -> ISM_ERR_ARG (nothing changed). */
ism_status ism_set_options(ism_ctx *ctx, const ism_options *opt);

/* ism_solve -- solve A_f p = rhs to ||rhs - A_f p||_2 <= tol ||rhs||_2.
 * Sec. 3.4 (two-level sparse V cycle) with the cycle of Sec. 4.3.1
 * restated as: r = b - A_f p, r_c = R r (block sums), e_c = A_c^+ r_c
 * (exact), p += P e_c, nu red-black sweeps.
 *   rhs         device, nx*ny doubles (read only).  With all faces Neumann
 *               its mean is removed before solving (compatibility).
 *   p           device, nx*ny doubles; in: initial guess, out: solution
 *               (mean 0 when all faces are Neumann).
 *   tol         relative L2 residual target (> 0).
 *   max_cycles  cap on coarse corrections (FP64) or on single-precision
 *               cycles over all refinement iterations (mixed).
 *   cycles_out  host, may be NULL: cycles applied.
 *   relres_out  host, may be NULL: final relative residual (FP64 measure).
 * Synchronises the context's stream. */
ism_status ism_solve(ism_ctx *ctx, const double *rhs, double *p, double tol,
                     int max_cycles, int *cycles_out, double *relres_out);

/* ism_autotune -- choose the sweeps per cycle and per fused pass (and, for
 * ISM_MIXED, whether the middle passes stream, the refinement's inner
 * stopping factor inner_tol, the height of the fused pass's tiled region,
 * tile_rows, and the coarse engine, coarse_tc) for this context by timing
 * complete solves of rhs (device, nx*ny doubles) from a zero initial guess over a fixed
 * candidate list; keeps the fastest candidate in the context's options and
 * copies it to *best (host, may be NULL).  No counterpart in the paper (its
 * tile size and coarse tolerance were tuned by hand, Sec. 4.1, 4.3.1).
 * Allocates one nx*ny double buffer for the duration of the call.
 * Synchronises. */
ism_status ism_autotune(ism_ctx *ctx, const double *rhs, double tol, int max_cycles,
                        ism_options *best);

/* ism_autotune_from -- ism_autotune with every timed solve started from the
 * initial guess p0 (device, nx*ny doubles, not modified; NULL: zero, which is
 * ism_autotune).  A time stepper whose solves start from the previous step's
 * increment tunes on such a solve: a warm start needs fewer cycles, and the
 * fastest options differ from those of a cold one. */
ism_status ism_autotune_from(ism_ctx *ctx, const double *rhs, const double *p0, double tol,
                             int max_cycles, ism_options *best);

/* Coarsening factor m of a context (0 for NULL). */
int ism_coarsening(const ism_ctx *ctx);

/* Relative-residual history of the last solve: one entry per cycle (FP64)
 * or per refinement iteration (mixed), starting with the initial guess.
 * hist: host array of cap doubles; returns the number of entries written. */
int ism_last_history(const ism_ctx *ctx, double *hist, int cap);

/* Right-hand side of the last ism_solve or proj_step.  With every face
 * Neumann (or periodic) A_f is singular and A_f p = b is solvable only when
 * sum(b) = 0; the solve removes the mean of b first (the paper is silent on
 * this; its Neumann benchmarks have compatible data).  *mean_removed (host,
 * may be NULL): that mean, 0 when a face is Dirichlet-0.  *incompatible
 * (host, may be NULL): 1 when |sum(b)| > 1e-12 sum|b|, i.e. the removal
 * changed the problem beyond rounding, else 0.  Not set by the batched
 * solve. */
ism_status ism_last_rhs(const ism_ctx *ctx, double *mean_removed, int *incompatible);

/* Counters of the last solve (host, any may be NULL): refinement iterations
 * (mixed; 0 for FP64; coarse Gauss-Seidel iterations with cycle 1),
 * single-precision or FP64 cycles (fine sweeps with cycle 1), kernel launches. */
ism_status ism_last_counts(const ism_ctx *ctx, int *outer, int *cycles, long long *launches);

/* ---------------- kernel-level entry points (one step of the cycle) ------
 * Device arrays in the context's precision T (double for ISM_FP64, float
 * for ISM_MIXED); results are asynchronous on the context's stream. */

/* k red-black Gauss-Seidel sweeps in place on p (Sec. 3.1): red cells
 * ((i+j) even) first; p_c = (sum of in-domain neighbours - b_c) / d_c with
 * d_c = in-domain neighbours + 2 per Dirichlet-0 face. */
ism_status ism_smooth(ism_ctx *ctx, void *p, const void *b, int sweeps);

/* r_c = R (b - A_f p) (block sums over m x m, Sec. 3.2-3.3); rc: device,
 * ceil(ny/m)*ceil(nx/m) values of T.  norms: host, 2 doubles or NULL:
 * ||b - A_f p||_2 and sum(p). */
ism_status ism_residual_restrict(ism_ctx *ctx, const void *p, const void *b,
                                 void *rc, double *norms);

/* ism_residual_restrict_noalloc -- the FP64 residual and restriction of
 * ism_residual_restrict for callers that must not allocate device memory
 * when they need it: real-time loops that cannot take the implicit device
 * synchronisation of cudaMalloc/cudaFree, and hosts whose device memory is
 * handed out by their own arena and may not be allocated behind its back.
 * The paper has no counterpart; this is a library convenience.  It needs no
 * context and allocates nothing, on the device or the host: the per-block
 * partial sums live in a fixed 768 KiB array compiled into the library
 * (held by every GPU that loads it until the process exits).
 *   nx, ny, coarsen, bc  as for ism_setup (bc: host, 4 ints);
 *                        ceil(nx/coarsen)*ceil(ny/coarsen) must be <= 32768, else
 *                        ISM_ERR_ARG (nothing launched).
 *   p, b                 device, nx*ny doubles (read only).
 *   rc                   device, ceil(ny/m)*ceil(nx/m) doubles: block sums of b - A_f p.
 *   norms                device, 2 doubles: ||b - A_f p||_2 and sum(p).
 *   stream               cudaStream_t (NULL = legacy default stream); the
 *                        call is asynchronous on it.
 * The first call on each device (and the first after that device's context
 * was re-created, e.g. by cudaDeviceReset) looks up the array's device
 * address with cudaGetSymbolAddress; make that first call before any stream
 * capture.  Every call uses the same array, so calls whose kernels overlap
 * on the GPU (different streams without ordering) race and give wrong
 * results; calls on one stream, or otherwise ordered, are safe.  Each call
 * overwrites all the entries it reads, so nothing needs clearing between
 * calls. */
ism_status ism_residual_restrict_noalloc(int nx, int ny, int coarsen, const int bc[4],
                                         const double *p, const double *b, double *rc,
                                         double *norms, void *stream);

/* ism_residual_norms -- norms of the residual r = rhs - A_f p of an FP64
 * iterate, in FP64: *l2 = ||r||_2 (the solver's stopping quantity, relative
 * to ||rhs||_2 there) and *maxabs = max |r| (the paper's own criterion, an
 * absolute maximum norm, Sec. 4.3.1; a non-finite residual gives +inf).
 * Any context precision.  rhs, p: device, nx*ny doubles, row-major, read
 * only, used as given (an all-Neumann solve removes the mean of its
 * right-hand side first: pass the mean-free rhs to measure the equations it
 * solved).  l2, maxabs: host, either may be NULL, not both (ISM_ERR_ARG).
 * Ordered on the context's stream like ism_solve; synchronises. */
ism_status ism_residual_norms(ism_ctx *ctx, const double *rhs, const double *p, double *l2, double *maxabs);

/* e_c = A_c^+ r_c (exact coarse solve on the mean-free subspace when no
 * face is Dirichlet-0); rc, ec: device, ceil(ny/m)*ceil(nx/m) values of T. */
ism_status ism_coarse_solve(ism_ctx *ctx, const void *rc, void *ec);

/* p += P e_c (bilinear, Eq. 5, mirror ghost centres beyond a wall, the
 * periodic extension across a periodic face; constant per block for
 * ISM_COARSE_ACM). */
ism_status ism_prolong_add(ism_ctx *ctx, const void *ec, void *p);

/* Measurement helper: run `reps` smoothing passes of `sweeps` sweeps each
 * (as ism_smooth, one fused pass per call for ISM_MIXED; an odd reps is
 * rounded up to even there, so that the result ends in p) on p, b and return
 * in *us_per_pass the mean device time of one pass.  The passes are captured
 * into one CUDA graph on the library's work stream and replayed (once to
 * warm up, once timed between CUDA events on that stream), so consecutive
 * kernels run without host launch gaps, as inside a solve.  Synchronises.
 * No counterpart in the paper (Table 1 reports per-kernel wall times,
 * Sec. 4.1). */
ism_status ism_time_pass(ism_ctx *ctx, void *p, const void *b, int sweeps, int reps,
                         double *us_per_pass);

/* Measurement helper: run `reps` residual + restriction passes (those of
 * ism_residual_restrict, Sec. 3.2-3.3, norms left on the device) on p, b
 * into rc (device arrays as for ism_residual_restrict) and return in
 * *us_per_pass the mean device time of one pass, timed like ism_time_pass
 * (one captured graph of the passes, replayed between CUDA events on the
 * work stream).  Synchronises. */
ism_status ism_time_restrict(ism_ctx *ctx, const void *p, const void *b, void *rc, int reps,
                             double *us_per_pass);

/* Measurement helper: *us_per_solve the mean device time of one exact coarse
 * solve ec = A_c^+ rc (device arrays as in ism_coarse_solve, in the context's
 * precision; the engine the options select: the tensor-core kernels under
 * coarse_tc, else the CUDA cores), timed like ism_time_pass over `reps`
 * solves captured in one graph.  Synchronises. */
ism_status ism_time_coarse(ism_ctx *ctx, const void *rc, void *ec, int reps, double *us_per_solve);

/* ---------------- projection time step (Sec. 2.2-2.3, Eq. 3-4) ---------- */

/* Velocity boundary setup for proj_step.
 *   vel_bc  host, 4 ints (ism_vel_bc).  INFLOW only on the west face,
 *           OUTFLOW only on the east face; the pressure boundary given to
 *           ism_setup must be Dirichlet-0 exactly on OUTFLOW faces and
 *           periodic exactly on PERIODIC faces, else ISM_ERR_ARG.  (The paper's
 *           benchmarks have walls, inflow and outflow; Sec. 4.1 states that its
 *           kernels also take periodic faces.)  proj_step_adjoint, and
 *           proj_rollout_grad when it forms a gradient, reject periodic faces
 *           (ISM_ERR_ARG).
 *   wall_u  host, 4 doubles: tangential wall speed of NOSLIP faces.
 *   u_in    device, ny floats: west inflow profile (NULL if no inflow);
 *           read at every proj_step, so the caller may update it.
 *   conv_u  convective outflow speed (> 0 when an OUTFLOW face exists). */
ism_status ism_set_flow(ism_ctx *ctx, const int vel_bc[4], const double wall_u[4],
                        const float *u_in, double conv_u);

/* One Goda incremental pressure-correction step, in place:
 *   v* = v + dt [ -(v.grad) v + nu lap v - grad p ]  (forward Euler,
 *        second-order central differences on the MAC grid)
 *   A_f dp = h div(v*) / dt  solved by ism_solve to tol (see ism_proj_tol)
 *   v = v* - dt grad dp,  p = p + dp.
 *   u  device, ny*(nx+1) floats (x-faces);  v  device, (ny+1)*nx floats
 *   (y-faces);  p  device, nx*ny floats.  dt > 0, nu >= 0.
 * Returns the status of the pressure solve. */
ism_status proj_step(ism_ctx *ctx, float *u, float *v, float *p, double dt, double nu);

/* Pressure-solve controls used by proj_step (defaults tol 1e-8,
 * max_cycles 100000, warm start off). */
ism_status ism_proj_tol(ism_ctx *ctx, double tol, int max_cycles, int warm_start);

/* Last pressure increment dp of proj_step: device, nx*ny doubles owned by
 * the context (valid until the next call on it). */
const double *ism_last_dp(const ism_ctx *ctx);

/* Right-hand side of the context's last pressure solve as it was solved
 * (ism_solve, proj_step or an adjoint step: Eq. 4's h div(v*)/dt in flux
 * units for a projection step, its mean removed when every face is Neumann
 * or periodic): device, nx*ny doubles owned by the context, valid until the
 * next call on it.  With ism_last_dp it lets a caller check the equations a
 * step solved (e.g. the residual b - A_f dp). */
const double *ism_last_b(const ism_ctx *ctx);

/* Set the pressure increment that the next proj_step starts its solve from
 * when warm start is on (ism_proj_tol), as if it were the last increment:
 * dp0 device, nx*ny doubles, copied (asynchronously, on the context's
 * stream).  Restarts a run from a saved state (u, v, p and the last dp) with
 * the same solves as the uninterrupted run.  No counterpart in the paper. */
ism_status ism_set_warm_start(ism_ctx *ctx, const double *dp0);

/* ---------------- adjoint of the projection step ------------------------
 * No counterpart in the paper, which runs the step forwards only.  The
 * adjoint is the transpose of the linearisation of proj_step (Sec. 2.2-2.3,
 * Eq. 3-4) at the step's input state: transposed correction, the pressure
 * solve again (A_f is symmetric, so its adjoint is the same ISM solve, run
 * to the tolerance set by ism_proj_tol from a zero initial guess), transposed
 * divergence (= minus the gradient), transposed predictor.  The exact solve
 * is differentiated: the solver's own iterations are not. */

/* Given the input velocities (u, v) of one proj_step and the adjoints
 * (gu, gv, gp) of its outputs (u', v', p'), overwrite gu, gv, gp with the
 * adjoints of its inputs (u, v, p).  The step is linear in p, so p is not
 * needed.  Layouts as proj_step; all device, float.  Uses the flow setup of
 * ism_set_flow and the dt, nu given; the context's predicted-velocity
 * buffers are overwritten, its last increment (ism_last_dp) is not.
 * Returns the status of the adjoint pressure solve. */
ism_status proj_step_adjoint(ism_ctx *ctx, const float *u, const float *v, double dt,
                             double nu, float *gu, float *gv, float *gp);

/* Enstrophy of a MAC velocity field, E = 1/2 sum_nodes w^2 h^2 with the
 * vorticity w = dv/dx - du/dy at the interior grid nodes (boundary nodes
 * left out).  value: host, may be NULL; gu, gv: device (layouts as
 * proj_step), receive dE/du, dE/dv when not NULL.  Synchronises when value
 * is requested.  Not in the paper: the loss of the differentiable rollout. */
ism_status ism_enstrophy(ism_ctx *ctx, const float *u, const float *v, double *value,
                         float *gu, float *gv);

/* Differentiable rollout: `steps` proj_steps from (u0, v0, p0) (device,
 * not modified), loss = ism_enstrophy of the final velocity (host *loss, may
 * be NULL).  With gu, gv, gp all non-NULL (device) they receive the gradient
 * of the loss with respect to u0, v0, p0, by reverse sweeps with checkpoints
 * every `every` steps (>= 1): the forward keeps the state before every
 * every-th step, each segment is replayed from its checkpoint and then
 * traversed by proj_step_adjoint.  All three NULL: forward and loss only.
 * Device memory: (steps/every + 2) states of ~20 bytes per cell plus `every`
 * velocity pairs, owned by the context and kept for the next call.
 * Synchronises.  Returns ISM_OK, or the first non-OK solve status
 * (ISM_ERR_NOT_CONVERGED keeps going; other errors stop the call). */
ism_status proj_rollout_grad(ism_ctx *ctx, const float *u0, const float *v0, const float *p0,
                             double dt, double nu, int steps, int every, double *loss,
                             float *gu, float *gv, float *gp);

/* ---------------- batched ensemble ----------------------------------------
 * ism_solve_batched -- solve n independent problems, each described by its
 * own context, to ||rhs - A_f p|| <= tol ||rhs|| each (an ensemble of
 * uneven problems; the paper solves one problem at a time).  All contexts must be ISM_MIXED, on
 * the same device, with equal nu, sweeps_per_pass, max_outer and inner_max;
 * grids, coarsening and boundary faces may differ.  The solve is one CUDA
 * graph on ctxs[0]'s stream: every launch covers the work items of all
 * unfinished problems (a finished problem drops out), so one set of
 * launches advances every problem by one cycle; per problem the arithmetic
 * and the decisions are those of ism_solve.  The coarse solves run on the
 * tensor cores when every context has coarse_tc set and a coarse grid of at
 * most 256 x 256: one CTA per problem when every coarse grid is at most
 * 64 x 64 and no context asks for the chain (coarse_tc 2), else the tiled
 * split-TF32 chain, four launches over all problems' blocks; otherwise on the
 * CUDA cores.  The graph is
 * built on the first call with a given list of contexts and reused while the
 * list is unchanged and no member's options were set since.
 *   ctxs   host, n distinct contexts.  rhs, p: host arrays of n device pointers
 *          (as for ism_solve: p holds the initial guess and receives the result).
 *   max_cycles  cap on single-precision cycles per problem (>= 1).
 *   cycles_out, relres_out: host, n entries each, or NULL.
 * Returns ISM_OK if every problem converged, else the first failing status;
 * ISM_ERR_ARG (nothing launched) for invalid or mismatched contexts. */
ism_status ism_solve_batched(int n, ism_ctx *const *ctxs, const double *const *rhs,
                             double *const *p, double tol, int max_cycles,
                             int *cycles_out, double *relres_out);

/* ism_autotune_batched -- choose the sweeps per cycle of a batched ensemble
 * (nu in {16, 32, 64, 128}, 8 sweeps per fused pass, the same for every
 * problem as ism_solve_batched requires) and the engine of its coarse solves
 * (coarse_tc 0, 1 or 2), by timing ism_solve_batched on the given
 * right-hand sides; p: host array of n device iterates, overwritten
 * (zero initial guesses).  Sets the winner in every context (on failure the
 * options are restored) and returns it in *nu_out (host, may be NULL).  No
 * counterpart in the paper.  Synchronises. */
ism_status ism_autotune_batched(int n, ism_ctx *const *ctxs, const double *const *rhs,
                                double *const *p, double tol, int *nu_out);

#ifdef __cplusplus
}
#endif
#endif /* ISM_H */
