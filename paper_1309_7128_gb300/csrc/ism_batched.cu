// ism_batched.cu -- many independent pressure solves advanced together.
//
// Every problem keeps its own context (grid, coarsening, boundary faces,
// workspaces, control block).  The solve runs as one CUDA graph: a prologue
// (right-hand-side preparation and the first FP64 residual of every problem)
// and a while node whose body advances every unfinished problem by one step:
//   1. problems whose single-precision solve has finished take the FP64
//      refinement update and its control (finished, or a new inner solve);
//   2. problems starting a new inner solve get e = 0 and the restriction of r;
//   3. problems in an inner solve run one cycle: coarse solve, nu / K fused
//      passes, per-problem control in the last CTA of that problem;
//   4. a one-thread kernel keeps the loop running while problems remain.
// Each launch covers the work items (tiles, coarse rows, cell chunks) of all
// problems; items of problems in another phase return at once.  The per-
// problem arithmetic is exactly that of ism_solve (same kernels' bodies).
#include <string.h>

#include <algorithm>
#include <vector>

#include "ism_kernels.cuh"
#include "ism_sweep32.cuh"

namespace {

constexpr int kChunk = 8192;     // cells per CTA in the per-cell kernels

struct BDom {
    IsmState *st;
    double *partials;
    const double *rhs;           // caller's right-hand side (per solve)
    double *puser;               // caller's iterate / result (per solve)
    double *b64, *p0, *p1;
    float *e0, *e1, *r32;
    float *rcpart, *ec, *Tm;
    const float *Qx, *QxT, *Qy, *QyT, *Minv;
    long long n;
    int nx, ny, m, ncx, ncy, bcmask, kind, singular;
    int nchunk;                  // per-cell kernels: CTAs of this problem
};

struct BState {
    int n;                       // problems
    int ndone;                   // problems finished
    int iter, max_iter;
    double tol;
    int max_cycles, max_outer, inner_max, npass;
    double inner_tol, floor_mult;
};

struct Plan {
    std::vector<unsigned long long> uids, gens;   // member contexts and their option generations
    int n = 0, nu = 0, K = 0;
    BDom *dom = nullptr;         // device, n
    BState *bst = nullptr;       // device
    int2 *chunks = nullptr;      // (problem, chunk)
    int nchunks = 0;
    int2 *crows = nullptr;       // (problem, coarse row)
    int ncrows = 0;
    // fused-pass tables and work lists: index 0 = init pass (K = 0, residual),
    // 1 = plain pass geometry, 2 = residual pass geometry
    std::vector<SweepArgs *> tab;   // per pass q (q < npass = nu / K)
    SweepArgs *tab_init = nullptr;  // the init pass (K = 0, residual)
    int engine = 0;                 // coarse solves: 0 CUDA cores, 1 single-CTA tensor-core kernel, 2 tiled chain
    void *ctc = nullptr;            // engine 1: per-problem arguments; engine 2: arguments and work list
    size_t ctc_smem = 0;
    size_t ctct_smem[4] = {};
    int ctct_nwork = 0;
    int4 *work_in[3] = {}, *work_ed[3] = {};
    int nwork_in[3] = {}, nwork_ed[3] = {};
    int maxncx = 1;
    cudaGraphExec_t gx = nullptr;
    long long launches_prologue = 0, launches_body = 0, launches_epilogue = 0;
    int *gather = nullptr;       // device: per problem (cycles, outer, status)
    double *gather_rel = nullptr;
};

}  // namespace

void ism_batch_free(void *p)
{
    Plan *P = (Plan *)p;
    if (!P) return;
    if (P->gx) cudaGraphExecDestroy(P->gx);
    void *bufs[] = {P->dom, P->bst, P->chunks, P->crows, P->gather, P->gather_rel};
    for (void *b : bufs)
        if (b) cudaFree(b);
    for (SweepArgs *t : P->tab)
        if (t) cudaFree(t);
    if (P->tab_init) cudaFree(P->tab_init);
    if (P->ctc) cudaFree(P->ctc);
    for (int i = 0; i < 3; ++i) {
        if (P->work_in[i]) cudaFree(P->work_in[i]);
        if (P->work_ed[i]) cudaFree(P->work_ed[i]);
    }
    delete P;
}

// ------------------------------------------------------------------ kernels

// Per-problem control block setup for one solve (one thread per problem).
__global__ void k_b_init_state(BDom *dom, const BState *bs)
{
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= bs->n) return;
    IsmState *st = dom[d].st;
    st->done = 0; st->status = 0; st->cycles = 0; st->outer = 0;
    st->inner_done = 0; st->inner_cycles = 0; st->cur = 0; st->zero_rhs = 0;
    st->max_cycles = bs->max_cycles; st->max_outer = bs->max_outer;
    st->inner_max = bs->inner_max; st->npass = bs->npass;
    st->tol = bs->tol; st->inner_tol = bs->inner_tol; st->floor_mult = bs->floor_mult;
    st->inv_n = 1.0 / (double)dom[d].n;
    st->bnorm = 0.0; st->relres = 0.0; st->mean = 0.0; st->mean_e = 0.0;
    st->r32norm = 0.0; st->rin = 0.0; st->enorm = 0.0;
    st->c64 = 0; st->skip_init = 1; st->ticket = 0;
}

__global__ void k_b_reset(BState *bs)
{
    bs->ndone = 0;
    bs->iter = 0;
}

// Last CTA of problem st (nblk CTAs): control decision; a problem that
// becomes finished is counted once in bs->ndone.
__device__ __forceinline__ void b_last_block(IsmState *st, const double *partials, int nblk, int nq,
                                             int mode, BState *bs)
{
    __shared__ int am_last;
    __shared__ double S[ISM_NQ];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) am_last = (atomicAdd(&st->ticket, 1u) == (unsigned)(nblk - 1));
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    ctl_reduce(partials, nblk, nq, S);
    if (threadIdx.x == 0) {
        const int was = st->done;
        ctl_decide(st, S, mode);
        st->ticket = 0;
        if (st->done && !was) atomicAdd(&bs->ndone, 1);
    }
}

// Right-hand side preparation per problem: mode 0: sum b (mean); mode 1:
// b64 = b - mean (all-Neumann), ||b64||^2; per-problem last-CTA control.
// Also copies the initial guess (mode 0).
__global__ void k_b_rhs(BDom *dom, const int2 *chunks, int mode, BState *bs)
{
    const int2 w = chunks[blockIdx.x];
    const BDom &D = dom[w.x];
    IsmState *st = D.st;
    const long long i0 = (long long)w.y * kChunk, i1 = min(D.n, i0 + kChunk);
    double s = 0.0;
    const double mu = (mode == 1 && D.singular) ? st->mean : 0.0;
    for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        double v = D.rhs[i];
        if (mode == 0) {
            s += v;
            D.p0[i] = D.puser[i];
        } else {
            v -= mu;
            D.b64[i] = v;
            s += v * v;
        }
    }
    double v1[1] = {s};
    block_partials<1>(v1, D.partials, D.nchunk, w.y);
    b_last_block(st, D.partials, D.nchunk, 1, mode == 0 ? CTL_RHS_MEAN : CTL_RHS_NORM, bs);
}

// FP64 refinement per problem (the arithmetic of the single-problem refinement, cells in chunks):
// UPDATE: only problems whose inner solve finished and which are not done.
template <bool UPDATE>
__global__ void k_b_refine(BDom *dom, const int2 *chunks, BState *bs)
{
    const int2 w = chunks[blockIdx.x];
    const BDom &D = dom[w.x];
    IsmState *st = D.st;
    if (UPDATE ? (!st->inner_done || st->done) : (st->done != 0)) return;
    const int nx = D.nx, ny = D.ny;
    const float *e = (UPDATE && st->cur) ? D.e1 : D.e0;
    const double *p_in = st->c64 ? D.p1 : D.p0;
    double *p_out = st->c64 ? D.p0 : D.p1;
    const long long i0 = (long long)w.y * kChunk, i1 = min(D.n, i0 + kChunk);
    double r2 = 0.0, ps = 0.0;
    for (long long idx = i0 + threadIdx.x; idx < i1; idx += blockDim.x) {
        const int j = (int)(idx / nx), i = (int)(idx - (long long)j * nx);
        auto P = [&](long long k) -> double {
            double v = p_in[k];
            if (UPDATE) v += (double)e[k];
            return v;
        };
        const double pc = P(idx);
        const double s = nb_sum<double>(P, idx, i, j, nx, ny, D.bcmask);
        const double r = D.b64[idx] - (s - (double)diag_count(i, j, nx, ny, D.bcmask) * pc);
        if (UPDATE) p_out[idx] = pc;
        D.r32[idx] = (float)r;
        r2 += r * r;
        ps += pc;
    }
    double v[2] = {r2, ps};
    block_partials<2>(v, D.partials, D.nchunk, w.y);
    b_last_block(st, D.partials, D.nchunk, 2, UPDATE ? CTL_OUTER_AFTER : CTL_OUTER_INIT, bs);
}

// Problems starting an inner solve: e = 0 and cleared partial block sums.
__global__ void k_b_zero(BDom *dom, const int2 *chunks)
{
    const int2 w = chunks[blockIdx.x];
    const BDom &D = dom[w.x];
    if (D.st->skip_init) return;
    const long long i0 = (long long)w.y * kChunk, i1 = min(D.n, i0 + kChunk);
    for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) D.e0[i] = 0.0f;
    if (w.y == 0)
        for (int i = threadIdx.x; i < 4 * D.ncx * D.ncy; i += blockDim.x) D.rcpart[i] = 0.0f;
}

// Coarse solve, one CTA per (problem, coarse row); problems not in an inner
// solve return.  Row 0 of coarse1 marks the first restriction as consumed.
__global__ void k_b_coarse1(BDom *dom, const int2 *rows)
{
    const int2 w = rows[blockIdx.x];
    const BDom &D = dom[w.x];
    if (D.st->inner_done) return;
    coarse1_row<float, true>(D.rcpart, D.QyT, D.Qx, D.Minv, D.Tm, D.ncx, D.ncy, w.y);
    if (w.y == 0 && threadIdx.x == 0) D.st->skip_init = 1;
}

__global__ void k_b_coarse2(BDom *dom, const int2 *rows)
{
    const int2 w = rows[blockIdx.x];
    const BDom &D = dom[w.x];
    if (D.st->inner_done) return;
    coarse2_row<float, true>(D.Tm, D.Qy, D.QxT, D.ec, D.ncx, D.ncy, D.rcpart, w.y);
}

// Loop condition: run while problems remain (with a hard iteration cap).
__global__ void k_b_cond(BState *bs, unsigned long long cond)
{
    const int it = ++bs->iter;
    const unsigned run = (bs->ndone < bs->n && it < bs->max_iter) ? 1u : 0u;
    cudaGraphSetConditional((cudaGraphConditionalHandle)cond, run);
}

// Result: p = final iterate - mean (zero for a vanishing right-hand side).
__global__ void k_b_finalize(BDom *dom, const int2 *chunks)
{
    const int2 w = chunks[blockIdx.x];
    const BDom &D = dom[w.x];
    const IsmState *st = D.st;
    const double *in = st->c64 ? D.p1 : D.p0;
    const double mu = D.singular ? st->mean : 0.0;
    const bool zero = st->zero_rhs != 0;
    const long long i0 = (long long)w.y * kChunk, i1 = min(D.n, i0 + kChunk);
    for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) D.puser[i] = zero ? 0.0 : in[i] - mu;
}

__global__ void k_b_gather(BDom *dom, const BState *bs, int *out, double *rel)
{
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= bs->n) return;
    const IsmState *st = dom[d].st;
    out[3 * d + 0] = st->cycles;
    out[3 * d + 1] = st->outer;
    out[3 * d + 2] = st->tc_fail ? ISM_ERR_CUDA : (st->done ? st->status : ISM_ERR_NOT_CONVERGED);
    rel[d] = st->relres;
}

// ------------------------------------------------------------------ host

#define TRY(x)                                                                   \
    do {                                                                         \
        ism_status _s = (x);                                                     \
        if (_s != ISM_OK) return _s;                                             \
    } while (0)

static ism_status cuda_ok(cudaError_t e)
{
    if (e == cudaSuccess) return ISM_OK;
    cudaGetLastError();
    return ISM_ERR_CUDA;
}

template <typename T>
static ism_status upload(T **dst, const std::vector<T> &v)
{
    if (v.empty()) { *dst = nullptr; return ISM_OK; }
    if (cudaMalloc((void **)dst, v.size() * sizeof(T)) != cudaSuccess) { cudaGetLastError(); return ISM_ERR_NOMEM; }
    return cuda_ok(cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
}

static SweepArgs pass_args(ism_ctx *c, int K, bool resid, int q, bool init)
{
    SweepArgs a;
    memset(&a, 0, sizeof(a));
    a.e0 = c->e32[0]; a.e1 = c->e32[1]; a.b = c->r32; a.E = c->ec32; a.rcpart = c->rcpart;
    a.partials = c->partials; a.st = c->st;
    a.skip = init ? &c->st->skip_init : &c->st->inner_done;
    a.curp = init ? nullptr : &c->st->cur;
    a.nx = c->nx; a.ny = c->ny; a.m = c->m; a.lm = c->m == 8 ? 3 : c->m == 16 ? 4 : 5;
    a.ncx = c->ncx; a.ncy = c->ncy; a.bcmask = c->bcmask; a.kind = c->opt.kind;
    a.K = K; a.q = q; a.use_mean = c->singular;
    a.ctl_mode = (!init && resid) ? CTL_INNER : -1;
    a.H = sweep_halo(K, resid); a.Hc = sweep_halo_cols(K, resid);
    a.TW = sweep_tile_w(K, resid); a.TH = sweep_tile_h(K, resid);
    a.gx = (c->nx + a.TW - 1) / a.TW;
    a.gy = (c->ny + a.TH - 1) / a.TH;
    a.cond = 0;
    return a;
}

// Work items of one pass geometry over all problems, split into tiles whose
// region lies strictly inside the domain and the others.
static void pass_work(const std::vector<ism_ctx *> &cs, int K, bool resid, std::vector<int4> &in,
                      std::vector<int4> &ed)
{
    for (size_t d = 0; d < cs.size(); ++d) {
        const ism_ctx *c = cs[d];
        const int tw = sweep_tile_w(K, resid), th = sweep_tile_h(K, resid);
        const int Hc = sweep_halo_cols(K, resid), H = sweep_halo(K, resid);
        const int gx = (c->nx + tw - 1) / tw, gy = (c->ny + th - 1) / th;
        for (int by = 0; by < gy; ++by)
            for (int bx = 0; bx < gx; ++bx) {
                const int x0 = bx * tw - Hc, y0 = by * th - H;
                const bool interior = x0 >= 1 && x0 + SRW <= c->nx - 1 && y0 >= 1 && y0 + SRH <= c->ny - 1;
                (interior ? in : ed).push_back(make_int4((int)d, bx, by, 0));
            }
    }
}

// Engine of the coarse solves: the tensor cores when every problem has
// coarse_tc set and a coarse grid they take -- the single-CTA kernel when all
// are <= 64 x 64 and none asks for the chain (coarse_tc 2), else the tiled
// split-TF32 chain -- and the CUDA cores otherwise.
static int batch_engine(const std::vector<ism_ctx *> &cs)
{
    bool small = true, chain = false;
    for (ism_ctx *c : cs) {
        if (!c->opt.coarse_tc || !ism_coarse_tc_supported(c)) return 0;
        small = small && ism_coarse_tc_small(c);
        chain = chain || c->opt.coarse_tc == 2;
    }
    return small && !chain ? 1 : 2;
}

static ism_status build_plan(Plan *P, const std::vector<ism_ctx *> &cs)
{
    ism_ctx *c0 = cs[0];
    P->n = (int)cs.size();
    P->nu = c0->opt.nu;
    P->K = c0->opt.sweeps_per_pass;
    std::vector<BDom> dom(P->n);
    std::vector<int2> chunks, crows;
    for (int d = 0; d < P->n; ++d) {
        ism_ctx *c = cs[d];
        BDom &D = dom[d];
        memset(&D, 0, sizeof(D));
        D.st = c->st; D.partials = c->partials;
        D.b64 = c->b64; D.p0 = c->p64[0]; D.p1 = c->p64[1];
        D.e0 = c->e32[0]; D.e1 = c->e32[1]; D.r32 = c->r32;
        D.rcpart = c->rcpart; D.ec = c->ec32; D.Tm = c->T32;
        D.Qx = c->Qx32; D.QxT = c->QxT32; D.Qy = c->Qy32; D.QyT = c->QyT32; D.Minv = c->Minv32;
        D.n = c->n; D.nx = c->nx; D.ny = c->ny; D.m = c->m; D.ncx = c->ncx; D.ncy = c->ncy;
        D.bcmask = c->bcmask; D.kind = c->opt.kind; D.singular = c->singular;
        D.nchunk = (int)((c->n + kChunk - 1) / kChunk);
        for (int k = 0; k < D.nchunk; ++k) chunks.push_back(make_int2(d, k));
        for (int l = 0; l < c->ncy; ++l) crows.push_back(make_int2(d, l));
        P->maxncx = std::max(P->maxncx, c->ncx);
        P->uids.push_back(c->uid);
        P->gens.push_back(c->opt_gen);
    }
    P->nchunks = (int)chunks.size();
    P->ncrows = (int)crows.size();
    TRY(upload(&P->dom, dom));
    TRY(upload(&P->chunks, chunks));
    TRY(upload(&P->crows, crows));
    if (cudaMalloc((void **)&P->bst, sizeof(BState)) != cudaSuccess ||
        cudaMalloc((void **)&P->gather, 3 * P->n * sizeof(int)) != cudaSuccess ||
        cudaMalloc((void **)&P->gather_rel, P->n * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return ISM_ERR_NOMEM;
    }
    P->engine = batch_engine(cs);
    if (P->engine == 1) TRY(ism_coarse_tc_batch_table(cs.data(), P->n, &P->ctc, &P->ctc_smem));
    if (P->engine == 2) TRY(ism_coarse_tct_batch_table(cs.data(), P->n, &P->ctc, &P->ctct_nwork, P->ctct_smem));
    const int npass = P->nu / P->K;
    P->tab.assign(npass, nullptr);
    for (int q = 0; q < npass; ++q) {
        std::vector<SweepArgs> t(P->n);
        for (int d = 0; d < P->n; ++d) t[d] = pass_args(cs[d], P->K, q == npass - 1, q, false);
        TRY(upload(&P->tab[q], t));
    }
    {
        std::vector<SweepArgs> t(P->n);
        for (int d = 0; d < P->n; ++d) t[d] = pass_args(cs[d], 0, true, 0, true);
        TRY(upload(&P->tab_init, t));
    }
    const int geomK[3] = {0, P->K, P->K};
    const bool geomR[3] = {true, false, true};
    for (int g = 0; g < 3; ++g) {
        std::vector<int4> in, ed;
        pass_work(cs, geomK[g], geomR[g], in, ed);
        P->nwork_in[g] = (int)in.size();
        P->nwork_ed[g] = (int)ed.size();
        TRY(upload(&P->work_in[g], in));
        TRY(upload(&P->work_ed[g], ed));
    }
    return ISM_OK;
}

template <bool PR, bool RE>
static ism_status launch_pass(ism_ctx *c0, const SweepArgs *tab, const int4 *win, int nin,
                              const int4 *wed, int ned, long long &count)
{
    const size_t sm = sweep_smem_bytes();
    const bool both = nin > 0 && ned > 0;
    if (both) {
        TRY(cuda_ok(cudaEventRecord(c0->ev_fork, c0->ws)));
        TRY(cuda_ok(cudaStreamWaitEvent(c0->ws2, c0->ev_fork, 0)));
        k_sweep32_batch<PR, RE, true><<<ned, STHREADS, sm, c0->ws2>>>(tab, wed);
        k_sweep32_batch<PR, RE, false><<<nin, STHREADS, sm, c0->ws>>>(tab, win);
        TRY(cuda_ok(cudaEventRecord(c0->ev_join, c0->ws2)));
        TRY(cuda_ok(cudaStreamWaitEvent(c0->ws, c0->ev_join, 0)));
        count += 2;
    } else if (nin > 0) {
        k_sweep32_batch<PR, RE, false><<<nin, STHREADS, sm, c0->ws>>>(tab, win);
        count += 1;
    } else if (ned > 0) {
        k_sweep32_batch<PR, RE, true><<<ned, STHREADS, sm, c0->ws>>>(tab, wed);
        count += 1;
    }
    return cuda_ok(cudaGetLastError());
}

static ism_status capture(ism_ctx *c0, cudaGraph_t g, const cudaGraphNode_t *deps, size_t nd,
                          ism_status (*fn)(ism_ctx *, Plan *, unsigned long long, long long &), Plan *P,
                          unsigned long long cond, long long &count, cudaGraphNode_t *last)
{
    TRY(cuda_ok(cudaStreamBeginCaptureToGraph(c0->ws, g, deps, nullptr, nd, cudaStreamCaptureModeThreadLocal)));
    ism_status s = fn(c0, P, cond, count);
    if (s == ISM_OK && last) {
        cudaStreamCaptureStatus cs;
        const cudaGraphNode_t *d = nullptr;
        size_t n = 0;
        if (cudaStreamGetCaptureInfo(c0->ws, &cs, nullptr, nullptr, &d, nullptr, &n) != cudaSuccess || n != 1)
            s = ISM_ERR_CUDA;
        else
            *last = d[0];
    }
    cudaGraph_t out = nullptr;
    const cudaError_t e = cudaStreamEndCapture(c0->ws, &out);
    if (s != ISM_OK) return s;
    return cuda_ok(e);
}

static ism_status prologue(ism_ctx *c0, Plan *P, unsigned long long, long long &count)
{
    k_b_reset<<<1, 1, 0, c0->ws>>>(P->bst);
    k_b_init_state<<<(P->n + 127) / 128, 128, 0, c0->ws>>>(P->dom, P->bst);
    k_b_rhs<<<P->nchunks, 256, 0, c0->ws>>>(P->dom, P->chunks, 0, P->bst);
    k_b_rhs<<<P->nchunks, 256, 0, c0->ws>>>(P->dom, P->chunks, 1, P->bst);
    k_b_refine<false><<<P->nchunks, 256, 0, c0->ws>>>(P->dom, P->chunks, P->bst);
    count += 5;
    return cuda_ok(cudaGetLastError());
}

static ism_status body(ism_ctx *c0, Plan *P, unsigned long long cond, long long &count)
{
    const int npass = P->nu / P->K;
    const size_t csm = (size_t)(256 + 2 * P->maxncx) * sizeof(float);
    k_b_refine<true><<<P->nchunks, 256, 0, c0->ws>>>(P->dom, P->chunks, P->bst);
    k_b_zero<<<P->nchunks, 256, 0, c0->ws>>>(P->dom, P->chunks);
    count += 2;
    TRY((launch_pass<false, true>(c0, P->tab_init, P->work_in[0], P->nwork_in[0], P->work_ed[0],
                                  P->nwork_ed[0], count)));
    if (P->engine == 1) {
        TRY(ism_launch_coarse_tc_batch(c0->ws, P->ctc, P->n, P->ctc_smem));
        count -= 1;
    } else if (P->engine == 2) {
        TRY(ism_launch_coarse_tct_batch(c0->ws, P->ctc, P->n, P->ctct_nwork, P->ctct_smem));
        count += 2;
    } else {
        k_b_coarse1<<<P->ncrows, 256, csm, c0->ws>>>(P->dom, P->crows);
        k_b_coarse2<<<P->ncrows, 256, csm, c0->ws>>>(P->dom, P->crows);
    }
    count += 2;
    for (int q = 0; q < npass; ++q) {
        const int g = q == npass - 1 ? 2 : 1;
        ism_status s;
        if (q == 0 && npass == 1)
            s = launch_pass<true, true>(c0, P->tab[q], P->work_in[g], P->nwork_in[g], P->work_ed[g], P->nwork_ed[g], count);
        else if (q == 0)
            s = launch_pass<true, false>(c0, P->tab[q], P->work_in[g], P->nwork_in[g], P->work_ed[g], P->nwork_ed[g], count);
        else if (q == npass - 1)
            s = launch_pass<false, true>(c0, P->tab[q], P->work_in[g], P->nwork_in[g], P->work_ed[g], P->nwork_ed[g], count);
        else
            s = launch_pass<false, false>(c0, P->tab[q], P->work_in[g], P->nwork_in[g], P->work_ed[g], P->nwork_ed[g], count);
        if (s != ISM_OK) return s;
    }
    k_b_cond<<<1, 1, 0, c0->ws>>>(P->bst, cond);
    count += 1;
    return cuda_ok(cudaGetLastError());
}

static ism_status epilogue(ism_ctx *c0, Plan *P, unsigned long long, long long &count)
{
    k_b_finalize<<<P->nchunks, 256, 0, c0->ws>>>(P->dom, P->chunks);
    k_b_gather<<<(P->n + 127) / 128, 128, 0, c0->ws>>>(P->dom, P->bst, P->gather, P->gather_rel);
    count += 2;
    return cuda_ok(cudaGetLastError());
}

static ism_status build_graph(ism_ctx *c0, Plan *P)
{
    cudaGraph_t g;
    TRY(cuda_ok(cudaGraphCreate(&g, 0)));
    ism_status s = ISM_OK;
    cudaGraphNode_t lastA, nloop;
    cudaGraphConditionalHandle h;
    s = capture(c0, g, nullptr, 0, prologue, P, 0, P->launches_prologue, &lastA);
    if (s == ISM_OK) s = cuda_ok(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
    cudaGraph_t bodyg = nullptr;
    if (s == ISM_OK) {
        cudaGraphNodeParams p = {};
        p.type = cudaGraphNodeTypeConditional;
        p.conditional.handle = h;
        p.conditional.type = cudaGraphCondTypeWhile;
        p.conditional.size = 1;
        s = cuda_ok(cudaGraphAddNode(&nloop, g, &lastA, nullptr, 1, &p));
        bodyg = p.conditional.phGraph_out[0];
    }
    if (s == ISM_OK) s = capture(c0, bodyg, nullptr, 0, body, P, (unsigned long long)h, P->launches_body, nullptr);
    if (s == ISM_OK) s = capture(c0, g, &nloop, 1, epilogue, P, 0, P->launches_epilogue, nullptr);
    if (s == ISM_OK) s = cuda_ok(cudaGraphInstantiate(&P->gx, g, 0));
    cudaGraphDestroy(g);
    return s;
}

static bool plan_matches(const Plan *P, const std::vector<ism_ctx *> &cs)
{
    if (!P || (int)cs.size() != P->n || cs[0]->opt.nu != P->nu || cs[0]->opt.sweeps_per_pass != P->K) return false;
    if (P->engine != batch_engine(cs)) return false;
    for (size_t d = 0; d < cs.size(); ++d)
        if (cs[d]->uid != P->uids[d] || cs[d]->opt_gen != P->gens[d]) return false;
    return true;
}

extern "C" ism_status ism_solve_batched(int n, ism_ctx *const *ctxs, const double *const *rhs,
                                        double *const *p, double tol, int max_cycles,
                                        int *cycles_out, double *relres_out)
{
    if (n < 0 || (n > 0 && (!ctxs || !rhs || !p)) || !(tol > 0.0) || max_cycles < 1) return ISM_ERR_ARG;
    if (n == 0) return ISM_OK;
    std::vector<ism_ctx *> cs(ctxs, ctxs + n);
    for (int d = 0; d < n; ++d) {
        if (!cs[d] || !rhs[d] || !p[d]) return ISM_ERR_ARG;
        if (cs[d]->prec != ISM_MIXED) return ISM_ERR_ARG;
        if (cs[d]->opt.nu != cs[0]->opt.nu || cs[d]->opt.sweeps_per_pass != cs[0]->opt.sweeps_per_pass ||
            cs[d]->opt.max_outer != cs[0]->opt.max_outer || cs[d]->opt.inner_max != cs[0]->opt.inner_max)
            return ISM_ERR_ARG;
        for (int e = 0; e < d; ++e)
            if (cs[e] == cs[d]) return ISM_ERR_ARG;
    }
    ism_ctx *c0 = cs[0];
    static bool attrs = false;
    if (!attrs) {
        const int smb = (int)sweep_smem_bytes();
        cudaFuncSetAttribute(k_sweep32_batch<true, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smb);
        cudaFuncSetAttribute(k_sweep32_batch<true, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smb);
        cudaFuncSetAttribute(k_sweep32_batch<false, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smb);
        cudaFuncSetAttribute(k_sweep32_batch<false, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smb);
        cudaFuncSetAttribute(k_sweep32_batch<true, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smb);
        cudaFuncSetAttribute(k_sweep32_batch<true, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smb);
        cudaFuncSetAttribute(k_sweep32_batch<false, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smb);
        cudaFuncSetAttribute(k_sweep32_batch<false, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smb);
        attrs = true;
    }
    Plan *P = (Plan *)c0->batch;
    if (!plan_matches(P, cs)) {
        if (P) ism_batch_free(P);
        c0->batch = nullptr;
        P = new Plan();
        ism_status s = build_plan(P, cs);
        if (s == ISM_OK) s = build_graph(c0, P);
        if (s != ISM_OK) {
            ism_batch_free(P);
            return s;
        }
        c0->batch = P;
    }
    // per-solve inputs: the callers' arrays and the tolerances
    std::vector<BDom> dom(n);
    TRY(cuda_ok(cudaMemcpy(dom.data(), P->dom, n * sizeof(BDom), cudaMemcpyDeviceToHost)));
    for (int d = 0; d < n; ++d) {
        dom[d].rhs = rhs[d];
        dom[d].puser = p[d];
    }
    BState bs;
    memset(&bs, 0, sizeof(bs));
    bs.n = n;
    bs.tol = tol;
    bs.max_cycles = max_cycles;
    bs.max_outer = c0->opt.max_outer;
    bs.inner_max = c0->opt.inner_max;
    bs.npass = P->nu / P->K;
    bs.inner_tol = c0->opt.inner_tol;
    bs.floor_mult = c0->opt.floor_mult;
    bs.max_iter = max_cycles + c0->opt.max_outer + 4;
    TRY(ism_enter(c0));
    TRY(cuda_ok(cudaMemcpyAsync(P->dom, dom.data(), n * sizeof(BDom), cudaMemcpyHostToDevice, c0->ws)));
    TRY(cuda_ok(cudaMemcpyAsync(P->bst, &bs, sizeof(bs), cudaMemcpyHostToDevice, c0->ws)));
    TRY(cuda_ok(cudaGraphLaunch(P->gx, c0->ws)));
    std::vector<int> g(3 * n);
    std::vector<double> rel(n);
    BState bs_out;
    TRY(cuda_ok(cudaMemcpyAsync(g.data(), P->gather, 3 * n * sizeof(int), cudaMemcpyDeviceToHost, c0->ws)));
    TRY(cuda_ok(cudaMemcpyAsync(rel.data(), P->gather_rel, n * sizeof(double), cudaMemcpyDeviceToHost, c0->ws)));
    TRY(cuda_ok(cudaMemcpyAsync(&bs_out, P->bst, sizeof(bs_out), cudaMemcpyDeviceToHost, c0->ws)));
    TRY(ism_leave(c0));
    TRY(cuda_ok(cudaStreamSynchronize(c0->ws)));
    c0->launches += P->launches_prologue + P->launches_epilogue + (long long)bs_out.iter * P->launches_body;
    ism_status first = ISM_OK;
    for (int d = 0; d < n; ++d) {
        if (cycles_out) cycles_out[d] = g[3 * d];
        if (relres_out) relres_out[d] = rel[d];
        cs[d]->last_cycles = g[3 * d];
        cs[d]->last_outer = g[3 * d + 1];
        cs[d]->last_status = g[3 * d + 2];
        cs[d]->last_relres = rel[d];
        cs[d]->last_nhist = std::min(ISM_HMAX, g[3 * d + 1] + 1);
        if (g[3 * d + 2] != ISM_OK && first == ISM_OK) first = (ism_status)g[3 * d + 2];
    }
    return first;
}
