// ism_kernels.cuh -- device kernels of the ISM solve (included by ism_core.cu
// and ism_batched.cu; everything here is internal).
//
// Fine-grid conventions: row-major (i fastest), face order W, E, S, N,
// bcmask bit f set when face f is Dirichlet-0, ISM_PER_X / ISM_PER_Y when an
// axis is periodic.  The five-point flux sum is
//   (A_f p)_c = sum_nb p_nb - d_c p_c,
//   d_c = (#neighbours) + 2 (#Dirichlet-0 faces of the cell),
// the cell at the other end of a periodic row / column counting as a
// neighbour, so the Gauss-Seidel point update is p_c = (sum_nb p_nb - b_c) / d_c.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ism_internal.cuh"

#define FULLMASK 0xffffffffu

// 1/d for d = 0..8 (d = 4 for interior cells, 2..8 on the boundary)
__constant__ double c_invd64[9] = {0.0, 1.0, 1.0 / 2, 1.0 / 3, 1.0 / 4,
                                   1.0 / 5, 1.0 / 6, 1.0 / 7, 1.0 / 8};
__constant__ float c_invd32[9] = {0.0f, 1.0f, 1.0f / 2, 1.0f / 3, 1.0f / 4,
                                  1.0f / 5, 1.0f / 6, 1.0f / 7, 1.0f / 8};

template <typename T> __device__ __forceinline__ T inv_diag(int d);
template <> __device__ __forceinline__ double inv_diag<double>(int d) { return c_invd64[d]; }
template <> __device__ __forceinline__ float inv_diag<float>(int d) { return c_invd32[d]; }

// d_c: each wall face of the cell removes its neighbour (-1) and, when
// Dirichlet-0, adds the ghost's 2 p_c (+2): net +1 (Dirichlet) or -1
// (Neumann); a periodic face keeps its (wrapped) neighbour.
__device__ __forceinline__ int diag_count(int x, int y, int nx, int ny, int bcmask)
{
    int d = 4;
    if (!(bcmask & ISM_PER_X)) {
        if (x == 0) d += (bcmask & 1) ? 1 : -1;
        if (x == nx - 1) d += (bcmask & 2) ? 1 : -1;
    }
    if (!(bcmask & ISM_PER_Y)) {
        if (y == 0) d += (bcmask & 4) ? 1 : -1;
        if (y == ny - 1) d += (bcmask & 8) ? 1 : -1;
    }
    return d;
}

// sum of the neighbour values of cell (x, y) at linear index idx, P(k) giving
// the value at index k: in-domain neighbours, and across a periodic face the
// cell at the other end of the row / column
template <typename T, typename F>
__device__ __forceinline__ T nb_sum(F P, long long idx, int x, int y, int nx, int ny, int bcmask)
{
    const long long wrap_y = (long long)(ny - 1) * nx;
    T s = (T)0;
    if (x > 0) s += P(idx - 1); else if (bcmask & ISM_PER_X) s += P(idx + (nx - 1));
    if (x < nx - 1) s += P(idx + 1); else if (bcmask & ISM_PER_X) s += P(idx - (nx - 1));
    if (y > 0) s += P(idx - nx); else if (bcmask & ISM_PER_Y) s += P(idx + wrap_y);
    if (y < ny - 1) s += P(idx + nx); else if (bcmask & ISM_PER_Y) s += P(idx - wrap_y);
    return s;
}

// v mod n in [0, n) for any int v
__device__ __forceinline__ int wrap_mod(int v, int n)
{
    const int r = v % n;
    return r < 0 ? r + n : r;
}

// ----------------------------------------------------------------- reductions

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULLMASK, v, o);
    return v;
}

// Deterministic block reduction of NQ doubles; thread 0 of the block writes
// partials[q * nblk + bid].  blockDim.x must be a multiple of 32, <= 1024.
template <int NQ>
__device__ __forceinline__ void block_partials(double (&v)[NQ], double *partials,
                                               int nblk, int bid)
{
    __shared__ double red[NQ][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q) v[q] = warp_sum(v[q]);
    __syncthreads();   // red[] may still be read by a previous call
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) red[q][w] = v[q];
    }
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            double t = lane < nw ? red[q][lane] : 0.0;
            t = warp_sum(t);
            if (lane == 0) partials[(size_t)q * nblk + bid] = t;
        }
    }
}

// ----------------------------------------------------------------- convergence control

enum CtlMode {
    CTL_RHS_MEAN = 0,   // S0 = sum b, S1 = sum |b|    -> st->mean, rhs_sum, rhs_l1
    CTL_RHS_NORM = 1,   // S0 = ||b - mean||^2          -> bnorm, zero_rhs, status
    CTL_FP64_INIT = 2,  // S0 = ||r||^2, S1 = sum p    -> hist[0], done?
    CTL_FP64_AFTER = 3, // same after one cycle         -> cycles++, hist, done?
    CTL_OUTER_INIT = 4, // S0 = ||r64||^2, S1 = sum p   -> hist[0], done?, inner reset
    CTL_OUTER_AFTER = 5,
    CTL_INNER = 6       // S0 = ||r_in||^2, S1 = sum e, S2 = ||e||^2
};

// Fixed-order reduction of nq partial-sum columns (q-major, nblk entries
// each) by one CTA (blockDim a multiple of 32); S[q] valid after return.
__device__ __forceinline__ void ctl_reduce(const double *partials, int nblk, int nq, double *S)
{
    __shared__ double wsum[32];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5, nw = blockDim.x >> 5;
    for (int q = 0; q < nq; ++q) {
        double s = 0.0;
        for (int b = t; b < nblk; b += blockDim.x) s += __ldcg(partials + (size_t)q * nblk + b);
        s = warp_sum(s);
        if (lane == 0) wsum[w] = s;
        __syncthreads();
        if (t == 0) {
            double u = 0.0;
            for (int k = 0; k < nw; ++k) u += wsum[k];
            S[q] = u;
        }
        __syncthreads();
    }
    if (t == 0)
        for (int q = nq; q < ISM_NQ; ++q) S[q] = 0.0;   // columns this control point does not form
    __syncthreads();
}

// Convergence bookkeeping of one control point (one thread).
__device__ __forceinline__ void ctl_decide(IsmState *st, const double *S, int mode)
{
    switch (mode) {
    case CTL_RHS_MEAN:
        st->mean = S[0] * st->inv_n;
        st->rhs_sum = S[0];
        st->rhs_l1 = S[1];
        break;
    case CTL_RHS_NORM: {
        const double bn = sqrt(S[0]);
        st->bnorm = bn;
        st->zero_rhs = (bn == 0.0);
        if (!isfinite(bn)) { st->status = ISM_ERR_NONFINITE; st->done = 1; }
        break;
    }
    case CTL_FP64_INIT:
    case CTL_FP64_AFTER:
    case CTL_OUTER_INIT:
    case CTL_OUTER_AFTER: {
        const bool fp64 = (mode == CTL_FP64_INIT || mode == CTL_FP64_AFTER);
        const bool after = (mode == CTL_FP64_AFTER || mode == CTL_OUTER_AFTER);
        int k;
        if (fp64) { if (after) st->cycles++; k = st->cycles; }
        else {
            if (after) { st->outer++; st->c64 ^= 1; }    // the refinement wrote the other buffer
            k = st->outer;
        }
        const double rel = st->bnorm > 0.0 ? sqrt(S[0]) / st->bnorm : 0.0;
        st->relres = rel;
        st->mean = S[1] * st->inv_n;
        if (k < ISM_HMAX) st->hist[k] = rel;
        if (st->tc_fail) { st->status = ISM_ERR_CUDA; st->done = 1; }   // a coarse solve gave up waiting
        else if (!isfinite(rel)) { st->status = ISM_ERR_NONFINITE; st->done = 1; }
        else if (rel <= st->tol || st->zero_rhs) { st->status = ISM_OK; st->done = 1; }
        else if (fp64 ? (st->cycles >= st->max_cycles)
                      : (st->outer >= st->max_outer || st->cycles >= st->max_cycles)) {
            st->status = ISM_ERR_NOT_CONVERGED;
            st->done = 1;
        }
        if (!fp64 && !st->done) {      // start a new inner solve on r = b - A p
            st->inner_done = 0;
            st->inner_cycles = 0;
            st->cur = 0;
            st->mean_e = 0.0;
            st->r32norm = sqrt(S[0]);
            st->skip_init = 0;
        }
        if (!fp64 && st->done) st->inner_done = 1;   // a finished problem runs no more cycles
        break;
    }
    case CTL_INNER: {
        st->inner_cycles++;
        st->cycles++;
        st->cur = (st->cur + st->npass) & 1;
        const double rin = sqrt(S[0]), en = sqrt(S[2]);
        st->rin = rin;
        st->enorm = en;
        st->mean_e = S[1] * st->inv_n;
        const double lim = fmax(st->inner_tol * st->r32norm, st->floor_mult * 0x1p-23 * en);
        if (!isfinite(rin) || st->tc_fail) st->inner_done = 1;
        else if (rin <= lim || st->inner_cycles >= st->inner_max || st->cycles >= st->max_cycles)
            st->inner_done = 1;
        break;
    }
    }
}

// Loop condition of a CUDA-graph while node driven by a control point: keep
// iterating while the phase is not finished.
__device__ __forceinline__ void ctl_set_condition(const IsmState *st, int mode, unsigned long long cond)
{
    if (!cond) return;
    const unsigned run = (mode == CTL_INNER) ? (st->inner_done ? 0u : 1u) : (st->done ? 0u : 1u);
    cudaGraphSetConditional((cudaGraphConditionalHandle)cond, run);
}

// Last-CTA-done control: every CTA has written its partial sums; the CTA
// that finishes last reduces them in fixed order and applies the control
// decision (and the loop condition of the enclosing graph node, when cond is
// nonzero), then re-arms the ticket.  No CTA waits for another.
__device__ __forceinline__ void ctl_last_block(IsmState *st, const double *partials, int nblk,
                                               int nq, int mode, unsigned long long cond = 0)
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
        ctl_decide(st, S, mode);
        st->ticket = 0;
        ctl_set_condition(st, mode, cond);
    }
}

static __global__ void k_zero(float *__restrict__ x, long long n)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        x[i] = 0.0f;
}

// Arm a graph while node: a handle created on a body graph starts each
// execution of that body with no defined value, so the enclosing body sets it.
static __global__ void k_arm_condition(unsigned long long cond)
{
    cudaGraphSetConditional((cudaGraphConditionalHandle)cond, 1u);
}

// ----------------------------------------------------------------- interpolation

// Bilinear prolongation value (Eq. 5) at fine cell (x, y) from coarse values
// q (ncy x ncx), coarse centre I at fine coordinate (I + 1/2) m.  Beyond the
// outermost centres the ghost centre mirrors the edge value: even at a
// Neumann face, odd (sign flip) at a Dirichlet-0 face.
template <typename T>
__device__ __forceinline__ T coarse_ghost(const T *__restrict__ q, int I, int J, int ncx,
                                          int ncy, int bcmask)
{
    bool neg = false;
    if (bcmask & ISM_PER_X) {
        I = wrap_mod(I, ncx);
    } else {
        if (I < 0) { I = 0; neg ^= (bcmask & 1) != 0; }
        if (I >= ncx) { I = ncx - 1; neg ^= (bcmask & 2) != 0; }
    }
    if (bcmask & ISM_PER_Y) {
        J = wrap_mod(J, ncy);
    } else {
        if (J < 0) { J = 0; neg ^= (bcmask & 4) != 0; }
        if (J >= ncy) { J = ncy - 1; neg ^= (bcmask & 8) != 0; }
    }
    T v = q[(size_t)J * ncx + I];
    return neg ? -v : v;
}

// Interpolation coordinate of fine cell x along an axis of n fine cells with
// coarse cells of m = 2^lm, nc of them, the last one w = n - (nc-1) m wide
// (w = m when m divides n): I0 is the coarse centre at or before the fine
// centre x + 1/2 (-1: the ghost before the first one), t the weight of
// I0 + 1.  Centre I sits at (I + 1/2) m except the last, at (nc-1) m + w/2;
// the ghost beyond it is mirrored across the wall (distance w).  Along a
// periodic axis (w = m) x may lie outside [0, n) and I0 runs over the
// periodic extension.
template <typename T>
__device__ __forceinline__ void interp_coord(int x, int n, int m, int lm, int nc, int &I0, T &t)
{
    const int hm = m >> 1;
    const int K = (nc - 1) << lm;          // first fine cell of the last coarse cell
    const int w = n - K;
    I0 = ((x - hm + m) >> lm) - 1;         // floor((x + 1/2)/m - 1/2)
    if (w == m || x < K - hm) {
        t = ((T)(x - I0 * m - hm) + (T)0.5) * ((T)1 / (T)m);   // m is a power of two: exact
    } else if (2 * x + 1 < 2 * K + w) {    // between centres nc-2 and nc-1, (m + w)/2 apart
        I0 = nc - 2;
        t = (T)(2 * (x - K + hm) + 1) / (T)(m + w);
    } else {                               // between the last centre and its ghost, w apart
        I0 = nc - 1;
        t = (T)(2 * (x - K) + 1 - w) / (T)(2 * w);
    }
}

template <typename T>
__device__ __forceinline__ T prolong_value(const T *__restrict__ q, int x, int y, int nx, int ny, int m,
                                           int ncx, int ncy, int bcmask, int kind)
{
    if (kind == ISM_COARSE_ACM) return q[(size_t)(y / m) * ncx + (x / m)];
    const int lm = __ffs(m) - 1;
    int I0, J0;
    T tx, ty;
    interp_coord<T>(x, nx, m, lm, ncx, I0, tx);
    interp_coord<T>(y, ny, m, lm, ncy, J0, ty);
    const T q11 = coarse_ghost(q, I0, J0, ncx, ncy, bcmask);
    const T q21 = coarse_ghost(q, I0 + 1, J0, ncx, ncy, bcmask);
    const T q12 = coarse_ghost(q, I0, J0 + 1, ncx, ncy, bcmask);
    const T q22 = coarse_ghost(q, I0 + 1, J0 + 1, ncx, ncy, bcmask);
    const T ux = (T)1 - tx, uy = (T)1 - ty;
    return q11 * ux * uy + q21 * tx * uy + q12 * ux * ty + q22 * tx * ty;
}

// ----------------------------------------------------------------- FP64 path

// One colour of a red-black Gauss-Seidel sweep, in place.  Each cell of the
// colour depends only on cells of the other colour, so the order inside a
// colour is free.  Grid: (ceil(ceil(nx/2)/blockDim), ny).
template <typename T>
__global__ void k_rbgs_colour(T *__restrict__ p, const T *__restrict__ b, int nx, int ny,
                              int bcmask, int colour, const int *skip, T scale = (T)1)
{
    if (skip && *skip) return;
    const int j = blockIdx.y;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = 2 * t + ((colour + j) & 1);
    if (i >= nx) return;
    const size_t idx = (size_t)j * nx + i;
    const T s = nb_sum<T>([&](long long k) -> T { return p[k]; }, (long long)idx, i, j, nx, ny, bcmask);
    p[idx] = (s - scale * b[idx]) * inv_diag<T>(diag_count(i, j, nx, ny, bcmask));
}

// ---- deep additive-correction V-cycle (2 x 2 agglomeration levels)

// out = 2 x 2 block sums of in (nx, ny even), sum order of the oracle.
template <typename T>
__global__ void k_restrict2(const T *__restrict__ in, T *__restrict__ out, int nx, int ny, const int *skip)
{
    if (skip && *skip) return;
    const int J = blockIdx.y, I = blockIdx.x * blockDim.x + threadIdx.x, ncx = nx >> 1;
    if (I >= ncx) return;
    const T *r0 = in + (size_t)(2 * J) * nx + 2 * I, *r1 = r0 + nx;
    out[(size_t)J * ncx + I] = ((r0[0] + r0[1]) + r1[0]) + r1[1];
}

// e = P e_c (piecewise constant over 2 x 2 blocks; overwrites e)
template <typename T>
__global__ void k_inject2(T *__restrict__ e, const T *__restrict__ ec, int nx, int ny, const int *skip)
{
    if (skip && *skip) return;
    const int j = blockIdx.y, i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nx) return;
    e[(size_t)j * nx + i] = ec[(size_t)(j >> 1) * (nx >> 1) + (i >> 1)];
}

// Residual r = b - A_f p, its 2 x 2 block sums and the partial sums
// (||r||^2, sum p, sum p^2), with the fused control; one thread per block.
template <typename T>
__global__ void k_resid2(const T *__restrict__ p, const T *__restrict__ b, T *__restrict__ rc,
                         double *partials, int nx, int ny, int bcmask, const int *skip, IsmState *ctl_st,
                         int ctl_mode, unsigned long long cond)
{
    if (skip && *skip) return;
    const int J = blockIdx.y, I = blockIdx.x * blockDim.x + threadIdx.x, ncx = nx >> 1;
    double r2 = 0.0, ps = 0.0, p2 = 0.0;
    if (I < ncx) {
        T acc = 0;
        for (int k = 0; k < 4; ++k) {                 // (2I, 2J), (2I+1, 2J), (2I, 2J+1), (2I+1, 2J+1)
            const int i = 2 * I + (k & 1), j = 2 * J + (k >> 1);
            const size_t idx = (size_t)j * nx + i;
            const T pc = p[idx];
            const T s = nb_sum<T>([&](long long q) -> T { return p[q]; }, (long long)idx, i, j, nx, ny, bcmask);
            const T r = b[idx] - (s - (T)diag_count(i, j, nx, ny, bcmask) * pc);
            acc += r;
            r2 += (double)r * (double)r;
            ps += (double)pc;
            p2 += (double)pc * (double)pc;
        }
        rc[(size_t)J * ncx + I] = acc;
    }
    double v[3] = {r2, ps, p2};
    block_partials<3>(v, partials, gridDim.x * gridDim.y, blockIdx.y * gridDim.x + blockIdx.x);
    if (ctl_mode >= 0) ctl_last_block(ctl_st, partials, gridDim.x * gridDim.y, 3, ctl_mode, cond);
}

// Residual r = b - A_f p, its m x m block sums (restriction) and the partial
// sums (||r||^2, sum p, sum p^2).  One CTA per coarse cell.
template <typename T>
__global__ void k_resid(const T *__restrict__ p, const T *__restrict__ b, T *__restrict__ rc,
                        double *partials, int nx, int ny, int m, int bcmask, const int *skip,
                        IsmState *ctl_st = nullptr, int ctl_mode = -1, unsigned long long cond = 0)
{
    if (skip && *skip) return;
    const int I = blockIdx.x, J = blockIdx.y, ncx = gridDim.x;
    const int mm = m * m;
    T acc = 0, r2 = 0, ps = 0, p2 = 0;
    for (int k = threadIdx.x; k < mm; k += blockDim.x) {
        const int i = I * m + (k % m), j = J * m + (k / m);
        if (i >= nx || j >= ny) continue;      // narrower last coarse cell
        const size_t idx = (size_t)j * nx + i;
        const T pc = p[idx];
        const T s = nb_sum<T>([&](long long q) -> T { return p[q]; }, (long long)idx, i, j, nx, ny, bcmask);
        const T r = b[idx] - (s - (T)diag_count(i, j, nx, ny, bcmask) * pc);
        acc += r;
        r2 += r * r;
        ps += pc;
        p2 += pc * pc;
    }
    // block sum of r (deterministic tree) -> rc
    __shared__ T redT[32];
    T a = warp_sum(acc);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if (lane == 0) redT[w] = a;
    __syncthreads();
    if (w == 0) {
        T t = lane < nw ? redT[lane] : (T)0;
        t = warp_sum(t);
        if (lane == 0) rc[(size_t)J * ncx + I] = t;
    }
    double v[3] = {(double)r2, (double)ps, (double)p2};
    block_partials<3>(v, partials, ncx * gridDim.y, J * ncx + I);
    if (ctl_mode >= 0) ctl_last_block(ctl_st, partials, ncx * gridDim.y, 3, ctl_mode, cond);
}

// p = p - mean + P e_c  (mean: state field when use_mean, else 0)
template <typename T>
__global__ void k_prolong(T *__restrict__ p, const T *__restrict__ ec, int nx, int ny, int m,
                          int ncx, int ncy, int bcmask, int kind, const IsmState *st,
                          int use_mean, const int *skip)
{
    if (skip && *skip) return;
    const int j = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nx) return;
    const size_t idx = (size_t)j * nx + i;
    T v = p[idx];
    if (use_mean) v -= (T)st->mean;
    p[idx] = v + prolong_value<T>(ec, i, j, nx, ny, m, ncx, ncy, bcmask, kind);
}

// Separable form of the bilinear prolongation (Eq. 5), used by the FP64
// cycle, where every FP64 operation counts (the FP64 pipe of this GPU runs at
// 1/64 of the FP32 rate).  First the coarse rows are interpolated along x:
// G[J][x] = (1 - t_x) e_c[J][I0] + t_x e_c[J][I0 + 1], with the ghost centres
// beyond a face along x as in coarse_ghost.  Grid (ceil(nx / 128), ncy).
template <typename T>
__global__ void k_prolong_x(const T *__restrict__ q, T *__restrict__ G, int nx, int m, int ncx, int ncy,
                            int bcmask, const int *skip)
{
    if (skip && *skip) return;
    const int J = blockIdx.y, x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= nx) return;
    int I0;
    T tx;
    interp_coord<T>(x, nx, m, __ffs(m) - 1, ncx, I0, tx);
    const T a = coarse_ghost(q, I0, J, ncx, ncy, bcmask), c = coarse_ghost(q, I0 + 1, J, ncx, ncy, bcmask);
    G[(size_t)J * nx + x] = ((T)1 - tx) * a + tx * c;
}

// Then along y: p = p - mean + (1 - t_y) G[J0][x] + t_y G[J0 + 1][x], the
// ghost rows beyond a south / north face folded into the two row weights
// (the sign of an odd ghost) or wrapped (periodic).  Grid (ceil(nx / 1024),
// ny), several cells per thread so that the row's weights are amortised.
template <typename T>
__global__ void k_prolong_y(T *__restrict__ p, const T *__restrict__ G, int nx, int ny, int m, int ncy,
                            int bcmask, const IsmState *st, int use_mean, const int *skip)
{
    if (skip && *skip) return;
    const int y = blockIdx.y;
    int J0;
    T ty;
    interp_coord<T>(y, ny, m, __ffs(m) - 1, ncy, J0, ty);
    T w0 = (T)1 - ty, w1 = ty;
    int J1 = J0 + 1;
    if (bcmask & ISM_PER_Y) {
        J0 = wrap_mod(J0, ncy);
        J1 = wrap_mod(J1, ncy);
    } else {
        if (J0 < 0) { J0 = 0; if (bcmask & 4) w0 = -w0; }
        if (J1 >= ncy) { J1 = ncy - 1; if (bcmask & 8) w1 = -w1; }
    }
    const T *__restrict__ g0 = G + (size_t)J0 * nx, *__restrict__ g1 = G + (size_t)J1 * nx;
    T *__restrict__ row = p + (size_t)y * nx;
    const T mu = use_mean ? (T)st->mean : (T)0;
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < nx; x += gridDim.x * blockDim.x) {
        T v = row[x];
        if (use_mean) v -= mu;
        row[x] = v + (w0 * g0[x] + w1 * g1[x]);
    }
}

// ----------------------------------------------------------------- coarse solve
// A_c = (Qy x Qx) diag(mu) (Qy x Qx)^T, so A_c^+ r_c = Qy [(Qy^T R Qx) / mu] Qx^T
// with 1/mu := 0 on the null mode.  R, E are ncy x ncx row-major.

// Row-parallel dense products with the j (or i) sums split over JS chunks
// of threads so that many loads are in flight; partial sums are combined in
// fixed order.  smem: (JS + 1) * n values.
template <typename T, typename F>
__device__ __forceinline__ void row_times_matrix(int n_out, int n_in, F term, T *part, T *out)
{
    const int nth = blockDim.x;
    const int JS = n_out >= nth ? 1 : nth / n_out;
    const int chunk = (n_in + JS - 1) / JS;
    for (int t = threadIdx.x; t < n_out * JS; t += nth) {
        const int o = t % n_out, c = t / n_out;
        const int j0 = c * chunk, j1 = min(n_in, j0 + chunk);
        T s = (T)0;
        int j = j0;
        for (; j + 8 <= j1; j += 8) {          // 8 independent terms in flight
            T u[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) u[q] = term(j + q, o);
#pragma unroll
            for (int q = 0; q < 8; ++q) s += u[q];
        }
        for (; j < j1; ++j) s += term(j, o);
        part[c * n_out + o] = s;
    }
    __syncthreads();
    for (int o = threadIdx.x; o < n_out; o += nth) {
        T s = (T)0;
        for (int c = 0; c < JS; ++c) s += part[c * n_out + o];
        out[o] = s;
    }
    __syncthreads();
}

// T[l][k] = Minv[l][k] * sum_i (sum_j QyT[l][j] R[j][i]) Qx[i][k] for row l (one CTA).
// FROM_PARTS: R[j][i] is the fixed-order sum of the 4 partial block sums.
template <typename T, bool FROM_PARTS>
__device__ __forceinline__ void coarse1_row(const T *__restrict__ R, const T *__restrict__ QyT,
                                            const T *__restrict__ Qx, const T *__restrict__ Minv,
                                            T *__restrict__ Tm, int ncx, int ncy, int l)
{
    extern __shared__ unsigned char smraw[];
    T *w = reinterpret_cast<T *>(smraw);
    T *v = w + ncx;
    T *part = v + ncx;
    const T *qrow = QyT + (size_t)l * ncy;
    row_times_matrix<T>(ncx, ncy, [&](int j, int i) -> T {
        const size_t k = (size_t)j * ncx + i;
        T rv;
        if (FROM_PARTS) {
            const T *q4 = R + 4 * k;
            rv = ((q4[0] + q4[1]) + q4[2]) + q4[3];
        } else {
            rv = R[k];
        }
        return qrow[j] * rv;
    }, part, w);
    row_times_matrix<T>(ncx, ncx, [&](int i, int k) -> T { return w[i] * Qx[(size_t)i * ncx + k]; }, part, v);
    for (int k = threadIdx.x; k < ncx; k += blockDim.x)
        Tm[(size_t)l * ncx + k] = v[k] * Minv[(size_t)l * ncx + k];
}

template <typename T, bool FROM_PARTS>
__global__ void k_coarse1(const T *__restrict__ R, const T *__restrict__ QyT,
                          const T *__restrict__ Qx, const T *__restrict__ Minv,
                          T *__restrict__ Tm, int ncx, int ncy, const int *skip)
{
    if (skip && *skip) return;
    coarse1_row<T, FROM_PARTS>(R, QyT, Qx, Minv, Tm, ncx, ncy, blockIdx.x);
}

// E[j][i] = sum_k (sum_l Qy[j][l] T[l][k]) QxT[k][i] for row j (one CTA).
// CLEAR_PARTS: the partial block sums of row j are cleared for the next
// restriction (fused single-precision cycle).
template <typename T, bool CLEAR_PARTS>
__device__ __forceinline__ void coarse2_row(const T *__restrict__ Tm, const T *__restrict__ Qy,
                                            const T *__restrict__ QxT, T *__restrict__ E, int ncx,
                                            int ncy, T *__restrict__ rcpart, int j)
{
    extern __shared__ unsigned char smraw[];
    T *w = reinterpret_cast<T *>(smraw);
    T *erow = w + ncx;
    T *part = erow + ncx;
    const T *qrow = Qy + (size_t)j * ncy;
    row_times_matrix<T>(ncx, ncy, [&](int l, int k) -> T { return qrow[l] * Tm[(size_t)l * ncx + k]; }, part, w);
    row_times_matrix<T>(ncx, ncx, [&](int k, int i) -> T { return w[k] * QxT[(size_t)k * ncx + i]; }, part, erow);
    for (int i = threadIdx.x; i < ncx; i += blockDim.x) E[(size_t)j * ncx + i] = erow[i];
    if (CLEAR_PARTS)
        for (int i = threadIdx.x; i < 4 * ncx; i += blockDim.x) rcpart[(size_t)j * ncx * 4 + i] = (T)0;
}

template <typename T, bool CLEAR_PARTS>
__global__ void k_coarse2(const T *__restrict__ Tm, const T *__restrict__ Qy,
                          const T *__restrict__ QxT, T *__restrict__ E, int ncx, int ncy,
                          const int *skip, T *__restrict__ rcpart)
{
    if (skip && *skip) return;
    coarse2_row<T, CLEAR_PARTS>(Tm, Qy, QxT, E, ncx, ncy, rcpart, blockIdx.x);
}
