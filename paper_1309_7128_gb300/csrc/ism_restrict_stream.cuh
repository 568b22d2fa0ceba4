// ism_restrict_stream.cuh -- residual r = b - A_f p and its aggregating
// restriction (Sec. 3.2-3.3: the block sums of r over the coarse cells), plus
// the partial sums (||r||^2, sum p, and in FP32 sum p^2) for the convergence
// control, in one streaming pass over p and b (FP32 or FP64).
//
// Each warp owns a strip of 128 columns starting at a multiple of 128 (so
// every coarse cell of the strip is whole: m/4 adjacent lanes) and a chunk of
// rows starting at a multiple of m (every coarse row is whole), and marches
// down the rows: p rows y-1, y, y+1 and b row y in registers, the rows ahead
// in a per-warp shared-memory ring filled by cp.async (each lane copies and
// reads only its own pieces: no barrier).  A lane sums r over its 4 columns
// and the m rows of the current coarse row in a fixed order; at the end of
// the coarse row the m/4 lanes of each coarse column combine their sums by a
// fixed butterfly and one of them writes the block sum.  The left and right
// neighbours of the strip's outer columns come through the ring as well
// (lanes 0 and 31 copy one more 16-byte group of p each; the other lanes
// copy zeros into a sink, so that no row takes a divergent branch).
// Cells outside the domain are 0 and add exactly 0; along a periodic axis the
// loads wrap (index mod n).  The pass reads 8 (FP32) or 16 (FP64) bytes per
// cell and writes one value per coarse cell.
#pragma once

#include "ism_stream32.cuh"

constexpr int RR_NW = 4;   // warps per CTA

template <typename T>
struct RestrictShape {
    static constexpr int PIECES = 4 * (int)sizeof(T) / 16;          // 16-byte pieces per lane and row
    static constexpr int RS = 8;                                     // ring rows (divides m)
    static constexpr int SLOT = 2 * 32 * 4 + 8;                      // p, b of 32 lanes, 2 halo groups
    static constexpr int WARP = RS * SLOT + 32 * 4;                  // + a sink for the halo copies of lanes 1..30
    static constexpr size_t smem = (size_t)RR_NW * WARP * sizeof(T);
};

// M = m (8, 16 or 32): the loop over the m rows of a coarse row is unrolled,
// and as the ring length divides m, every ring slot index is a constant.
template <typename T, int M>
__global__ void __launch_bounds__(32 * RR_NW)
k_restrict_stream(const T *__restrict__ p, const T *__restrict__ b, T *__restrict__ rc, double *partials, int nx,
                  int ny, int ncx, int bcmask, int nstrip, int chunk_h, int ntask, const int *skip,
                  IsmState *ctl_st, int ctl_mode, unsigned long long cond)
{
    using S = RestrictShape<T>;
    constexpr int RS = S::RS, PIECES = S::PIECES, SLOT = S::SLOT, E16 = 16 / (int)sizeof(T);
    constexpr int GL = M / 4;                                // lanes per coarse column
    constexpr int LM = M == 8 ? 3 : M == 16 ? 4 : 5;
    static_assert(M % RS == 0, "the ring length must divide m");
    if (skip && *skip) return;                               // the whole grid
    extern __shared__ __align__(16) unsigned char rr_raw[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // ring of this warp: [RS] slots of p [32 lanes][4], b [32][4], halo [2][4]; then the sink
    T *wring = reinterpret_cast<T *>(rr_raw) + (size_t)w * S::WARP;
    T *ring = wring + lane * 4;
    const int task = blockIdx.x * RR_NW + w;
    const bool active = task < ntask;                        // warp-uniform
    const bool per_x = (bcmask & ISM_PER_X) != 0, per_y = (bcmask & ISM_PER_Y) != 0;
    // norm partials per lane in T (a lane sums a few hundred cells; the
    // warp and CTA combine them in double)
    T r2 = (T)0, ps = (T)0, p2 = (T)0;

    if (active) {
        const int strip = task % nstrip, chunk = task / nstrip;
        const int x0 = strip * SRW;
        const int ya = chunk * chunk_h, yb = min(ny, ya + chunk_h);   // chunk_h: multiple of m
        const int cx = x0 + SNC * lane;
        const bool coldom = cx < nx;
        const bool colin = coldom || per_x;
        const T *pcol = p + (colin ? (per_x ? wrap_mod(cx, nx) : cx) : 0);
        const T *bcol = b + (colin ? (per_x ? wrap_mod(cx, nx) : cx) : 0);
        // halo group of this lane: lane 0 the 4 columns left of the strip,
        // lane 31 the 4 right of it
        const bool hlane = lane == 0 || lane == 31;
        const int hx = lane == 0 ? x0 - 4 : x0 + SRW;
        const bool hin = hlane && ((unsigned)hx < (unsigned)nx || per_x);
        const T *hcol = p + (hin ? (per_x ? wrap_mod(hx, nx) : hx) : 0);
        // every lane issues the halo copy (no divergent branch per row): lanes 0
        // and 31 into the slot's halo groups, the others 16 zero bytes into
        // their own place in the sink, which nothing reads
        T *hring = hlane ? wring + 2 * 32 * 4 + (lane == 0 ? 0 : 4) : wring + RS * SLOT + lane * 4;
        const int hstride = hlane ? SLOT : 0;

        // copies of row y into ring slot `slot` (zeros outside the domain)
        auto fetch = [&](int y, int slot) {
            bool rowin = (unsigned)y < (unsigned)ny;
            if (per_y) {                                     // |overhang| < ny
                y = y < 0 ? y + ny : (y >= ny ? y - ny : y);
                rowin = true;
            }
            const size_t roff = rowin ? (size_t)y * nx : 0;
            const int nb = rowin && colin ? 16 : 0;
            T *sl = ring + slot * SLOT;
#pragma unroll
            for (int c = 0; c < PIECES; ++c) {
                cp_async16(sl + c * E16, pcol + roff + c * E16, nb);
                cp_async16(sl + 32 * 4 + c * E16, bcol + roff + c * E16, nb);
            }
            const int nh = rowin && hin ? 16 : 0;
#pragma unroll
            for (int c = 0; c < PIECES; ++c) cp_async16(hring + slot * hstride + c * E16, hcol + roff + c * E16, nh);
            cp_async_commit();
        };
        // per-column divisor part (W / E faces) for diag = 4 + column part + row part
        T colD[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int x = cx + q;
            T d = (T)4;
            if (!per_x && x == 0) d += (bcmask & 1) ? (T)1 : (T)-1;
            if (!per_x && x == nx - 1) d += (bcmask & 2) ? (T)1 : (T)-1;
            colD[q] = d;
        }
        const T dS = (bcmask & 4) ? (T)1 : (T)-1, dN = (bcmask & 8) ? (T)1 : (T)-1;

        // row ya - 1 + k goes to slot k % RS; rows ya - 1 .. ya + RS - 3 first
#pragma unroll
        for (int k = 0; k < RS - 1; ++k) fetch(ya - 1 + k, k);
        T Pm[4], P0[4], Pn[4];
        cp_async_wait<RS - 3>();                             // rows ya - 1 and ya
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            Pm[q] = ring[q];
            P0[q] = ring[SLOT + q];
        }
        // coarse rows of the chunk; row y = ya + t sits in slot (t + 1) % RS,
        // and t = J M + j with RS | M, so the slot is (j + 1) % RS
        for (int yJ = ya; yJ < yb; yJ += M) {
            T acc = (T)0;
#pragma unroll
            for (int j = 0; j < M; ++j) {
                const int y = yJ + j;
                if (y < yb) {                                // warp-uniform
                    cp_async_wait<RS - 4>();                 // row y + 1 has landed
                    const T *sn = ring + ((j + 2) % RS) * SLOT;
                    const T *sb = ring + ((j + 1) % RS) * SLOT + 32 * 4;
                    const T *sh = wring + ((j + 1) % RS) * SLOT + 2 * 32 * 4;   // halo of row y
                    T bv[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) { Pn[q] = sn[q]; bv[q] = sb[q]; }
                    // left / right neighbours across lanes, and beyond the strip
                    T left = __shfl_up_sync(FULLMASK, P0[3], 1), right = __shfl_down_sync(FULLMASK, P0[0], 1);
                    if (lane == 0) left = sh[3];
                    if (lane == 31) right = sh[4];
                    // a lane beyond the east wall holds zeros; with a zero west
                    // neighbour as well its residuals are exactly 0, so every lane
                    // accumulates without a branch (a periodic x axis takes this
                    // pass only when its strips are whole, nx % 128 == 0)
                    if (!coldom) left = (T)0;
                    // refill the slot of row y - 2 (consumed) with row y + RS - 2
                    fetch(y + RS - 2, (j + RS - 1) % RS);
                    // diagonal: the south / north faces only change it on the
                    // domain's first and last rows (uniform branch)
                    T dg[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) dg[q] = colD[q];
                    if (!per_y && (y == 0 || y == ny - 1)) {
                        T rowD = (T)0;
                        if (y == 0) rowD += dS;
                        if (y == ny - 1) rowD += dN;
#pragma unroll
                        for (int q = 0; q < 4; ++q) dg[q] = colD[q] + rowD;
                    }
                    T rowsum = (T)0;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const T lf = q == 0 ? left : P0[q - 1], rt = q == 3 ? right : P0[q + 1];
                        // neighbour sum in the order of nb_sum (west, east, south, north);
                        // a neighbour outside the domain was loaded as 0, so adding it is exact
                        const T s = ((lf + rt) + Pm[q]) + Pn[q];
                        const T r = bv[q] - (s - dg[q] * P0[q]);
                        rowsum += r;
                        r2 = fma(r, r, r2);
                        ps += P0[q];
                        // sum p^2 feeds only the single-precision inner control
                        // (the FP64 controls read ||r|| and sum p)
                        if (sizeof(T) == 4) p2 = fma(P0[q], P0[q], p2);
                    }
                    acc += rowsum;
#pragma unroll
                    for (int q = 0; q < 4; ++q) { Pm[q] = P0[q]; P0[q] = Pn[q]; }
                }
            }
            // end of the coarse row: combine the m/4 lanes of each coarse column
            T v = acc;
#pragma unroll
            for (int o = 1; o < GL; o <<= 1) v += __shfl_xor_sync(FULLMASK, v, o);
            const int I = cx >> LM;
            if ((lane & (GL - 1)) == 0 && coldom && I < ncx) rc[(size_t)(yJ >> LM) * ncx + I] = v;
        }
        cp_async_wait<0>();
    }
    double v[3] = {(double)r2, (double)ps, (double)p2};
    block_partials<3>(v, partials, gridDim.x, blockIdx.x);
    if (ctl_mode >= 0) ctl_last_block(ctl_st, partials, gridDim.x, 3, ctl_mode, cond);
}
