// ism_sweep32.cuh -- single-precision fused smoothing pass, register tiled.
//
// One CTA owns a 128 x 128 region of the fine grid: 8 warps stacked along y,
// 16 rows each; lane l of a warp holds columns 4l..4l+3 of its 16 rows in
// registers, plus one halo row above and below.  A red-black half-sweep
// (Sec. 3.1) updates, in every row, the two cells of the active colour:
//   * the vertical neighbours are registers of the same thread,
//   * the in-thread horizontal neighbours are registers,
//   * the one outer horizontal neighbour comes from lane l-1 or l+1 with a
//     single warp shuffle (the active colour alternates by row, so a row
//     needs either the left or the right one, never both),
// i.e. five instructions per cell update.  After each half-sweep the first
// and last rows of every warp are exchanged through shared memory
// (double-buffered, one barrier per half-sweep).  The right-hand side b of
// the region is staged once per pass in tensor memory (TMEM, tcgen05.st),
// ordered so that one tcgen05.ld of four columns gives the b values of two
// rows of a half-sweep: the shared-memory pipe, which the shuffles and the
// row exchange also use, is left to them (TMEM has its own data path; with b
// in shared memory the pass was 6-11% slower, results bit-identical).
// Interior tiles hold -b/4 there, the edge tiles b.  The interior launch may
// update the two cells of a row with packed FP32 pair instructions
// (add.rn.f32x2, fma.rn.f32x2): each lane rounds like the scalar op, so the
// results are bit-identical; fewer instructions help when a pass runs many
// waves of tiles (issue-bound), the longer latency hurts when it runs few.
//
// K sweeps run on the region before it is written back.  Values at the
// region edge are stale (shuffles wrap to the lane itself, the outermost
// halo rows are never refreshed); the error front moves one cell per
// half-sweep, so after 2K half-sweeps every cell at distance >= 2K from the
// region edge equals K sequential sweeps.  The CTA writes back its valid
// tile, the region minus a halo H = 2K (+1 with the residual) on each side.
//
// Cells outside the domain are 0 and never updated (the neighbour sum then
// equals the sum over in-domain neighbours).  CTAs whose region lies strictly
// inside the domain take a path with divisor 4 everywhere and the right-hand
// side pre-scaled by 1/4; CTAs touching the boundary compute each cell's
// divisor d = 4 +- 1 per boundary face (Neumann -1, Dirichlet-0 +1).  Along
// a periodic axis the boundary CTAs load the region's out-of-domain rows /
// columns from the other end of the domain (index mod n) and update them like
// any other cell: they are copies, and the error front argument above holds
// unchanged.
//
// Interior tiles (region strictly inside the domain) read their rows without
// bounds checks, and while they sweep they start an L2 prefetch of the rows
// of the interior tile one wave of resident CTAs ahead (cp.async.bulk
// .prefetch.L2): that tile's CTA then loads from L2 what would otherwise come
// from HBM.
//
// Options fused into the pass:
//  PROLONG: add P e_c - mean while loading.  P e_c is evaluated in the
//           separable form of Eq. 5 (interpolation coordinates from
//           interp_coord, which also covers a narrower last coarse cell):
//           the CTA first interpolates the coarse rows it needs along x into
//           shared memory,
//           G[J][x] = (1 - t_x) e_c[J][I0] + t_x e_c[J][I0+1] (mirror ghosts
//           at the ends), then p += (1 - t_y) G[J0][x] + t_y G[J0+1][x].
//  RESID:   residual r = b - A_f p of the valid tile, its partial m x m block
//           sums (rcpart: 4 slots per coarse cell, one per covering tile,
//           summed in fixed order by the coarse solve) and the norm partials.
#pragma once

#include "ism_kernels.cuh"
#include "ism_tc.cuh"

constexpr int SNC = 4;                  // columns per thread
constexpr int SRR = 16;                 // rows per warp
constexpr int SNW = 8;                  // warps per CTA of the default region (NW template parameter below)
constexpr int SRW = 32 * SNC;           // region width 128
constexpr int SRH = SNW * SRR;          // region height 128
constexpr int STHREADS = 32 * SNW;      // 256
constexpr int SMAXK = 8;                // sweeps per pass (H <= 17, valid tile >= 94)

struct SweepArgs {
    float *e0, *e1;           // ping-pong iterate buffers
    const float *b;           // right-hand side
    const float *E;           // coarse correction e_c, ncy x ncx (PROLONG)
    float *rcpart;            // 4 partial block sums per coarse cell (RESID), zeroed before
    double *partials;         // per-CTA ||r||^2, sum p, sum p^2 (RESID)
    IsmState *st;             // mean_e (PROLONG); control block (RESID with ctl_mode >= 0)
    const int *skip;          // phase-finished flag or NULL
    const int *curp;          // buffer index of the input at q = 0, or NULL (= 0)
    int nx, ny, m, lm, ncx, ncy, bcmask, kind, K, q, use_mean, ctl_mode;
    int H, Hc, TW, TH;        // row halo, column halo (multiple of 4), valid tile width / height
    int gx, gy;               // tile grid
    int ix0, iy0;             // interior launch: tile = block + (ix0, iy0)
    const int2 *edge_tiles;   // edge launch: tile = edge_tiles[block]
    unsigned long long cond;  // graph while-node handle set by the control, or 0
    int pf_ahead;             // interior tiles: prefetch into L2 the tile this many tiles ahead (0: off)
    int pgx, pn;              // interior tile grid: columns and number of tiles (row-major from ix0, iy0)
};

// Row halo 2K (+1 for the residual); the column halo is rounded up to a
// multiple of 4 so that every thread's 4 columns are one aligned float4.
__host__ __device__ inline int sweep_halo(int K, bool resid) { return 2 * K + (resid ? 1 : 0); }
__host__ __device__ inline int sweep_halo_cols(int K, bool resid) { return (sweep_halo(K, resid) + 3) & ~3; }
__host__ __device__ inline int sweep_tile_w(int K, bool resid) { return SRW - 2 * sweep_halo_cols(K, resid); }
__host__ __device__ inline int sweep_tile_h(int K, bool resid, int nw = SNW)
{
    return nw * SRR - 2 * sweep_halo(K, resid);
}

// Bulk prefetch of `bytes` (a multiple of 16, 16-byte aligned) into L2.
__device__ __forceinline__ void prefetch_l2(const void *p, unsigned bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" :: "l"(p), "r"(bytes) : "memory");
}

// Start bringing the rows of p and b that interior tile `id` (row-major
// over the interior tiles) loads into L2 (one bulk prefetch per row of its
// region, clipped to the domain), so that the CTA that runs it about one
// wave later finds them there instead of in HBM.  Same tile geometry as
// sweep_tile.
template <int NW>
__device__ __forceinline__ void prefetch_tile(const SweepArgs &a, const float *pin, int id)
{
    if (id >= a.pn) return;
    const int bx = id % a.pgx + a.ix0, by = id / a.pgx + a.iy0;
    const int x0 = bx * a.TW - a.Hc, y0 = by * a.TH - a.H;
    const int xa = max(x0, 0), xb = min(x0 + SRW, a.nx);
    if (xb <= xa) return;
    const unsigned bytes = (unsigned)(xb - xa) * 4u;       // x0, nx multiples of 4: 16-byte pieces
    for (int k = threadIdx.x; k < 2 * ((NW * SRR) + 2); k += (32 * NW)) {
        const bool isb = k >= (NW * SRR) + 2;
        const int y = y0 - 1 + (isb ? k - ((NW * SRR) + 2) : k);
        if ((unsigned)y >= (unsigned)a.ny || (isb && (y < y0 || y >= y0 + (NW * SRR)))) continue;
        prefetch_l2((isb ? a.b : pin) + (size_t)y * a.nx + xa, bytes);
    }
}

// b in tensor memory (TMEM): warp w owns 64 columns of TMEM lane quarter
// w % 4 (lane l of the warp = TMEM lane 32 (w % 4) + l), from column
// 64 (w / 4).  Column PAR 32 + 2 r + j holds, for region row r of the warp,
// b at column 4l + qp + 2j with qp = PAR ^ (r & 1): the two cells row r
// updates in a half-sweep of colour parity PAR.  A half-sweep reads its
// rows' values in pairs of rows (four consecutive columns).
__device__ __forceinline__ void tmem_st8(uint32_t taddr, float v0, float v1, float v2, float v3, float v4, float v5,
                                         float v6, float v7)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};"
                 :: "r"(taddr), "r"(__float_as_uint(v0)), "r"(__float_as_uint(v1)), "r"(__float_as_uint(v2)),
                    "r"(__float_as_uint(v3)), "r"(__float_as_uint(v4)), "r"(__float_as_uint(v5)),
                    "r"(__float_as_uint(v6)), "r"(__float_as_uint(v7))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float4 &lo, float4 &hi)
{
    uint32_t r0, r1, r2, r3, r4, r5, r6, r7;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3), "=r"(r4), "=r"(r5), "=r"(r6), "=r"(r7) : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r0), "+r"(r1), "+r"(r2), "+r"(r3), "+r"(r4), "+r"(r5), "+r"(r6), "+r"(r7) :: "memory");
    lo = make_float4(__uint_as_float(r0), __uint_as_float(r1), __uint_as_float(r2), __uint_as_float(r3));
    hi = make_float4(__uint_as_float(r4), __uint_as_float(r5), __uint_as_float(r6), __uint_as_float(r7));
}

__device__ __forceinline__ float4 tmem_ld4(uint32_t taddr)
{
    uint32_t r0, r1, r2, r3;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" : "+r"(r0), "+r"(r1), "+r"(r2), "+r"(r3) :: "memory");
    return make_float4(__uint_as_float(r0), __uint_as_float(r1), __uint_as_float(r2), __uint_as_float(r3));
}

// Rows r0..r0+3 of b (one float4 per row: the thread's 4 columns) into TMEM.
__device__ __forceinline__ void b_store4(uint32_t tb, int r0, const float4 (&v)[4])
{
    // PAR 0: even row (b0, b2), odd row (b1, b3); PAR 1: even (b1, b3), odd (b0, b2)
    tmem_st8(tb + 2 * r0, v[0].x, v[0].z, v[1].y, v[1].w, v[2].x, v[2].z, v[3].y, v[3].w);
    tmem_st8(tb + 32 + 2 * r0, v[0].y, v[0].w, v[1].x, v[1].z, v[2].y, v[2].w, v[3].x, v[3].z);
}

// Divisor contribution of the south / north faces for global row y.
__device__ __forceinline__ float row_adj(int y, int ny, int bcmask)
{
    float d = 0.0f;
    if (bcmask & ISM_PER_Y) return d;
    if (y == 0) d += (bcmask & 4) ? 1.0f : -1.0f;
    if (y == ny - 1) d += (bcmask & 8) ? 1.0f : -1.0f;
    return d;
}

// Boundary data of a warp for the edge launch: rows [rlo, rhi) of the warp
// lie in the domain; row rs (rn) is the domain's south (north) row, or -1;
// the divisor of a cell is 4 + column part + adjS/adjN on those rows.
struct EdgeRows {
    int rlo, rhi, rs, rn;
    float inv_s[SNC], inv_n[SNC];   // 1/d on the south and north domain rows
};

__device__ __forceinline__ float edge_inv(const EdgeRows &er, const float (&rq)[SNC], int r, int q)
{
    return r == er.rs ? er.inv_s[q] : (r == er.rn ? er.inv_n[q] : rq[q]);
}

// Half-sweep of colour parity PAR over the warp's rows; EDGE selects the
// boundary-aware update (out-of-domain cells are never updated).
// Packed FP32 pairs (sm_100+): one instruction for the two same-colour
// cells of a row; each lane of the pair rounds exactly like the scalar op.
__device__ __forceinline__ float2 add2(float2 a, float2 b)
{
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\t"
        "mov.b64 rb, {%4, %5};\n\t"
        "add.rn.f32x2 rd, ra, rb;\n\t"
        "mov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c)
{
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\t"
        "mov.b64 rb, {%4, %5};\n\t"
        "mov.b64 rc, {%6, %7};\n\t"
        "fma.rn.f32x2 rd, ra, rb, rc;\n\t"
        "mov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}

template <int PAR, bool EDGE, bool PK>
__device__ __forceinline__ void half_sweep(float (&P)[SRR + 2][SNC], const uint32_t tb, const int lane,
                                           const float (&idq)[SNC], const float (&rq)[SNC],
                                           const bool colin, const EdgeRows &er)
{
    float4 bb2 = make_float4(0.f, 0.f, 0.f, 0.f), bb3 = bb2;
#pragma unroll
    for (int r = 0; r < SRR; ++r) {
        const int qp = PAR ^ (r & 1);            // which pair of columns has the active colour
        if ((r & 3) == 0) tmem_ld8(tb + PAR * 32 + 2 * r, bb2, bb3);
        else if ((r & 3) == 2) bb2 = bb3;
        const float2 bb = (r & 1) ? make_float2(bb2.z, bb2.w) : make_float2(bb2.x, bb2.y);
        if (qp == 0) {
            const float left = __shfl_up_sync(FULLMASK, P[r + 1][3], 1);
            if (!EDGE && PK) {
                float2 t = add2(make_float2(left, P[r + 1][1]), make_float2(P[r + 1][1], P[r + 1][3]));
                t = add2(t, make_float2(P[r][0], P[r][2]));
                t = add2(t, make_float2(P[r + 2][0], P[r + 2][2]));
                t = fma2(t, make_float2(0.25f, 0.25f), bb);          // bb holds -b / 4
                P[r + 1][0] = t.x;
                P[r + 1][2] = t.y;
            } else if (!EDGE) {
                const float s0 = ((left + P[r + 1][1]) + P[r][0]) + P[r + 2][0];
                const float s2 = ((P[r + 1][1] + P[r + 1][3]) + P[r][2]) + P[r + 2][2];
                P[r + 1][0] = fmaf(s0, 0.25f, bb.x);
                P[r + 1][2] = fmaf(s2, 0.25f, bb.y);
            } else if (colin && r >= er.rlo && r < er.rhi) {
                const float s0 = ((left + P[r + 1][1]) + P[r][0]) + P[r + 2][0];
                const float s2 = ((P[r + 1][1] + P[r + 1][3]) + P[r][2]) + P[r + 2][2];
                P[r + 1][0] = (s0 - bb.x) * edge_inv(er, rq, r, 0);
                P[r + 1][2] = (s2 - bb.y) * edge_inv(er, rq, r, 2);
            }
        } else {
            const float right = __shfl_down_sync(FULLMASK, P[r + 1][0], 1);
            if (!EDGE && PK) {
                float2 t = add2(make_float2(P[r + 1][0], P[r + 1][2]), make_float2(P[r + 1][2], right));
                t = add2(t, make_float2(P[r][1], P[r][3]));
                t = add2(t, make_float2(P[r + 2][1], P[r + 2][3]));
                t = fma2(t, make_float2(0.25f, 0.25f), bb);          // bb holds -b / 4
                P[r + 1][1] = t.x;
                P[r + 1][3] = t.y;
            } else if (!EDGE) {
                const float s1 = ((P[r + 1][0] + P[r + 1][2]) + P[r][1]) + P[r + 2][1];
                const float s3 = ((P[r + 1][2] + right) + P[r][3]) + P[r + 2][3];
                P[r + 1][1] = fmaf(s1, 0.25f, bb.x);
                P[r + 1][3] = fmaf(s3, 0.25f, bb.y);
            } else if (colin && r >= er.rlo && r < er.rhi) {
                const float s1 = ((P[r + 1][0] + P[r + 1][2]) + P[r][1]) + P[r + 2][1];
                const float s3 = ((P[r + 1][2] + right) + P[r][3]) + P[r + 2][3];
                P[r + 1][1] = (s1 - bb.x) * edge_inv(er, rq, r, 1);
                P[r + 1][3] = (s3 - bb.y) * edge_inv(er, rq, r, 3);
            }
        }
    }
}

// After a half-sweep of colour parity PAR only the cells of that colour in a
// warp's first and last rows changed, and only those are read across the
// warp boundary before the next exchange (a cell's vertical neighbour has
// the other colour): each boundary row passes one float2 per lane, the pair
// (q, q + 2) with q = PAR for the first (even) row and PAR ^ 1 for the last
// (odd) row.  Two consecutive exchanges bring both colours of the halo rows
// up to date.
template <int NW, int PAR>
__device__ __forceinline__ void exchange_rows(float (&P)[SRR + 2][SNC], float *xch, int buf, int w, int lane)
{
    constexpr int q0 = PAR, q1 = PAR ^ 1;
    float2 *X = reinterpret_cast<float2 *>(xch);
    // xch layout: [2 buffers][NW warps][2 rows][32 lanes] float2
    const int base = buf * NW * 2 * 32;
    X[base + (w * 2 + 0) * 32 + lane] = make_float2(P[1][q0], P[1][q0 + 2]);
    X[base + (w * 2 + 1) * 32 + lane] = make_float2(P[SRR][q1], P[SRR][q1 + 2]);
    __syncthreads();
    // the first and last warps read their own slots instead of a missing
    // neighbour's and keep their outer halo rows (no branches)
    const bool up = w > 0, dn = w < NW - 1;
    const float2 vu = X[base + ((up ? w - 1 : w) * 2 + 1) * 32 + lane];
    const float2 vd = X[base + ((dn ? w + 1 : w) * 2 + 0) * 32 + lane];
    P[0][q1] = up ? vu.x : P[0][q1];
    P[0][q1 + 2] = up ? vu.y : P[0][q1 + 2];
    P[SRR + 1][q0] = dn ? vd.x : P[SRR + 1][q0];
    P[SRR + 1][q0 + 2] = dn ? vd.y : P[SRR + 1][q0 + 2];
}

// G rows needed by a region of NW warps: its rows span at most 16 NW / 8 + 3
// coarse rows (m >= 8); its columns at most SRW/8 + 3 coarse columns (e_c
// block staged before G)
__host__ __device__ constexpr int sweep_grows(int nw) { return nw * SRR / 8 + 3; }
constexpr int SGCOLS = SRW / 8 + 3;
inline size_t sweep_smem_bytes(int nw = SNW)
{
    return (size_t)2 * nw * 2 * SRW * 4 + (size_t)sweep_grows(nw) * SRW * 4 +
           (size_t)sweep_grows(nw) * SGCOLS * 4;
}

// EDGE: the launch over the tiles whose region touches the domain boundary
// (listed in edge_tiles); otherwise the launch over the interior tiles.
// PK (interior tiles): the two same-colour cells of a row in packed FP32
// pairs (fewer instructions, longer latency; bit-identical results).
// The pass on tile (bx, by) of the problem described by a; one CTA.
template <int NW, bool PROLONG, bool RESID, bool EDGE, bool PK = false>
__device__ __forceinline__ void sweep_tile(const SweepArgs &a, const int bx, const int by, const int pf_id)
{
    extern __shared__ __align__(16) float sm[];
    float *xch = sm;                       // row exchange buffers
    float *gsm = xch + 2 * NW * 2 * SRW;  // coarse correction rows G[Jg0 ..] of this region
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nx = a.nx, ny = a.ny, H = a.H, Hc = a.Hc, TW = a.TW, TH = a.TH;
    const int x0 = bx * TW - Hc, y0 = by * TH - H;  // region origin, x0 % 4 == 0
    const int cx = x0 + SNC * lane;        // first column of this thread
    const int ry0 = w * SRR;               // first region row of this warp
    constexpr bool edge = EDGE;
    const int in = ((a.curp ? *a.curp : 0) + a.q) & 1;
    const float *__restrict__ pin = in ? a.e1 : a.e0;
    float *__restrict__ pout = in ? a.e0 : a.e1;
    // TMEM for b: NW x 16 columns (64 per warp; warps w and w + 4 share a
    // lane quarter).  At most 256 columns per SM (two CTAs of 8 warps or one
    // of 16, as registers allow), of 512, so the allocation never waits long.
    __shared__ uint32_t tslot;
    if (w == 0) tc::tmem_alloc(&tslot, (uint32_t)(NW * 16));
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tb = tslot + ((uint32_t)(32 * (w & 3)) << 16) + (uint32_t)(64 * (w >> 2));
    // nx % 4 == 0 and cx % 4 == 0: a thread's 4 columns are all in or all out
    const bool per_x = EDGE && (a.bcmask & ISM_PER_X), per_y = EDGE && (a.bcmask & ISM_PER_Y);
    const bool coldom = (unsigned)cx < (unsigned)nx;
    const bool colin = coldom || per_x;    // columns loaded and updated
    const bool colvalid = coldom && (SNC * lane >= Hc) && (SNC * lane < Hc + TW);
    const int cxl = per_x ? wrap_mod(cx, nx) : cx;   // column loaded from

    // divisor part from the W/E faces and its reciprocal (edge launch)
    float idq[SNC], rq[SNC];
#pragma unroll
    for (int q = 0; q < SNC; ++q) {
        const int x = cx + q;
        float d = 4.0f;
        if (!per_x && x == 0) d += (a.bcmask & 1) ? 1.0f : -1.0f;
        if (!per_x && x == nx - 1) d += (a.bcmask & 2) ? 1.0f : -1.0f;
        idq[q] = d;
        rq[q] = __frcp_rn(d);
    }
    EdgeRows er;
    {
        const int yw = y0 + ry0;                     // global row of the warp's row 0
        er.rlo = per_y ? 0 : max(0, -yw);
        er.rhi = per_y ? SRR : min(SRR, ny - yw);
        er.rs = (!per_y && yw <= 0 && 0 < yw + SRR) ? -yw : -1;
        er.rn = (!per_y && yw <= ny - 1 && ny - 1 < yw + SRR) ? ny - 1 - yw : -1;
        const float adjS = (a.bcmask & 4) ? 1.0f : -1.0f;
        const float adjN = (a.bcmask & 8) ? 1.0f : -1.0f;
#pragma unroll
        for (int q = 0; q < SNC; ++q) {
            er.inv_s[q] = __frcp_rn(idq[q] + adjS);   // ny >= 8: a row is never both
            er.inv_n[q] = __frcp_rn(idq[q] + adjN);
        }
    }

    // 1. load p (rows -1..SRR) and b; with PROLONG, the block of e_c the region
    //    needs is requested first, so that its latency overlaps the loads of p
    //    and b, and the prolongation is added to the registers afterwards
    float P[SRR + 2][SNC];
    const int m = a.m, lm = a.lm, hm = m >> 1;
    const bool acm = a.kind == ISM_COARSE_ACM;
    // rows of e_c used by region rows y0-1 .. y0+(NW * SRR) (clamped to the coarse grid)
    int Jg0 = 0, nrow = 0, Ic0 = 0, ncol = 0;
    float *esm = gsm + sweep_grows(NW) * SRW;
    if (PROLONG) {
        // along a periodic axis the coarse indices are not clamped: they run
        // over the periodic extension and wrap when e_c is read
        Jg0 = acm ? (y0 - 1) >> lm : ((y0 - 1 - hm + m) >> lm) - 1;
        int Jg1 = acm ? (y0 + (NW * SRR)) >> lm : ((y0 + (NW * SRR) - hm + m) >> lm);
        if (!per_y) { Jg0 = max(0, Jg0); Jg1 = min(a.ncy - 1, Jg1); }
        nrow = Jg1 - Jg0 + 1;
        // (a) columns Ic0..Ic1: the bilinear neighbours of the loaded columns
        const int xs = per_x ? x0 : max(x0, 0), xe = (per_x ? x0 + SRW : min(x0 + SRW, nx)) - 1;
        Ic0 = acm ? (xs >> lm) : ((xs - hm + m) >> lm) - 1;
        int Ic1 = acm ? xe >> lm : ((xe - hm + m) >> lm);
        if (!per_x) { Ic0 = max(0, Ic0); Ic1 = min(a.ncx - 1, Ic1); }
        ncol = Ic1 - Ic0 + 1;
        for (int t = threadIdx.x; t < nrow * ncol; t += (32 * NW)) {
            const int jr = t / ncol, c = t - jr * ncol;
            const int J = per_y ? wrap_mod(Jg0 + jr, a.ncy) : Jg0 + jr;
            const int I = per_x ? wrap_mod(Ic0 + c, a.ncx) : Ic0 + c;
            esm[t] = a.E[(size_t)J * a.ncx + I];
        }
    }
    if (!EDGE) {
        // interior tile: every row and column of the region lies in the domain,
        // so the rows are read without bounds checks (fewer instructions in
        // the load phase: 8% of the pass at 8192 x 4096)
        const float *src = pin + (size_t)(y0 + ry0 - 1) * nx + cx;
#pragma unroll
        for (int r = 0; r < SRR + 2; ++r) {
            const float4 v = *reinterpret_cast<const float4 *>(src + (size_t)r * nx);
            P[r][0] = v.x; P[r][1] = v.y; P[r][2] = v.z; P[r][3] = v.w;
        }
        const float *bsrc = a.b + (size_t)(y0 + ry0) * nx + cx;
#pragma unroll
        for (int r0 = 0; r0 < SRR; r0 += 4) {
            float4 v[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                v[k] = *reinterpret_cast<const float4 *>(bsrc + (size_t)(r0 + k) * nx);
                v[k].x *= -0.25f; v[k].y *= -0.25f; v[k].z *= -0.25f; v[k].w *= -0.25f;
            }
            b_store4(tb, r0, v);
        }
    } else {
#pragma unroll
        for (int r = 0; r < SRR + 2; ++r) {
            int y = y0 + ry0 + r - 1;
            bool rowin = (unsigned)y < (unsigned)ny;
            if (per_y && !rowin) { y = wrap_mod(y, ny); rowin = true; }   // periodic copy
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (rowin && colin) v = *reinterpret_cast<const float4 *>(pin + (size_t)y * nx + cxl);
            P[r][0] = v.x; P[r][1] = v.y; P[r][2] = v.z; P[r][3] = v.w;
        }
#pragma unroll
        for (int r0 = 0; r0 < SRR; r0 += 4) {
            float4 v[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                int y = y0 + ry0 + r0 + k;
                bool rowin = (unsigned)y < (unsigned)ny;
                if (per_y && !rowin) { y = wrap_mod(y, ny); rowin = true; }
                v[k] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (rowin && colin) v[k] = *reinterpret_cast<const float4 *>(a.b + (size_t)y * nx + cxl);
            }
            b_store4(tb, r0, v);
        }
    }
    if (PROLONG) {
        const float mean = a.use_mean ? (float)a.st->mean_e : 0.f;
        const int ncx = a.ncx;
        __syncthreads();
        // (b) G[J][x] = e_c interpolated along x for the region's columns
        for (int t = threadIdx.x; t < nrow * 32; t += (32 * NW)) {
            const int jr = t >> 5, l = t & 31, xb = x0 + SNC * l;
            float g[SNC] = {0.f, 0.f, 0.f, 0.f};
            if ((unsigned)xb < (unsigned)nx || per_x) {
                const float *er = esm + jr * ncol - Ic0;      // er[I] = e_c[Jg0 + jr][I], Ic0 <= I <= Ic1
#pragma unroll
                for (int q = 0; q < SNC; ++q) {
                    const int x = xb + q;
                    if (acm) {
                        g[q] = er[x >> lm];
                    } else {
                        int I0;
                        float tx;
                        interp_coord<float>(x, nx, m, lm, ncx, I0, tx);
                        float qa, qb;
                        if (per_x) {
                            qa = er[I0];
                            qb = er[I0 + 1];
                        } else {
                            qa = I0 < 0 ? ((a.bcmask & 1) ? -er[0] : er[0]) : er[I0];
                            qb = I0 + 1 >= ncx ? ((a.bcmask & 2) ? -er[ncx - 1] : er[ncx - 1]) : er[I0 + 1];
                        }
                        g[q] = (1.0f - tx) * qa + tx * qb;
                    }
                }
            }
            reinterpret_cast<float4 *>(gsm)[jr * 32 + l] = make_float4(g[0], g[1], g[2], g[3]);
        }
        __syncthreads();
        // (c) p += P e_c - mean along y, per loaded row
        const float4 *gs4 = reinterpret_cast<const float4 *>(gsm) + lane;
#pragma unroll
        for (int r = 0; r < SRR + 2; ++r) {
            const int y = y0 + ry0 + r - 1;
            if (((unsigned)y < (unsigned)ny || per_y) && colin) {
                float4 ga, gb;
                float wa, wb;
                if (acm) {
                    ga = gs4[((y >> lm) - Jg0) * 32];
                    gb = ga;
                    wa = 1.0f;
                    wb = 0.0f;
                } else {
                    int J0;
                    float ty;
                    interp_coord<float>(y, ny, m, lm, a.ncy, J0, ty);
                    int Ja = J0, Jb = J0 + 1;
                    float sa = 1.f, sb = 1.f;
                    if (!per_y && Ja < 0) { Ja = 0; if (a.bcmask & 4) sa = -1.f; }
                    if (!per_y && Jb >= a.ncy) { Jb = a.ncy - 1; if (a.bcmask & 8) sb = -1.f; }
                    ga = gs4[(Ja - Jg0) * 32];
                    gb = gs4[(Jb - Jg0) * 32];
                    wa = sa * (1.0f - ty);
                    wb = sb * ty;
                }
                P[r][0] = (P[r][0] - mean) + fmaf(wa, ga.x, wb * gb.x);
                P[r][1] = (P[r][1] - mean) + fmaf(wa, ga.y, wb * gb.y);
                P[r][2] = (P[r][2] - mean) + fmaf(wa, ga.z, wb * gb.z);
                P[r][3] = (P[r][3] - mean) + fmaf(wa, ga.w, wb * gb.w);
            }
        }
    }

    if (!EDGE && pf_id >= 0) prefetch_tile<NW>(a, pin, pf_id);
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");

    // 2. 2K half-sweeps, red ((x+y) even) first
    const int base = (x0 + y0 + ry0) & 1;      // colour parity of (column 0, row 0) of this warp
    if (base == 0) {
        for (int s = 0; s < a.K; ++s) {
            half_sweep<0, EDGE, PK>(P, tb, lane, idq, rq, colin, er);
            exchange_rows<NW, 0>(P, xch, 0, w, lane);
            half_sweep<1, EDGE, PK>(P, tb, lane, idq, rq, colin, er);
            exchange_rows<NW, 1>(P, xch, 1, w, lane);
        }
    } else {
        for (int s = 0; s < a.K; ++s) {
            half_sweep<1, EDGE, PK>(P, tb, lane, idq, rq, colin, er);
            exchange_rows<NW, 1>(P, xch, 0, w, lane);
            half_sweep<0, EDGE, PK>(P, tb, lane, idq, rq, colin, er);
            exchange_rows<NW, 0>(P, xch, 1, w, lane);
        }
    }

    // 3. write back the valid tile (rows [H, H+TH), columns [Hc, Hc+TW) of the region)
    if (!EDGE) {
        if (SNC * lane >= Hc && SNC * lane < Hc + TW) {
            float *dst = pout + (size_t)(y0 + ry0) * nx + cx;
#pragma unroll
            for (int r = 0; r < SRR; ++r) {
                const int rr = ry0 + r;
                if (rr >= H && rr < H + TH)
                    *reinterpret_cast<float4 *>(dst + (size_t)r * nx) =
                        make_float4(P[r + 1][0], P[r + 1][1], P[r + 1][2], P[r + 1][3]);
            }
        }
    } else if (colvalid) {
#pragma unroll
        for (int r = 0; r < SRR; ++r) {
            const int rr = ry0 + r, y = y0 + rr;
            if (rr >= H && rr < H + TH && (unsigned)y < (unsigned)ny)
                *reinterpret_cast<float4 *>(pout + (size_t)y * nx + cx) =
                    make_float4(P[r + 1][0], P[r + 1][1], P[r + 1][2], P[r + 1][3]);
        }
    }

    if (RESID) {
        // 4. residual of the valid tile; per-thread sums of r over the (up to
        //    three) coarse rows that this warp's 16 rows touch
        const int yw = y0 + ry0, Jw = yw >> lm;          // floor division (yw may be < 0)
        const int r1 = ((Jw + 1) << lm) - yw, r2 = ((Jw + 2) << lm) - yw;
        float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f;
        float r2s = 0.f, ps = 0.f, p2 = 0.f;
        float4 bA = make_float4(0.f, 0.f, 0.f, 0.f), bB = bA;
#pragma unroll
        for (int r = 0; r < SRR; ++r) {
            if ((r & 1) == 0) {
                bA = tmem_ld4(tb + 2 * r);          // row r: (b0, b2), row r + 1: (b1, b3)
                bB = tmem_ld4(tb + 32 + 2 * r);     // row r: (b1, b3), row r + 1: (b0, b2)
            }
            const float left = __shfl_up_sync(FULLMASK, P[r + 1][3], 1);
            const float right = __shfl_down_sync(FULLMASK, P[r + 1][0], 1);
            const int rr = ry0 + r, y = y0 + rr;
            const bool ok = colvalid && rr >= H && rr < H + TH && (unsigned)y < (unsigned)ny;
            const float bq[SNC] = {(r & 1) ? bB.z : bA.x, (r & 1) ? bA.z : bB.x, (r & 1) ? bB.w : bA.y,
                                   (r & 1) ? bA.w : bB.y};
            const float ra = row_adj(y, ny, a.bcmask);
            float rowsum = 0.f;
#pragma unroll
            for (int q = 0; q < SNC; ++q) {
                const float lf = q == 0 ? left : P[r + 1][q - 1];
                const float rt = q == SNC - 1 ? right : P[r + 1][q + 1];
                const float pc = P[r + 1][q];
                const float sn = ((lf + rt) + P[r][q]) + P[r + 2][q];
                const float bb = EDGE ? bq[q] : -4.0f * bq[q];
                const float res = EDGE ? bb - (sn - (idq[q] + ra) * pc) : bb - fmaf(-4.0f, pc, sn);
                if (ok) { rowsum += res; r2s = fmaf(res, res, r2s); ps += pc; p2 = fmaf(pc, pc, p2); }
            }
            if (r < r1) acc0 += rowsum;
            else if (r < r2) acc1 += rowsum;
            else acc2 += rowsum;
        }
        // 5. partial block sums over (coarse cell) x (valid tile): gather the
        //    per-thread sums of every coarse cell in fixed (warp, row-part,
        //    lane) order
        __syncthreads();                                  // xch is reused below
        float *racc = xch;                                // [NW][3][32]
        racc[(w * 3 + 0) * 32 + lane] = acc0;
        racc[(w * 3 + 1) * 32 + lane] = acc1;
        racc[(w * 3 + 2) * 32 + lane] = acc2;
        __syncthreads();
        const int gx_lo = bx * TW, gx_hi = min(gx_lo + TW, nx);
        const int gy_lo = by * TH, gy_hi = min(gy_lo + TH, ny);
        const int I0 = gx_lo >> lm, I1 = (gx_hi - 1) >> lm, J0 = gy_lo >> lm, J1 = (gy_hi - 1) >> lm;
        const int nbx = I1 - I0 + 1, nb = nbx * (J1 - J0 + 1);
        for (int cb = threadIdx.x; cb < nb; cb += (32 * NW)) {
            const int I = I0 + cb % nbx, J = J0 + cb / nbx;
            // lanes whose 4 columns lie in coarse column I
            const int l0 = max(0, (I * m - x0 + 3) >> 2), l1 = min(32, ((I + 1) * m - x0 + 3) >> 2);
            float sacc = 0.f;
            for (int ww = 0; ww < NW; ++ww) {
                const int k = J - ((y0 + ww * SRR) >> lm);
                if (k < 0 || k > 2) continue;
                const float *row = racc + (ww * 3 + k) * 32;
                for (int l = l0; l < l1; ++l) sacc += row[l];
            }
            const int slot = (bx - (I * m) / TW) + 2 * (by - (J * m) / TH);
            a.rcpart[((size_t)J * a.ncx + I) * 4 + slot] = sacc;
        }
        // 6. norm partials (per-warp float sums combined in double), then the
        //    fused convergence control in the last CTA to finish
        __shared__ double red[3][NW];
        const double v0 = warp_sum(r2s), v1 = warp_sum(ps), v2 = warp_sum(p2);
        if (lane == 0) { red[0][w] = v0; red[1][w] = v1; red[2][w] = v2; }
        __syncthreads();
        const int nblk = a.gx * a.gy;
        if (threadIdx.x < 3) {
            double t = 0.0;
            for (int k = 0; k < NW; ++k) t += red[threadIdx.x][k];
            a.partials[(size_t)threadIdx.x * nblk + by * a.gx + bx] = t;
        }
        if (a.ctl_mode >= 0) ctl_last_block(a.st, a.partials, nblk, 3, a.ctl_mode, a.cond);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (w == 0) tc::tmem_dealloc(tslot, (uint32_t)(NW * 16));
}

template <int NW, bool PROLONG, bool RESID, bool EDGE, bool PK = false>
__global__ void __launch_bounds__(32 * NW, 16 / NW) k_sweep32(SweepArgs a)
{
    if (a.skip && *a.skip) return;
    if (EDGE) {
        const int2 t = a.edge_tiles[blockIdx.x];
        sweep_tile<NW, PROLONG, RESID, EDGE>(a, t.x, t.y, -1);
    } else {
        const int id = blockIdx.y * gridDim.x + blockIdx.x;
        sweep_tile<NW, PROLONG, RESID, EDGE, PK>(a, blockIdx.x + a.ix0, blockIdx.y + a.iy0,
                                             a.pf_ahead > 0 ? id + a.pf_ahead : -1);
    }
}

// Batched form: work item (problem, tile x, tile y) per CTA over the per-problem
// argument table; problems whose phase is finished return at once.
template <bool PROLONG, bool RESID, bool EDGE>
__global__ void __launch_bounds__(STHREADS, 2) k_sweep32_batch(const SweepArgs *__restrict__ table,
                                                               const int4 *__restrict__ work)
{
    const int4 w = work[blockIdx.x];
    const SweepArgs &a = table[w.x];
    if (a.skip && *a.skip) return;
    sweep_tile<SNW, PROLONG, RESID, EDGE>(a, w.y, w.z, -1);
}

// Sum of the 4 partial block sums (fixed order) -> R (ncy x ncx).
__device__ __forceinline__ float rc_from_parts(const float *rcpart, size_t k)
{
    const float4 v = reinterpret_cast<const float4 *>(rcpart)[k];
    return ((v.x + v.y) + v.z) + v.w;
}
