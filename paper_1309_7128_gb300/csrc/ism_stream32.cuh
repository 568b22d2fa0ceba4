// ism_stream32.cuh -- single-precision red-black smoothing pass that streams
// the grid through registers (for grids larger than L2, where a pass is bound
// by HBM bandwidth).
//
// Every warp works alone (no barriers): it owns a strip of 128 columns (lane
// l holds columns 4l..4l+3) and a chunk of rows, and marches down the rows.
// At step t it takes input row y_t = ya - 2K + t (p and b) from a per-warp
// ring of RS rows in shared memory that cp.async keeps RS - 1 rows ahead
// (each lane copies and later reads only its own 16-byte pieces, so no
// barrier is needed), then runs the 2K half-sweeps of K
// red-black sweeps (Sec. 3.1, red first) as a wavefront: half-sweep s updates
// row y_t - 1 - s, whose neighbours already carry half-sweep s - 1 (row
// y_t - s was just updated by it, row y_t - 2 - s one step earlier), and row
// y_t - 2K is final and stored.  The rows in flight live in registers, a
// window of 2K + 2 rows; the step loop is unrolled over one turn of the
// window so that every slot is a fixed set of registers.
//
// Values at the strip's side edges are stale (the shuffles wrap to the lane
// itself) and the error front moves one column per half-sweep, so the warp
// stores the strip minus HC >= 2K columns on each side; likewise the rows
// before the chunk are read from y = ya - 2K on and the chunk's first stored
// row is clean.  Cells outside the domain are 0 and never updated, except
// along a periodic axis, where they are loaded from the other end (index
// mod n) and updated like any cell.  Input and output are different buffers
// (ping-pong), so chunks may read each other's rows freely.
//
// One pass moves 12 bytes per cell (read p, b; write p) plus the side halo
// (128 / (128 - 2 HC)) and the 4K rows a chunk reads twice.
#pragma once

#include "ism_sweep32.cuh"

constexpr int ST_NW = 4;          // warps per CTA (independent)

template <int K>
struct StreamShape {
    static constexpr int NS = 2 * K;                   // half-sweeps
    static constexpr int HC = ((NS + 3) / 4) * 4;      // side halo columns, multiple of 4
    static constexpr int VW = SRW - 2 * HC;            // stored columns per strip
    static constexpr int WN = NS + 2;                  // register window rows (even)
    static constexpr int RS = 8;                       // shared-memory ring rows per warp
    static constexpr size_t smem = (size_t)ST_NW * RS * 2 * 32 * sizeof(float4);
};

// 16-byte asynchronous copy global -> shared; src_bytes = 0 fills zeros
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc, int src_bytes)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(gsrc), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <int K>
__global__ void __launch_bounds__(32 * ST_NW) k_stream32(SweepArgs a, int nstrip, int chunk_h, int ntask)
{
    using S = StreamShape<K>;
    constexpr int NS = S::NS, HC = S::HC, VW = S::VW, WN = S::WN, RS = S::RS;
    extern __shared__ __align__(16) float4 ring_sm[];
    const int lane = threadIdx.x & 31;
    // this warp's ring: [RS][2][32] float4 (p, b), indexed by lane
    float4 *ring = ring_sm + (size_t)(threadIdx.x >> 5) * RS * 2 * 32 + lane;
    const int task = blockIdx.x * ST_NW + (threadIdx.x >> 5);
    if (task >= ntask) return;                         // whole warps
    if (a.skip && *a.skip) return;
    const int nx = a.nx, ny = a.ny;
    const int strip = task % nstrip, chunk = task / nstrip;
    const int x0 = strip * VW - HC;                    // even, multiple of 4
    const int ya = chunk * chunk_h, yb = min(ny, ya + chunk_h);   // chunk_h even: ya even
    const int T = (yb - ya) + 2 * NS;                  // steps
    const int cx = x0 + SNC * lane;
    const bool per_x = (a.bcmask & ISM_PER_X) != 0, per_y = (a.bcmask & ISM_PER_Y) != 0;
    const bool coldom = (unsigned)cx < (unsigned)nx;
    const bool colin = coldom || per_x;
    const bool colvalid = coldom && SNC * lane >= HC && SNC * lane < HC + VW;
    const int cxl = per_x ? wrap_mod(cx, nx) : cx;
    const int in = ((a.curp ? *a.curp : 0) + a.q) & 1;
    const float *__restrict__ pin = in ? a.e1 : a.e0;
    float *__restrict__ pout = in ? a.e0 : a.e1;

    // 1/d per column (W/E faces) and on the south / north rows
    float rq[SNC], inv_s[SNC], inv_n[SNC];
    {
        const float adjS = (a.bcmask & 4) ? 1.0f : -1.0f, adjN = (a.bcmask & 8) ? 1.0f : -1.0f;
#pragma unroll
        for (int q = 0; q < SNC; ++q) {
            const int x = cx + q;
            float d = 4.0f;
            if (!per_x && x == 0) d += (a.bcmask & 1) ? 1.0f : -1.0f;
            if (!per_x && x == nx - 1) d += (a.bcmask & 2) ? 1.0f : -1.0f;
            rq[q] = __frcp_rn(d);
            inv_s[q] = __frcp_rn(d + (per_y ? 0.0f : adjS));
            inv_n[q] = __frcp_rn(d + (per_y ? 0.0f : adjN));
        }
    }

    float P[WN][SNC], B[WN][SNC];
#pragma unroll
    for (int r = 0; r < WN; ++r)
#pragma unroll
        for (int q = 0; q < SNC; ++q) P[r][q] = B[r][q] = 0.0f;

    // start the copies of input row y into ring slot `slot` (zeros outside the
    // domain); one commit group per row, also when nothing is copied
    auto fetch = [&](int slot, int y) {
        bool rowin = (unsigned)y < (unsigned)ny;
        if (per_y && !rowin) { y = wrap_mod(y, ny); rowin = true; }
        const bool ok = rowin && colin;
        const size_t off = ok ? (size_t)y * nx + cxl : 0;
        cp_async16(ring + slot * 64, pin + off, ok ? 16 : 0);
        cp_async16(ring + slot * 64 + 32, a.b + off, ok ? 16 : 0);
        cp_async_commit();
    };

    const int y00 = ya - NS;                           // input row of step 0
#pragma unroll
    for (int u = 0; u < RS - 1; ++u) fetch(u, y00 + u); // rows past the chunk's end are harmless copies

    for (int t0 = 0; t0 < T; t0 += WN) {
#pragma unroll
        for (int u = 0; u < WN; ++u) {
            const int t = t0 + u;
            if (t < T) {
                // row of step t: its copy group is the oldest of the RS - 1 in flight
                cp_async_wait<RS - 2>();
                {
                    const float4 vp = ring[(t % RS) * 64], vb = ring[(t % RS) * 64 + 32];
                    P[u][0] = vp.x; P[u][1] = vp.y; P[u][2] = vp.z; P[u][3] = vp.w;
                    B[u][0] = vb.x; B[u][1] = vb.y; B[u][2] = vb.z; B[u][3] = vb.w;
                }
                // refill the slot read at step t - 1 with the row of step t + RS - 1
                fetch((t + RS - 1) % RS, y00 + t + RS - 1);
                const int yt = y00 + t;
#pragma unroll
                for (int s = 0; s < NS; ++s) {
                    const int y = yt - 1 - s;
                    const int r = (u + 2 * WN - 1 - s) % WN, rd = (u + 2 * WN - 2 - s) % WN,
                              ru = (u + 2 * WN - s) % WN;   // rows y, y - 1, y + 1
                    const bool rowok = per_y || (unsigned)y < (unsigned)ny;
                    // colour c = s & 1 updates q with (q + y) & 1 == c; ya is even,
                    // so the parity of y is that of t - 1 - s
                    const int qp = ((s & 1) + (u + 1 + s)) & 1;   // == ((s & 1) + y) & 1 as t0 is even
                    const bool south = !per_y && y == 0, north = !per_y && y == ny - 1;
                    if (qp == 0) {
                        const float left = __shfl_up_sync(FULLMASK, P[r][3], 1);
                        const float s0 = ((left + P[r][1]) + P[rd][0]) + P[ru][0];
                        const float s2 = ((P[r][1] + P[r][3]) + P[rd][2]) + P[ru][2];
                        if (rowok && colin) {
                            P[r][0] = (s0 - B[r][0]) * (south ? inv_s[0] : north ? inv_n[0] : rq[0]);
                            P[r][2] = (s2 - B[r][2]) * (south ? inv_s[2] : north ? inv_n[2] : rq[2]);
                        }
                    } else {
                        const float right = __shfl_down_sync(FULLMASK, P[r][0], 1);
                        const float s1 = ((P[r][0] + P[r][2]) + P[rd][1]) + P[ru][1];
                        const float s3 = ((P[r][2] + right) + P[rd][3]) + P[ru][3];
                        if (rowok && colin) {
                            P[r][1] = (s1 - B[r][1]) * (south ? inv_s[1] : north ? inv_n[1] : rq[1]);
                            P[r][3] = (s3 - B[r][3]) * (south ? inv_s[3] : north ? inv_n[3] : rq[3]);
                        }
                    }
                }
                // row y_t - 2K is final
                const int yo = yt - NS;
                const int ro = (u + 2 * WN - NS) % WN;
                if (colvalid && yo >= ya && yo < yb)
                    *reinterpret_cast<float4 *>(pout + (size_t)yo * nx + cx) =
                        make_float4(P[ro][0], P[ro][1], P[ro][2], P[ro][3]);
            }
        }
    }
    cp_async_wait<0>();                                // no copy outlives the warp
}
