// ism_coarse_tct.cu -- tensor-core coarse solve of the single-precision cycle
// for coarse grids up to 256 x 256 (tcgen05, TF32 operands, FP32 accumulation
// in TMEM), as a chain of four launches of one tiled GEMM kernel.
//
// The exact solve of the separable coarse operator (Sec. 3.3-3.4, Eq. 5-7),
// A_c = (Qy x Qx) diag(mu) (Qy x Qx)^T, is the product chain
//   T1 = Qy^T R,  T2 = (T1 Qx) .* Minv,  T3 = Qy T2,  E = T3 Qx^T
// (R the ncy x ncx restricted residual, Minv = 1/mu, 0 on the null mode).
// The single-CTA kernel of ism_coarse_tc.cu keeps every operand of the chain
// in one SM's shared memory, which caps it at 64 x 64 coarse cells; here each
// product is its own launch over a grid of CTAs, each CTA one 128-row x
// 32-column block of D = A B:
//   * every operand lives in global memory as a "chunked K-major" tile of TF32
//     words: K is cut into chunks of 32 columns, and chunk c holds columns
//     32c..32c+31 of every row as a K-major no-swizzle tile with K = 32,
//       byte(row, k) = (k / 32) rows 128 + (row / 8) 1024 + (k % 32 / 4) 128
//                      + (row % 8) 16 + (k % 4) 4,
//     so that a CTA's 128 A rows (or 32 B rows) of one chunk are one
//     contiguous run of bytes: one bulk asynchronous copy (cp.async.bulk);
//   * the chunks stream through a ring of shared-memory stages: one thread
//     requests the first stages at once (each completes on its own mbarrier),
//     issues the K = 8 MMAs of a chunk as soon as it has landed, and refills a
//     stage once the MMAs reading it have completed (tcgen05.commit);
//   * the epilogue reads the accumulator from TMEM (warp w: lanes 32w..32w+31,
//     one row per thread) and writes it straight into the chunked tile the
//     next product reads: T1 and T3 as A operands, T2 .* Minv transposed as
//     the B operand of the third product, E in plain row-major FP32;
//   * the first product builds its B operand, R^T, from the four partial
//     block sums per coarse cell that the last fused pass leaves (or from R
//     itself), and the last product clears those partial sums.
// Precision: the first two products form the spectral coefficients that
// Minv = 1/mu then scales, by up to 1/mu_min on the smoothest modes, so an
// error of one TF32 rounding (2^-11) relative to the largest coefficient is
// amplified there by mu_max/mu_min (thousands at 128 cells per axis); the
// last two map the coefficients back, and a TF32 rounding there leaves rough
// coarse-scale noise in the correction whose fine residual is again large
// next to the correction's own.  Measured, either costs extra cycles.  All
// four products therefore run in split TF32: each operand x = hi + lo with
// hi = tf32(x), lo = tf32(x - hi), and D = A_hi B_hi + A_hi B_lo + A_lo B_hi
// (three MMAs per K step, the lo x lo term of order 2^-22 dropped), accurate
// to about FP32 rounding like the CUDA-core solve.
// Every wait has a time limit on the global timer; a wait that runs out sets
// the state's tc_fail (the solve then ends with ISM_ERR_CUDA), lets the bulk
// copies and MMAs still in flight finish (again with a limit), frees the
// TMEM and returns.  Under the fault_test option the first product waits for
// an mbarrier phase that nothing completes.
#include <string.h>

#include <algorithm>
#include <vector>

#include "ism_kernels.cuh"
#include "ism_tc.cuh"

namespace {

constexpr int TT_THREADS = 128;               // 4 warps: one TMEM lane quarter each
constexpr int TT_MAXC = 256;                  // max ncx, ncy
constexpr int TT_N = 32;                      // accumulator columns per CTA
constexpr int TT_KC = 32;                     // K columns per chunk
constexpr uint32_t TT_ACH = 128u * TT_KC * 4; // bytes of one A chunk slice (128 rows)
constexpr uint32_t TT_BCH = TT_N * TT_KC * 4; // bytes of one B chunk slice (32 rows)
constexpr uint64_t TT_WAIT_NS = 200000000ull; // time limit of every mbarrier wait (0.2 s)

__host__ __device__ inline size_t tt_off(int row, int k, int rows)
{
    return (size_t)(k >> 5) * rows * 128 + (size_t)(row >> 3) * 1024 + ((k & 31) >> 2) * 128 + (row & 7) * 16 +
           (k & 3) * 4;
}

// Padded extents and the byte offsets of the operand tiles in one block,
// each operand as a hi and a lo tile of the same shape: constants Qy^T and
// Qy (A tiles, MP x KY), Qx and Qx^T as B tiles (NP x NP); then the
// intermediates T1 and T3 (A tiles, MP x NP, T3 over T1) and T2 .* Minv
// transposed (B tile, NP x KY).  `lo` is the distance of a lo tile from its
// hi tile.
struct TctLayout {
    int ncx, ncy, MP, KY, NP;
    size_t qyt, qy, qx2, qx4, t1, bufB, cbytes, bytes;
    size_t lo_ay, lo_bx, lo_t1, lo_b;
};

inline TctLayout tct_layout(int ncx, int ncy)
{
    TctLayout L;
    L.ncx = ncx;
    L.ncy = ncy;
    L.MP = (ncy + 127) & ~127;
    L.KY = (ncy + 31) & ~31;
    L.NP = (ncx + 31) & ~31;
    L.lo_ay = (size_t)L.MP * L.KY * 4;
    L.lo_bx = (size_t)L.NP * L.NP * 4;
    L.lo_t1 = (size_t)L.MP * L.NP * 4;
    L.lo_b = (size_t)L.NP * L.KY * 4;
    size_t o = 0;
    L.qyt = o; o += 2 * L.lo_ay;
    L.qy = o;  o += 2 * L.lo_ay;
    L.qx2 = o; o += 2 * L.lo_bx;
    L.qx4 = o; o += 2 * L.lo_bx;
    L.cbytes = o;
    L.t1 = o;   o += 2 * L.lo_t1;
    L.bufB = o; o += 2 * L.lo_b;
    L.bytes = o;
    return L;
}

// host: FP32 -> TF32 bits, round to nearest with ties away from zero (as cvt.rna.tf32.f32)
inline uint32_t host_tf32(float x)
{
    uint32_t u;
    memcpy(&u, &x, 4);
    if ((u & 0x7F800000u) == 0x7F800000u) return u;
    return (u + 0x1000u) & 0xFFFFE000u;
}

struct TctArgs {
    const unsigned char *A, *Alo;   // chunked A tile (MP rows): hi and lo parts
    const unsigned char *B, *Blo;   // chunked B tile (NP rows; BSRC 0): hi and lo parts
    const float *R;           // BSRC 1: 4 partial block sums per coarse cell; BSRC 2: R itself
    void *out, *outlo;        // OUT 0, 1: chunked tile, hi and lo parts; OUT 2: E (ncy x ncx)
    const float *minv;        // OUT 1: Minv (ncy x ncx)
    float *rcpart;            // OUT 2: partial block sums to clear, or NULL
    int *consumed;            // OUT 2: set to 1 once the solve has used R (batched: first restriction), or NULL
    const int *skip;
    IsmState *st;
    int K;                    // padded K of this product (a multiple of 32, <= 256)
    int ncx, ncy, MP, KY, NP;
    int fault_test;
};

// Shared memory of one launch: a ring of TT_STAGES stages, each the hi and
// lo parts of the A slice and, for BSRC 0, of the B slice of one chunk; for
// BSRC 1 and 2 the B operand (hi and lo) of every chunk after the ring.
constexpr int TT_STAGES = 4;
__host__ __device__ constexpr uint32_t tct_stage_bytes(int bsrc)
{
    return 2u * (TT_ACH + (bsrc == 0 ? TT_BCH : 0u));
}
__host__ __device__ inline uint32_t tct_smem(int bsrc, int K)
{
    const int nch = K / TT_KC, S = nch < TT_STAGES ? nch : TT_STAGES;
    return (uint32_t)S * tct_stage_bytes(bsrc) + (bsrc != 0 ? (uint32_t)nch * 2u * TT_BCH : 0u);
}

__device__ __forceinline__ void tf32_split(float x, uint32_t &hi, uint32_t &lo)
{
    hi = tc::to_tf32(x);
    lo = tc::to_tf32(x - __uint_as_float(hi));   // x - hi is exact in FP32
}

// D = A B for the CTA's block (rows m0..m0+127, columns n0..n0+31).
//   BSRC  0: B bulk-copied from a chunked tile; 1: B = R^T from the partial
//            block sums; 2: B = R^T from R.
//   OUT   0: D as an A operand (MP rows, K = NP); 1: D .* Minv transposed as
//            a B operand (NP rows, K = KY); 2: D into E, then clear rcpart.
// A and B in hi and lo parts, three MMAs per K step; OUT 0 and 1 write the
// hi and lo parts of the next operand.
// (cta, ncta): this CTA's index among the problem's CTAs and their number,
// which share the clearing of the partial block sums.
template <int BSRC, int OUT>
__device__ __forceinline__ void tct_body(const TctArgs &a, int n0, int m0, int cta, int ncta)
{
    constexpr int NS = TT_STAGES, NPART = 2;
    constexpr uint32_t SB = tct_stage_bytes(BSRC);
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t bar_full[NS], bar_empty[NS];
    __shared__ uint64_t bar_mma, bar_never;
    __shared__ uint32_t tslot;
    __shared__ int s_issued;
    const int t = threadIdx.x, nch = a.K >> 5, S = nch < NS ? nch : NS;
    unsigned char *ring = smem, *sBall = smem + S * SB;

    // chunk c into stage c % S: the A part(s), and for BSRC 0 the B part(s)
    auto copy_chunk = [&](int c) {
        const int st = c % S;
        unsigned char *base = ring + st * SB;
        const size_t ao = (size_t)c * a.MP * 128 + (size_t)m0 * 128;
        tc::mbar_expect_tx(&bar_full[st], SB);
        tc::bulk_g2s(base, a.A + ao, TT_ACH, &bar_full[st]);
        tc::bulk_g2s(base + TT_ACH, a.Alo + ao, TT_ACH, &bar_full[st]);
        if (BSRC == 0) {
            const size_t bo = (size_t)c * a.NP * 128 + (size_t)n0 * 128;
            tc::bulk_g2s(base + NPART * TT_ACH, a.B + bo, TT_BCH, &bar_full[st]);
            tc::bulk_g2s(base + NPART * TT_ACH + TT_BCH, a.Blo + bo, TT_BCH, &bar_full[st]);
        }
    };
    if (t == 0) {
        for (int q = 0; q < S; ++q) {
            tc::mbar_init(&bar_full[q], 1);
            tc::mbar_init(&bar_empty[q], 1);
        }
        tc::mbar_init(&bar_mma, 1);
        tc::mbar_init(&bar_never, 1);   // no thread ever arrives on it
        for (int c = 0; c < S; ++c) copy_chunk(c);
    }

    // first product: B rows n0..n0+31 of R^T (K = KY) for every chunk, four k
    // per 16-byte store; the loads of four items are issued before their sums
    if (BSRC != 0) {
        const int nit = TT_N * (a.K >> 2);
        for (int i0 = 0; i0 < nit; i0 += 4 * TT_THREADS) {
            float4 v[4][4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int i = i0 + u * TT_THREADS + t, row = i & (TT_N - 1), k0 = 4 * (i / TT_N), n = n0 + row;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int k = k0 + q;
                    v[u][q] = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (i < nit && n < a.ncx && k < a.ncy) {
                        if (BSRC == 1) v[u][q] = __ldcg(reinterpret_cast<const float4 *>(a.R) + (size_t)k * a.ncx + n);
                        else v[u][q].x = __ldcg(a.R + (size_t)k * a.ncx + n);
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int i = i0 + u * TT_THREADS + t, row = i & (TT_N - 1), k0 = 4 * (i / TT_N);
                if (i < nit) {
                    uint32_t hi[4], lo[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float r = ((v[u][q].x + v[u][q].y) + v[u][q].z) + v[u][q].w;
                        tf32_split(r, hi[q], lo[q]);
                    }
                    unsigned char *d = sBall + (size_t)(k0 >> 5) * NPART * TT_BCH + (row >> 3) * 1024 +
                                       ((k0 & 31) >> 2) * 128 + (row & 7) * 16;
                    *reinterpret_cast<uint4 *>(d) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
                    *reinterpret_cast<uint4 *>(d + TT_BCH) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
                }
            }
        }
    }

    if (t < 32) tc::tmem_alloc(&tslot, 32);
    tc::fence_smem_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tslot;

    // one thread issues the MMAs chunk by chunk as the copies land and
    // refills each stage once the MMAs reading it are done
    bool ok = true;
    int nfull = 0, ncopied = S;                  // thread 0: chunks landed / requested
    if (t == 0) {
        if (a.fault_test) ok = tc::mbar_wait(&bar_never, 0, TT_WAIT_NS);
        const uint32_t idesc = tc::idesc_tf32(128, TT_N);
        int issued = 0;
        for (int c = 0; c < nch && ok; ++c) {
            const int st = c % S;
            const uint32_t ph = (uint32_t)(c / S) & 1u;
            ok = tc::mbar_wait(&bar_full[st], ph, TT_WAIT_NS);
            if (!ok) break;
            nfull = c + 1;
            const uint32_t a0 = tc::smem_u32(ring + st * SB);
            const uint32_t b0 = BSRC == 0 ? a0 + NPART * TT_ACH
                                          : tc::smem_u32(sBall + (size_t)c * NPART * TT_BCH);
#pragma unroll
            for (int s = 0; s < TT_KC / 8; ++s) {
                const uint64_t ah = tc::smem_desc(a0 + s * 256, 128, 1024);
                const uint64_t bh = tc::smem_desc(b0 + s * 256, 128, 1024);
                tc::mma_tf32(tmem, ah, bh, idesc, c > 0 || s > 0);
                tc::mma_tf32(tmem, ah, tc::smem_desc(b0 + TT_BCH + s * 256, 128, 1024), idesc, true);
                tc::mma_tf32(tmem, tc::smem_desc(a0 + TT_ACH + s * 256, 128, 1024), bh, idesc, true);
            }
            issued = 1;
            if (c + S < nch) {
                tc::mma_commit(&bar_empty[st]);
                ok = tc::mbar_wait(&bar_empty[st], ph, TT_WAIT_NS);
                if (!ok) break;
                copy_chunk(c + S);
                ncopied = c + S + 1;
            }
        }
        if (issued) tc::mma_commit(&bar_mma);
        s_issued = issued;
    }
    __syncthreads();
    const bool issued = s_issued != 0;
    bool done = true;
    if (issued) done = tc::mbar_wait(&bar_mma, 0, TT_WAIT_NS);
    tc::fence_after_sync();
    const bool all = __syncthreads_and(done && ok && issued) != 0;

    if (all) {
        const int w = t >> 5, l = m0 + 32 * w + (t & 31);
        float v[32];
        {
            float h[16];
            tc::tmem_ld16(tmem + ((uint32_t)(32 * w) << 16), h);
#pragma unroll
            for (int q = 0; q < 16; ++q) v[q] = h[q];
            tc::tmem_ld16(tmem + ((uint32_t)(32 * w) << 16) + 16u, h);
#pragma unroll
            for (int q = 0; q < 16; ++q) v[16 + q] = h[q];
        }
        if (OUT == 0) {
            const size_t off = tt_off(l, n0, a.MP);
            unsigned char *o = static_cast<unsigned char *>(a.out) + off;
            unsigned char *ol = static_cast<unsigned char *>(a.outlo) + off;
            const bool rowin = l < a.ncy;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                uint32_t hi[4], lo[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float x = (rowin && n0 + 4 * q + j < a.ncx) ? v[4 * q + j] : 0.f;
                    tf32_split(x, hi[j], lo[j]);
                }
                *reinterpret_cast<uint4 *>(o + q * 128) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
                *reinterpret_cast<uint4 *>(ol + q * 128) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
            }
        } else if (OUT == 1) {
            if (l < a.KY) {
                unsigned char *o = static_cast<unsigned char *>(a.out), *ol = static_cast<unsigned char *>(a.outlo);
                const float *mrow = a.minv + (size_t)l * a.ncx;
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int n = n0 + j;
                    const float x = (l < a.ncy && n < a.ncx) ? v[j] * __ldg(mrow + n) : 0.f;
                    uint32_t hi, lo;
                    tf32_split(x, hi, lo);
                    const size_t off = tt_off(n, l, a.NP);
                    *reinterpret_cast<uint32_t *>(o + off) = hi;
                    *reinterpret_cast<uint32_t *>(ol + off) = lo;
                }
            }
        } else {
            if (l < a.ncy) {
                float *e = static_cast<float *>(a.out) + (size_t)l * a.ncx;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int n = n0 + 4 * q;
                    if ((a.ncx & 3) == 0 && n + 3 < a.ncx) {
                        *reinterpret_cast<float4 *>(e + n) = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                    } else {
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            if (n + j < a.ncx) e[n + j] = v[4 * q + j];
                    }
                }
            }
        }
    } else {
        // a wait ran out: report it, and give the copies and MMAs still in
        // flight a bounded time to finish (their memory is released below);
        // the requested but unconsumed chunks sit in distinct stages
        if (t == 0) {
            atomicExch(&a.st->tc_fail, 1);
            for (int c = nfull; c < ncopied; ++c) tc::mbar_wait(&bar_full[c % S], (uint32_t)(c / S) & 1u, TT_WAIT_NS);
        }
        if (issued && !done) tc::mbar_wait(&bar_mma, 0, TT_WAIT_NS);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (t < 32) tc::tmem_dealloc(tmem, 32);
    if (OUT == 2 && all && a.rcpart) {
        float4 *rp = reinterpret_cast<float4 *>(a.rcpart);
        const size_t ncell = (size_t)a.ncx * a.ncy, stride = (size_t)ncta * TT_THREADS;
        for (size_t i = (size_t)cta * TT_THREADS + t; i < ncell; i += stride) rp[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (OUT == 2 && all && a.consumed && cta == 0 && t == 0) *a.consumed = 1;
}

template <int BSRC, int OUT>
__global__ void __launch_bounds__(TT_THREADS) k_coarse_tct(TctArgs a)
{
    if (a.skip && *a.skip) return;
    tct_body<BSRC, OUT>(a, blockIdx.x * TT_N, blockIdx.y * 128, blockIdx.y * gridDim.x + blockIdx.x,
                        gridDim.x * gridDim.y);
}

// Batched ensemble: one launch per product over the blocks of every problem;
// work[b] = (problem, block column, block row, index of the block within the
// problem), tab[problem] that problem's arguments; problems outside an
// inner solve return at once.
template <int BSRC, int OUT>
__global__ void __launch_bounds__(TT_THREADS) k_coarse_tct_batch(const TctArgs *__restrict__ tab,
                                                                 const int4 *__restrict__ work)
{
    const int4 w = work[blockIdx.x];
    const TctArgs a = tab[w.x];
    if (a.skip && *a.skip) return;
    tct_body<BSRC, OUT>(a, w.y * TT_N, w.z * 128, w.w, (a.NP / TT_N) * (a.MP / 128));
}

template <int BSRC, int OUT>
void set_tct_smem()
{
    cudaFuncSetAttribute(k_coarse_tct<BSRC, OUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)tct_smem(BSRC, TT_MAXC));
    cudaFuncSetAttribute(k_coarse_tct_batch<BSRC, OUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)tct_smem(BSRC, TT_MAXC));
}

// The arguments of the four products for one context (rc, ec, rcpart as in
// ism_launch_coarse_tct).
void tct_chain_args(ism_ctx *ctx, const float *rc, float *ec, float *rcpart, const int *skip, TctArgs p[4])
{
    const TctLayout L = tct_layout(ctx->ncx, ctx->ncy);
    unsigned char *blk = static_cast<unsigned char *>(ctx->tct_block);
    TctArgs a;
    memset(&a, 0, sizeof(a));
    a.skip = skip;
    a.st = ctx->st;
    a.ncx = L.ncx; a.ncy = L.ncy; a.MP = L.MP; a.KY = L.KY; a.NP = L.NP;
    // T1 = Qy^T R (B = R^T built in shared memory)
    p[0] = a;
    p[0].A = blk + L.qyt; p[0].Alo = p[0].A + L.lo_ay; p[0].R = rc; p[0].K = L.KY;
    p[0].out = blk + L.t1; p[0].outlo = blk + L.t1 + L.lo_t1; p[0].fault_test = ctx->opt.fault_test;
    // T2 .* Minv = (T1 Qx) .* Minv, stored transposed as the next B operand
    p[1] = a;
    p[1].A = blk + L.t1; p[1].Alo = p[1].A + L.lo_t1; p[1].B = blk + L.qx2; p[1].Blo = p[1].B + L.lo_bx;
    p[1].K = L.NP; p[1].out = blk + L.bufB; p[1].outlo = blk + L.bufB + L.lo_b; p[1].minv = ctx->Minv32;
    // T3 = Qy (T2 .* Minv), over T1
    p[2] = a;
    p[2].A = blk + L.qy; p[2].Alo = p[2].A + L.lo_ay; p[2].B = blk + L.bufB; p[2].Blo = p[2].B + L.lo_b;
    p[2].K = L.KY; p[2].out = blk + L.t1; p[2].outlo = blk + L.t1 + L.lo_t1;
    // E = T3 Qx^T; the partial block sums are cleared for the next restriction
    p[3] = a;
    p[3].A = blk + L.t1; p[3].Alo = p[3].A + L.lo_t1; p[3].B = blk + L.qx4; p[3].Blo = p[3].B + L.lo_bx;
    p[3].K = L.NP; p[3].out = ec; p[3].rcpart = rcpart;
}

}  // namespace

bool ism_coarse_tct_fits(int ncx, int ncy)
{
    return ncx >= 1 && ncy >= 1 && ncx <= TT_MAXC && ncy <= TT_MAXC;
}

void ism_coarse_tct_prepare()
{
    set_tct_smem<1, 0>();
    set_tct_smem<2, 0>();
    set_tct_smem<0, 1>();
    set_tct_smem<0, 0>();
    set_tct_smem<0, 2>();
}

ism_status ism_coarse_tct_upload(ism_ctx *ctx, const std::vector<double> &Qx, const std::vector<double> &QxT,
                                 const std::vector<double> &Qy, const std::vector<double> &QyT)
{
    const int ncx = ctx->ncx, ncy = ctx->ncy;
    if (!ism_coarse_tct_fits(ncx, ncy)) return ISM_OK;   // CUDA-core path only
    const TctLayout L = tct_layout(ncx, ncy);
    std::vector<unsigned char> h(L.cbytes, 0);
    // split operand: hi = tf32(v), lo = tf32(v - hi)
    auto put2 = [&](size_t base, size_t base_lo, int row, int k, int rows, double v) {
        const uint32_t hb = host_tf32((float)v);
        float hf;
        memcpy(&hf, &hb, 4);
        const uint32_t lb = host_tf32((float)(v - (double)hf));
        memcpy(h.data() + base + tt_off(row, k, rows), &hb, 4);
        memcpy(h.data() + base_lo + tt_off(row, k, rows), &lb, 4);
    };
    for (int l = 0; l < ncy; ++l)
        for (int k = 0; k < ncy; ++k) {
            put2(L.qyt, L.qyt + L.lo_ay, l, k, L.MP, QyT[(size_t)l * ncy + k]);   // A[l][k] = QyT[l][k]
            put2(L.qy, L.qy + L.lo_ay, l, k, L.MP, Qy[(size_t)l * ncy + k]);      // A[l][k] = Qy[l][k]
        }
    for (int n = 0; n < ncx; ++n)
        for (int k = 0; k < ncx; ++k) {
            put2(L.qx2, L.qx2 + L.lo_bx, n, k, L.NP, Qx[(size_t)k * ncx + n]);    // B[n][k] = Qx[k][n]: T1 Qx
            put2(L.qx4, L.qx4 + L.lo_bx, n, k, L.NP, QxT[(size_t)k * ncx + n]);   // B[n][k] = QxT[k][n]: T3 QxT
        }
    if (!ctx->tct_block || ctx->tct_bytes != L.bytes) {
        if (ctx->tct_block) cudaFree(ctx->tct_block);
        ctx->tct_block = nullptr;
        if (cudaMalloc(&ctx->tct_block, L.bytes) != cudaSuccess) {
            cudaGetLastError();
            ctx->tct_block = nullptr;
            return ISM_ERR_NOMEM;
        }
        ctx->tct_bytes = L.bytes;
    }
    ISM_CUDA_TRY(cudaMemset(ctx->tct_block, 0, L.bytes));
    ISM_CUDA_TRY(cudaMemcpy(ctx->tct_block, h.data(), L.cbytes, cudaMemcpyHostToDevice));
    return ISM_OK;
}

ism_status ism_launch_coarse_tct(ism_ctx *ctx, const float *rc, bool from_parts, float *ec, float *rcpart,
                                 const int *skip)
{
    if (!ctx->tct_block) return ISM_ERR_ARG;
    const TctLayout L = tct_layout(ctx->ncx, ctx->ncy);
    TctArgs p[4];
    tct_chain_args(ctx, rc, ec, rcpart, skip, p);
    const dim3 grid(L.NP / TT_N, L.MP / 128);
    cudaStream_t s = ctx->ws;
    if (from_parts) k_coarse_tct<1, 0><<<grid, TT_THREADS, tct_smem(1, p[0].K), s>>>(p[0]);
    else k_coarse_tct<2, 0><<<grid, TT_THREADS, tct_smem(2, p[0].K), s>>>(p[0]);
    ISM_LAUNCH_CHECK(ctx);
    k_coarse_tct<0, 1><<<grid, TT_THREADS, tct_smem(0, p[1].K), s>>>(p[1]);
    ISM_LAUNCH_CHECK(ctx);
    k_coarse_tct<0, 0><<<grid, TT_THREADS, tct_smem(0, p[2].K), s>>>(p[2]);
    ISM_LAUNCH_CHECK(ctx);
    k_coarse_tct<0, 2><<<grid, TT_THREADS, tct_smem(0, p[3].K), s>>>(p[3]);
    ISM_LAUNCH_CHECK(ctx);
    return ISM_OK;
}

ism_status ism_coarse_tct_batch_table(ism_ctx *const *ctxs, int n, void **table, int *nwork, size_t smem[4])
{
    std::vector<TctArgs> t((size_t)4 * n);
    std::vector<int4> work;
    for (int q = 0; q < 4; ++q) smem[q] = 0;
    for (int d = 0; d < n; ++d) {
        ism_ctx *c = ctxs[d];
        if (!c->tct_block) return ISM_ERR_ARG;
        TctArgs p[4];
        tct_chain_args(c, c->rcpart, c->ec32, c->rcpart, &c->st->inner_done, p);
        p[3].consumed = &c->st->skip_init;
        for (int q = 0; q < 4; ++q) {
            t[(size_t)q * n + d] = p[q];
            smem[q] = std::max(smem[q], (size_t)tct_smem(q == 0 ? 1 : 0, p[q].K));
        }
        const int gx = p[0].NP / TT_N, gy = p[0].MP / 128;
        for (int by = 0; by < gy; ++by)
            for (int bx = 0; bx < gx; ++bx) work.push_back(make_int4(d, bx, by, by * gx + bx));
    }
    const size_t tb = t.size() * sizeof(TctArgs), wb = work.size() * sizeof(int4);
    if (cudaMalloc(table, tb + wb) != cudaSuccess) {
        cudaGetLastError();
        *table = nullptr;
        return ISM_ERR_NOMEM;
    }
    ISM_CUDA_TRY(cudaMemcpy(*table, t.data(), tb, cudaMemcpyHostToDevice));
    ISM_CUDA_TRY(cudaMemcpy(static_cast<unsigned char *>(*table) + tb, work.data(), wb, cudaMemcpyHostToDevice));
    *nwork = (int)work.size();
    return ISM_OK;
}

ism_status ism_launch_coarse_tct_batch(cudaStream_t s, const void *table, int n, int nwork, const size_t smem[4])
{
    const TctArgs *t = static_cast<const TctArgs *>(table);
    const int4 *w = reinterpret_cast<const int4 *>(t + (size_t)4 * n);
    k_coarse_tct_batch<1, 0><<<nwork, TT_THREADS, smem[0], s>>>(t, w);
    k_coarse_tct_batch<0, 1><<<nwork, TT_THREADS, smem[1], s>>>(t + n, w);
    k_coarse_tct_batch<0, 0><<<nwork, TT_THREADS, smem[2], s>>>(t + 2 * (size_t)n, w);
    k_coarse_tct_batch<0, 2><<<nwork, TT_THREADS, smem[3], s>>>(t + 3 * (size_t)n, w);
    return cudaGetLastError() == cudaSuccess ? ISM_OK : ISM_ERR_CUDA;
}
