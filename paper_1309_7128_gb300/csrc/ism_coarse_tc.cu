// ism_coarse_tc.cu -- exact coarse solve of the single-precision cycle on the
// tensor cores (tcgen05, TF32 operands, FP32 accumulation in TMEM).
//
// The coarse operator of the ISM (Sec. 3.3-3.4, Eq. 5-7) is separable,
// A_c = (Qy x Qx) diag(mu) (Qy x Qx)^T, so the exact solve e_c = A_c^+ r_c is
// four small dense products (Sec. 3.4 solves the coarse system iteratively
// instead; the CUDA-core path of the same products is in ism_kernels.cuh):
//   T1 = Qy^T R,  T2 = (T1 Qx) .* Minv,  T3 = Qy T2,  E = T3 Qx^T,
// R the ncy x ncx restricted residual, Minv = 1/mu (0 on the null mode).
//
// One CTA runs the chain.  Every product is one accumulator of 128 TMEM lanes
// (rows; zero operand rows beyond ncy) x Np columns (ncx padded to a
// multiple of 16), fed from shared memory by K/8 MMA instructions that one
// thread issues.  The constant operands -- Qy^T and Qy as A tiles, Q_x in
// the two orientations as B tiles, and Minv -- are laid out once per context
// as TF32 tiles in global memory and arrive with bulk asynchronous copies
// while the threads stage R^T from the partial block sums; the intermediate
// products come back from TMEM with tcgen05.ld and are written as the next
// product's operand.  Operands are TF32 (10-bit mantissa, round to nearest);
// the FP64 refinement around the single-precision cycles removes the
// difference.
//
// Limits: ncx, ncy <= 64 (all operand tiles resident, <= 177 KB of shared
// memory); larger coarse grids, up to 256 x 256, take the tiled split-TF32
// chain of ism_coarse_tct.cu, and beyond that the CUDA-core path.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "ism_kernels.cuh"
#include "ism_tc.cuh"

namespace {

constexpr int CT_THREADS = 256;
constexpr int CT_MAXC = 64;                   // max ncx, ncy
constexpr uint64_t CT_WAIT_NS = 200000000ull; // time limit of every mbarrier wait (0.2 s)
constexpr uint32_t CT_CHUNK = 32768;          // bytes per bulk copy
constexpr int CT_RITEMS = (CT_MAXC * CT_MAXC / 4 + CT_THREADS - 1) / CT_THREADS;   // R^T items per thread

// Byte layout of the operand tiles (shared memory; the first part, the
// constants, is also the layout of the global block).
struct TcLayout {
    int ncx, ncy, Np, Kx, Ky;
    uint32_t cA1, cA3, cB2, cB4, minv, cbytes;    // constants: Qy^T, Qy (128 x Ky), B tiles of Qx (Np x Kx), Minv
    uint32_t dA, dB, scr, bytes;                   // products: A (128 x Kx), B (Np x Ky); transpose scratch
};

__host__ __device__ inline uint32_t up16(uint32_t b) { return (b + 15u) & ~15u; }

__host__ __device__ inline TcLayout tc_layout(int ncx, int ncy)
{
    TcLayout L;
    L.ncx = ncx; L.ncy = ncy;
    L.Np = (ncx + 15) & ~15;
    L.Kx = (ncx + 7) & ~7;
    L.Ky = (ncy + 7) & ~7;
    uint32_t o = 0;
    L.cA1 = o; o += 128u * L.Ky * 4;
    L.cA3 = o; o += 128u * L.Ky * 4;
    L.cB2 = o; o += (uint32_t)L.Np * L.Kx * 4;
    L.cB4 = o; o += (uint32_t)L.Np * L.Kx * 4;
    L.minv = o; o += up16((uint32_t)ncx * ncy * 4);
    L.cbytes = o;
    L.dA = o; o += 128u * L.Kx * 4;
    L.dB = o; o += (uint32_t)L.Np * L.Ky * 4;
    L.scr = o; o += (uint32_t)L.Ky * (L.Np + 4) * 4;
    L.bytes = o;
    return L;
}

// host: byte offset of (row, k) in a K-major tile (same rule as tc::kmajor_offset)
inline size_t host_kmajor(int row, int k, int K)
{
    return (size_t)(row >> 3) * (32 * K) + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4;
}

// host: FP32 -> TF32 bits, round to nearest with ties away from zero (as cvt.rna.tf32.f32)
inline uint32_t host_tf32(float x)
{
    uint32_t u;
    memcpy(&u, &x, 4);
    if ((u & 0x7F800000u) == 0x7F800000u) return u;   // inf / nan unchanged
    return (u + 0x1000u) & 0xFFFFE000u;
}

struct CoarseTcArgs {
    const float *R;           // FROM_PARTS: 4 partial block sums per coarse cell; else R itself
    const unsigned char *cst; // constant tiles (TcLayout, cbytes bytes)
    float *E;                 // ncy x ncx
    float *rcpart;            // cleared after use, or NULL
    TcLayout L;
    int tcols;                // TMEM columns allocated
    const int *skip;
    IsmState *st;             // tc_fail is set when a wait runs out
    int *consumed;            // set to 1 once R has been used (batched: first restriction), or NULL
    int fault_test;           // 1: wait first for a phase that nothing completes (failure-detection test)
};

__device__ __forceinline__ void put4(unsigned char *tile, int row, int k, int K, float a, float b, float c,
                                     float d)
{
    *reinterpret_cast<uint4 *>(tile + tc::kmajor_offset(row, k, K)) =
        make_uint4(tc::to_tf32(a), tc::to_tf32(b), tc::to_tf32(c), tc::to_tf32(d));
}

// Issue D = A B over K (one thread), commit, and wait for completion (all
// threads; CTA-uniform result).  On failure the MMAs may still be in flight:
// *pending receives the parity of their phase (else -1).
__device__ bool run_gemm(const unsigned char *sA, const unsigned char *sB, int K, uint32_t tmem, uint32_t idesc,
                         uint64_t *bar, uint32_t parity, int *pending)
{
    tc::fence_smem_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (threadIdx.x == 0) {
        const uint32_t a0 = tc::smem_u32(sA), b0 = tc::smem_u32(sB);
        for (int s = 0; s < K / 8; ++s)
            tc::mma_tf32(tmem, tc::smem_desc(a0 + s * 256, 128, 32 * K), tc::smem_desc(b0 + s * 256, 128, 32 * K),
                         idesc, s > 0);
        tc::mma_commit(bar);
    }
    const bool ok = tc::mbar_wait(bar, parity, CT_WAIT_NS);
    tc::fence_after_sync();
    const bool all = __syncthreads_and(ok) != 0;
    *pending = all ? -1 : (int)parity;
    return all;
}

// Accumulator row `row` (the TMEM lane of this warp's quarter), 16-column
// chunks c = 16 g for the g of this warp's half (warps w and w + 4 share a
// lane quarter).
template <typename F>
__device__ __forceinline__ void read_rows(uint32_t tmem, int Np, F f)
{
    const int w = threadIdx.x >> 5, row = 32 * (w & 3) + (threadIdx.x & 31);
    for (int c = 16 * (w >> 2); c < Np; c += 32) {
        float v[16];
        tc::tmem_ld16(tmem + ((uint32_t)(32 * (w & 3)) << 16) + (uint32_t)c, v);
        f(row, c, v);
    }
}

template <bool FROM_PARTS>
__device__ __forceinline__ void coarse_tc_body(const CoarseTcArgs &a)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t bar_mma, bar_ld, bar_never;
    __shared__ uint32_t tslot;
    const TcLayout &L = a.L;
    const int t = threadIdx.x, ncx = L.ncx, ncy = L.ncy, Np = L.Np, Kx = L.Kx, Ky = L.Ky;
    unsigned char *cA1 = smem + L.cA1, *cA3 = smem + L.cA3, *cB2 = smem + L.cB2, *cB4 = smem + L.cB4;
    const float *sMinv = reinterpret_cast<const float *>(smem + L.minv);
    unsigned char *dA = smem + L.dA, *dB = smem + L.dB;
    const uint32_t idesc = tc::idesc_tf32(128, Np);

    // constants: bulk copies issued by one thread at once, completing on bar_ld
    if (t == 0) {
        tc::mbar_init(&bar_mma, 1);
        tc::mbar_init(&bar_ld, 1);
        tc::mbar_init(&bar_never, 1);         // no thread ever arrives on it
        tc::mbar_expect_tx(&bar_ld, L.cbytes);
        for (uint32_t o = 0; o < L.cbytes; o += CT_CHUNK)
            tc::bulk_g2s(smem + o, a.cst + o, (L.cbytes - o) < CT_CHUNK ? (L.cbytes - o) : CT_CHUNK, &bar_ld);
    }

    // product 1, B = R^T (Np x Ky): four rows k of R per 16-byte store; all
    // loads of a thread are issued before their sums (<= CT_RITEMS items)
    {
        const int nkq = Ky >> 2, nit = Np * nkq;
        float4 v[CT_RITEMS][4];
#pragma unroll
        for (int it = 0; it < CT_RITEMS; ++it) {
            const int i = t + it * CT_THREADS, n = i % Np, k0 = 4 * (i / Np);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int k = k0 + q;
                v[it][q] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (i < nit && n < ncx && k < ncy) {
                    if (FROM_PARTS) v[it][q] = __ldcg(reinterpret_cast<const float4 *>(a.R) + (size_t)k * ncx + n);
                    else v[it][q].x = __ldcg(a.R + (size_t)k * ncx + n);
                }
            }
        }
#pragma unroll
        for (int it = 0; it < CT_RITEMS; ++it) {
            const int i = t + it * CT_THREADS, n = i % Np, k0 = 4 * (i / Np);
            float r[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) r[q] = ((v[it][q].x + v[it][q].y) + v[it][q].z) + v[it][q].w;
            if (i < nit) put4(dB, n, k0, Ky, r[0], r[1], r[2], r[3]);
        }
    }
    if (t < 32) tc::tmem_alloc(&tslot, (uint32_t)a.tcols);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tslot;
    // the constants; under fault_test a phase that nothing completes first
    // (the wait runs out and the failure path below is taken)
    bool ld_done = false;
    if (!a.fault_test) ld_done = tc::mbar_wait(&bar_ld, 0, CT_WAIT_NS);
    ld_done = __syncthreads_and(ld_done) != 0;
    const bool got = a.fault_test ? tc::mbar_wait(&bar_never, 0, CT_WAIT_NS) : ld_done;
    bool ok = __syncthreads_and(got) != 0;
    int pending = -1;                         // parity of MMAs still in flight after a failed wait
    if (ok) ok = run_gemm(cA1, dB, Ky, tmem, idesc, &bar_mma, 0, &pending);

    // product 2: A = T1 (rows l, K = Kx), B = Qx as (n, k) -> Qx[k][n]
    if (ok) {
        read_rows(tmem, Np, [&](int l, int c, const float (&v)[16]) {
#pragma unroll
            for (int q = 0; q < 16; q += 4)
                if (c + q < Kx) put4(dA, l, c + q, Kx, v[q], v[q + 1], v[q + 2], v[q + 3]);
        });
        ok = run_gemm(dA, cB2, Kx, tmem, idesc, &bar_mma, 1, &pending);
    }

    // product 3: A = Qy, B[n][k] = (T2 .* Minv)[k][n]: the rows k < Ky of T2
    // go row-major through a scratch area (row stride Np + 4 floats against
    // bank conflicts), then transposed into B with 16-byte stores, scaled by
    // Minv on the way
    if (ok) {
        float *scr = reinterpret_cast<float *>(smem + L.scr);
        const int SP = Np + 4;
        read_rows(tmem, Np, [&](int l, int c, const float (&v)[16]) {
            if (l < Ky) {
#pragma unroll
                for (int q = 0; q < 16; q += 4)
                    *reinterpret_cast<float4 *>(scr + l * SP + c + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
            }
        });
        __syncthreads();
        for (int i = t; i < Np * (Ky >> 2); i += CT_THREADS) {
            const int n = i % Np, k0 = 4 * (i / Np);
            float s[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int k = k0 + q;
                s[q] = (k < ncy && n < ncx) ? scr[k * SP + n] * sMinv[k * ncx + n] : 0.f;
            }
            put4(dB, n, k0, Ky, s[0], s[1], s[2], s[3]);
        }
        ok = run_gemm(cA3, dB, Ky, tmem, idesc, &bar_mma, 0, &pending);
    }

    // product 4: A = T3 (rows l, K = Kx), B = Qx^T as (n, k) -> Qx[n][k]
    if (ok) {
        read_rows(tmem, Np, [&](int l, int c, const float (&v)[16]) {
#pragma unroll
            for (int q = 0; q < 16; q += 4)
                if (c + q < Kx) put4(dA, l, c + q, Kx, v[q], v[q + 1], v[q + 2], v[q + 3]);
        });
        ok = run_gemm(dA, cB4, Kx, tmem, idesc, &bar_mma, 1, &pending);
    }

    if (ok) {
        read_rows(tmem, Np, [&](int l, int c, const float (&v)[16]) {
            if (l < ncy) {
#pragma unroll
                for (int q = 0; q < 16; q += 4) {
                    if ((ncx & 3) == 0 && c + q + 3 < ncx) {
                        *reinterpret_cast<float4 *>(a.E + l * ncx + c + q) =
                            make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
                    } else {
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            if (c + q + j < ncx) a.E[l * ncx + c + q + j] = v[q + j];
                    }
                }
            }
        });
    } else {
        // a wait ran out: report it, give the bulk copies and the MMAs still
        // in flight a bounded time to finish (their memory is freed below),
        // and leave E untouched
        if (t == 0) atomicExch(&a.st->tc_fail, 1);
        if (!ld_done) tc::mbar_wait(&bar_ld, 0, CT_WAIT_NS);
        if (pending >= 0) tc::mbar_wait(&bar_mma, (uint32_t)pending, CT_WAIT_NS);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (t < 32) tc::tmem_dealloc(tmem, (uint32_t)a.tcols);
    if (ok && a.rcpart) {
        float4 *rp = reinterpret_cast<float4 *>(a.rcpart);
        for (int i = t; i < ncx * ncy; i += CT_THREADS) rp[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (ok && a.consumed && t == 0) *a.consumed = 1;
}

template <bool FROM_PARTS>
__global__ void __launch_bounds__(CT_THREADS, 1) k_coarse_tc(CoarseTcArgs a)
{
    if (a.skip && *a.skip) return;
    coarse_tc_body<FROM_PARTS>(a);
}

// Batched ensemble: one CTA per problem (argument table); problems outside
// an inner solve return at once.
__global__ void __launch_bounds__(CT_THREADS, 1) k_coarse_tc_batch(const CoarseTcArgs *__restrict__ tab)
{
    const CoarseTcArgs a = tab[blockIdx.x];
    if (a.skip && *a.skip) return;
    coarse_tc_body<true>(a);
}

}  // namespace

bool ism_coarse_tc_small(const ism_ctx *ctx)
{
    return ctx->tc_block && ctx->ncx <= CT_MAXC && ctx->ncy <= CT_MAXC;
}

bool ism_coarse_tc_supported(const ism_ctx *ctx)
{
    return ism_coarse_tc_small(ctx) || ctx->tct_block != nullptr;
}

void ism_coarse_tc_prepare()
{
    const TcLayout L = tc_layout(CT_MAXC, CT_MAXC);
    cudaFuncSetAttribute(k_coarse_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.bytes);
    cudaFuncSetAttribute(k_coarse_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.bytes);
    cudaFuncSetAttribute(k_coarse_tc_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.bytes);
    ism_coarse_tct_prepare();
}

static CoarseTcArgs coarse_tc_args(ism_ctx *ctx, const float *rc, float *ec, float *rcpart, const int *skip)
{
    CoarseTcArgs a;
    a.R = rc;
    a.cst = (const unsigned char *)ctx->tc_block;
    a.E = ec;
    a.rcpart = rcpart;
    a.L = tc_layout(ctx->ncx, ctx->ncy);
    a.tcols = a.L.Np <= 32 ? 32 : 64;
    a.skip = skip;
    a.st = ctx->st;
    a.consumed = nullptr;
    a.fault_test = ctx->opt.fault_test;
    return a;
}

ism_status ism_coarse_tc_batch_table(ism_ctx *const *ctxs, int n, void **table, size_t *smem)
{
    std::vector<CoarseTcArgs> t(n);
    size_t sm = 0;
    for (int d = 0; d < n; ++d) {
        ism_ctx *c = ctxs[d];
        if (!ism_coarse_tc_small(c)) return ISM_ERR_ARG;
        t[d] = coarse_tc_args(c, c->rcpart, c->ec32, c->rcpart, &c->st->inner_done);
        t[d].consumed = &c->st->skip_init;
        sm = std::max(sm, (size_t)t[d].L.bytes);
    }
    if (cudaMalloc(table, n * sizeof(CoarseTcArgs)) != cudaSuccess) {
        cudaGetLastError();
        *table = nullptr;
        return ISM_ERR_NOMEM;
    }
    ISM_CUDA_TRY(cudaMemcpy(*table, t.data(), n * sizeof(CoarseTcArgs), cudaMemcpyHostToDevice));
    *smem = sm;
    return ISM_OK;
}

ism_status ism_launch_coarse_tc_batch(cudaStream_t s, const void *table, int n, size_t smem)
{
    k_coarse_tc_batch<<<n, CT_THREADS, smem, s>>>((const CoarseTcArgs *)table);
    return cudaGetLastError() == cudaSuccess ? ISM_OK : ISM_ERR_CUDA;
}

ism_status ism_coarse_tc_upload(ism_ctx *ctx, const std::vector<double> &Qx, const std::vector<double> &QxT,
                                const std::vector<double> &Qy, const std::vector<double> &QyT,
                                const std::vector<double> &Minv)
{
    const int ncx = ctx->ncx, ncy = ctx->ncy;
    const ism_status st = ism_coarse_tct_upload(ctx, Qx, QxT, Qy, QyT);
    if (st != ISM_OK) return st;
    if (ncx > CT_MAXC || ncy > CT_MAXC) return ISM_OK;   // tiled chain (or CUDA cores) only
    const TcLayout L = tc_layout(ncx, ncy);
    std::vector<unsigned char> h(L.cbytes, 0);
    auto put_h = [&](uint32_t base, int row, int k, int K, double v) {
        const uint32_t b = host_tf32((float)v);
        memcpy(h.data() + base + host_kmajor(row, k, K), &b, 4);
    };
    for (int l = 0; l < ncy; ++l)
        for (int k = 0; k < ncy; ++k) {
            put_h(L.cA1, l, k, L.Ky, QyT[(size_t)l * ncy + k]);  // QyT[l][k]
            put_h(L.cA3, l, k, L.Ky, Qy[(size_t)l * ncy + k]);   // Qy[l][k]
        }
    for (int n = 0; n < ncx; ++n)
        for (int k = 0; k < ncx; ++k) {
            put_h(L.cB2, n, k, L.Kx, Qx[(size_t)k * ncx + n]);   // B[n][k] = Qx[k][n]: product T1 Qx
            put_h(L.cB4, n, k, L.Kx, QxT[(size_t)k * ncx + n]);  // B[n][k] = QxT[k][n]: product T3 QxT
        }
    for (size_t i = 0; i < (size_t)ncx * ncy; ++i) {
        const float f = (float)Minv[i];
        memcpy(h.data() + L.minv + 4 * i, &f, 4);
    }
    if (!ctx->tc_block || ctx->tc_bytes != L.cbytes) {
        if (ctx->tc_block) cudaFree(ctx->tc_block);
        ctx->tc_block = nullptr;
        if (cudaMalloc(&ctx->tc_block, L.cbytes) != cudaSuccess) {
            cudaGetLastError();
            ctx->tc_block = nullptr;
            return ISM_ERR_NOMEM;
        }
        ctx->tc_bytes = L.cbytes;
    }
    ISM_CUDA_TRY(cudaMemcpy(ctx->tc_block, h.data(), L.cbytes, cudaMemcpyHostToDevice));
    return ISM_OK;
}

ism_status ism_launch_coarse_tc(ism_ctx *ctx, const float *rc, bool from_parts, float *ec, float *rcpart,
                                const int *skip)
{
    // coarse_tc 1 takes the single-CTA kernel where it fits, 2 the tiled chain always
    if (ctx->opt.coarse_tc == 2 || !ism_coarse_tc_small(ctx))
        return ism_launch_coarse_tct(ctx, rc, from_parts, ec, rcpart, skip);
    const CoarseTcArgs a = coarse_tc_args(ctx, rc, ec, rcpart, skip);
    if (from_parts) k_coarse_tc<true><<<1, CT_THREADS, a.L.bytes, ctx->ws>>>(a);
    else k_coarse_tc<false><<<1, CT_THREADS, a.L.bytes, ctx->ws>>>(a);
    ISM_LAUNCH_CHECK(ctx);
    return ISM_OK;
}
