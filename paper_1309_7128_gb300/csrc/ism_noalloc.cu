// ism_noalloc.cu -- residual + restriction without any allocation.
//
// Some callers cannot allocate device memory at the moment they need a
// residual: real-time loops that cannot take the implicit device
// synchronisation of cudaMalloc / cudaFree, and hosts that hand all device
// memory to their own arena and forbid allocations outside it.  A context
// (ism_setup) allocates its workspaces, so those callers use this entry
// point instead: it needs no context, and its only scratch -- the per-block
// partial sums of the norm reduction -- lives in a fixed array compiled into
// the library.
#include <cuda.h>

#include <mutex>

#include "ism_kernels.cuh"

// Largest coarse grid (ny/m)*(nx/m) the entry point accepts.
#define ISM_NOALLOC_MAX_COARSE 32768

// Per-block partial sums (||r||^2, sum p, sum p^2), q-major, for up to
// ISM_NOALLOC_MAX_COARSE blocks: 768 KiB, held by every GPU that loads the
// library until the process exits.  Shared by all calls.
static __device__ __align__(256) double g_noalloc_scratch[3 * ISM_NOALLOC_MAX_COARSE];

// One CTA: fixed-order sums of the partials into norms[0] = ||b - A_f p||_2
// and norms[1] = sum p.
__global__ void k_noalloc_norms(const double *partials, int nblk, double *norms)
{
    __shared__ double S[ISM_NQ];
    ctl_reduce(partials, nblk, 2, S);
    if (threadIdx.x == 0) {
        norms[0] = sqrt(S[0]);
        norms[1] = S[1];
    }
}

namespace {
std::mutex g_scratch_mu;
constexpr int kMaxDevices = 64;
// Per device: the address of the array and the id of the CUDA context it
// was looked up in.  A device reset (cudaDeviceReset, or the primary
// context released and re-created) unloads the module with the array; the
// next call then runs in a context with a new id and looks the address up
// again instead of reusing a stale one.
struct ScratchSlot {
    unsigned long long ctx_id;
    double *ptr;
};
ScratchSlot g_scratch[kMaxDevices] = {};

// Driver entry points for the id of the current context, fetched through
// the runtime so that the library does not link the driver library.
typedef CUresult (*PFN_ctxGetCurrent)(CUcontext *);
typedef CUresult (*PFN_ctxGetId)(CUcontext, unsigned long long *);
PFN_ctxGetCurrent g_ctx_get_current = nullptr;
PFN_ctxGetId g_ctx_get_id = nullptr;
bool g_entry_points_tried = false;

// Id of the context current on this thread; false when there is none yet
// or the driver does not offer the query.
bool current_ctx_id(unsigned long long *id)
{
    if (!g_entry_points_tried) {
        g_entry_points_tried = true;
        void *f = nullptr, *g = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &g, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess) {
            g_ctx_get_current = (PFN_ctxGetCurrent)f;
            g_ctx_get_id = (PFN_ctxGetId)g;
        }
        cudaGetLastError();
    }
    if (!g_ctx_get_current || !g_ctx_get_id) return false;
    CUcontext ctx = nullptr;
    if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
    return g_ctx_get_id(ctx, id) == CUDA_SUCCESS;
}
}  // namespace

// Device address of the scratch array in the current device's context.  In
// host code the name g_noalloc_scratch is only a stand-in for the symbol,
// not a device address, so the address is looked up with the device
// current: once per device and context (the first call on a device, and the
// first call after that device's context was re-created).
static ism_status scratch_address(double **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return ISM_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    unsigned long long id = 0;
    const bool have_id = current_ctx_id(&id);
    ScratchSlot &slot = g_scratch[dev];
    if (!slot.ptr || !have_id || slot.ctx_id != id) {
        void *ptr = nullptr;
        // also makes the device's primary context current when none was
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
            cudaGetLastError();
            return ISM_ERR_CUDA;
        }
        unsigned long long id2 = 0;
        // without the id query the address cannot be validated on a later
        // call, so the slot stays empty and every call looks it up again
        const bool known = current_ctx_id(&id2);
        slot.ptr = known ? (double *)ptr : nullptr;
        slot.ctx_id = known ? id2 : 0;
        *out = (double *)ptr;
        return ISM_OK;
    }
    *out = slot.ptr;
    return ISM_OK;
}

extern "C" ism_status ism_residual_restrict_noalloc(int nx, int ny, int coarsen, const int bc[4],
                                                    const double *p, const double *b, double *rc,
                                                    double *norms, void *stream)
{
    if (!bc || !p || !b || !rc || !norms) return ISM_ERR_ARG;
    if (coarsen != 8 && coarsen != 16 && coarsen != 32) return ISM_ERR_ARG;
    if (nx <= 0 || ny <= 0) return ISM_ERR_ARG;
    const int ncx = (nx + coarsen - 1) / coarsen, ncy = (ny + coarsen - 1) / coarsen;   // last cell may be narrower
    if ((long long)ncx * ncy > ISM_NOALLOC_MAX_COARSE) return ISM_ERR_ARG;
    const int bcmask = ism_bc_mask(bc);
    if (bcmask < 0) return ISM_ERR_ARG;
    double *scratch = nullptr;
    ism_status s = scratch_address(&scratch);
    if (s != ISM_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    // every partial read below is written by k_resid in the same call, so
    // nothing in the scratch array has to be cleared first
    const int th = coarsen * coarsen < 256 ? coarsen * coarsen : 256;
    k_resid<double><<<dim3(ncx, ncy), th, 0, st>>>(p, b, rc, scratch, nx, ny, coarsen, bcmask, nullptr);
    if (cudaGetLastError() != cudaSuccess) return ISM_ERR_CUDA;
    k_noalloc_norms<<<1, 256, 0, st>>>(scratch, ncx * ncy, norms);
    if (cudaGetLastError() != cudaSuccess) return ISM_ERR_CUDA;
    return ISM_OK;
}
