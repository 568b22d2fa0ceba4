// ism_noalloc.cu -- residual + restriction without any allocation.
//
// Some callers cannot allocate device memory at the time they need a
// residual: code that is recording a CUDA stream capture (a cudaMalloc there
// breaks the capture), real-time loops that cannot afford the implicit device
// synchronisation of cudaMalloc / cudaFree, and hosts that hand all device
// memory to their own arena and forbid allocations outside it.  A context
// (ism_setup) allocates its workspaces, so those callers use this entry
// point instead: it needs no context, and its only scratch -- the per-block
// partial sums of the norm reduction -- lives in a fixed array compiled into
// the library.
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
double *g_scratch_ptr[kMaxDevices] = {nullptr};
}  // namespace

// Device address of the scratch array on the current device.  The host-side
// name g_noalloc_scratch is only a stand-in for the symbol, not a device
// address, so the address is looked up once per device.
static ism_status scratch_address(double **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return ISM_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
            cudaGetLastError();
            return ISM_ERR_CUDA;
        }
        g_scratch_ptr[dev] = (double *)ptr;
    }
    *out = g_scratch_ptr[dev];
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
