// Allocation-free variant of the diagnostics entry point (pf_diagnostics_static).
//
// Who needs it: code that may not allocate device memory itself, for example
// a plug-in inside a host application that owns every device byte through its
// own pool allocator (a raw cudaMalloc would bypass the pool's accounting and
// its memory cap), or a latency-critical loop where cudaMalloc/cudaFree would
// synchronise the device.  Such a caller still passes its own fields and
// output buffer, but it cannot hand over the reduction workspace that
// pf_diagnostics takes.
//
// The workspace lives instead in one file-scope device array below.  Every GPU
// that loads this library holds it (about 39 KB) until the process exits.
// Host code must not pass the array's name to a kernel: on the host that name
// is only a stand-in for the device object.  Its device address is looked up
// with cudaGetSymbolAddress, with the caller's device current, on every call
// made outside a stream capture; the address is also remembered per device
// together with the CUDA context it belongs to.  A call made while `stream`
// is being captured uses the remembered address of the same context, so the
// first call on each device (and the first after a cudaDeviceReset, which
// makes a new context in which the array may sit elsewhere) should come
// before any stream capture.  All calls share the one array, so calls whose
// work overlaps on the GPU (different streams, no ordering between them) race
// on it.  No call allocates: there is no cudaMalloc, cudaFree or allocating
// library routine on this path.
#include <cudaTypedefs.h>

#include <cstdint>
#include <mutex>

#include "pf.h"
#include "pf_internal.h"

namespace {

// Capacity: per-block partials of 4 sums for the most reduction blocks the
// diagnostics pass ever launches, then the error word in its own 256 bytes.
constexpr int STATIC_DIAG_BLOCKS = pf::DIAG_MAX_BLOCKS;
constexpr size_t PARTIAL_DOUBLES = 4 * size_t(STATIC_DIAG_BLOCKS);
constexpr size_t SCRATCH_DOUBLES = PARTIAL_DOUBLES + 32;
static_assert(STATIC_DIAG_BLOCKS >= pf::DIAG_MAX_BLOCKS, "static scratch must hold every accepted grid");
static_assert((PARTIAL_DOUBLES * sizeof(double)) % 256 == 0, "error word on its own 256-byte line");

static __device__ __align__(256) double g_diag_scratch[SCRATCH_DOUBLES];

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mutex;
struct Cached {
    CUcontext ctx;
    double* ptr;
};
Cached g_cache[MAX_DEVICES] = {};

// The current context through the runtime's driver entry point (no link to libcuda).
cudaError_t current_context(CUcontext* ctx)
{
    static const PFN_cuCtxGetCurrent_v4000 get = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 4000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return (PFN_cuCtxGetCurrent_v4000) nullptr;
        return reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(f);
    }();
    if (!get) return cudaErrorNotSupported;
    return get(ctx) == CUDA_SUCCESS ? cudaSuccess : cudaErrorDeviceUninitialized;
}

// Device address of the scratch array in the current device's context.
cudaError_t scratch_address(cudaStream_t s, double** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    CUcontext ctx = nullptr;
    e = current_context(&ctx);
    if (e != cudaSuccess) return e;
    if (cap == cudaStreamCaptureStatusNone || g_cache[dev].ctx != ctx || !g_cache[dev].ptr) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_diag_scratch);
        if (e != cudaSuccess) return e;
        g_cache[dev].ctx = ctx;
        g_cache[dev].ptr = static_cast<double*>(p);
    }
    *out = g_cache[dev].ptr;
    return cudaSuccess;
}

}  // namespace

extern "C" {

int pf_diagnostics_static(const pf_params* p, int nx, int ny, int pitch, const float* phi, const float* c,
                          const float* rho, double* out_dev, int* err_dev, void* stream)
{
    if (!p || !phi || !c || !rho || !out_dev) return pf::fail(PF_ERR_ARG, "null pointer");
    if (!(p->dx > 0.0)) return pf::fail(PF_ERR_ARG, "dx must be positive");
    int rc = pf::check_sizes(nx, ny, pitch);
    if (rc) return rc;
    if (reinterpret_cast<uintptr_t>(out_dev) % 8 != 0) return pf::fail(PF_ERR_LAYOUT, "out_dev must be 8-byte aligned");

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double* scratch = nullptr;
    cudaError_t e = scratch_address(s, &scratch);
    if (e != cudaSuccess) return pf::cuda_fail(e, "static scratch address");
    int* err_word = reinterpret_cast<int*>(scratch + PARTIAL_DOUBLES);

    // The partials are fully rewritten by every call; only the error word must start at zero.
    e = cudaMemsetAsync(err_word, 0, sizeof(int), s);
    if (e != cudaSuccess) return pf::cuda_fail(e, "clear static error word");
    e = pf::launch_diag(pf::diag_const_of(*p, nx, ny, pitch), phi, c, rho, scratch, err_word, out_dev, nullptr, 0, s);
    if (e != cudaSuccess) return pf::cuda_fail(e, "diagnostic launch");
    if (err_dev) {
        e = cudaMemcpyAsync(err_dev, err_word, sizeof(int), cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return pf::cuda_fail(e, "error word copy");
    }
    return PF_OK;
}

}  // extern "C"
