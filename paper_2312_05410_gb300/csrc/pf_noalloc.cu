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
// is only a stand-in for the device object.  The first call on each device
// looks up the array's device address with cudaGetSymbolAddress (with that
// device current) and caches it; that first call should therefore come before
// any stream capture.  All calls share the one array, so calls whose work
// overlaps on the GPU (different streams, no ordering between them) race on
// it.  No call allocates: there is no cudaMalloc, cudaFree or allocating
// library routine on this path.
#include <cstdint>
#include <mutex>

#include "pf.h"
#include "pf_internal.h"

namespace {

// Capacity: per-block partials of 4 sums for up to PF_STATIC_DIAG_BLOCKS
// reduction blocks (the most the diagnostics reduction ever launches), then the
// error word.
constexpr int PF_STATIC_DIAG_BLOCKS = 1216;
constexpr size_t PARTIAL_DOUBLES = 4 * size_t(PF_STATIC_DIAG_BLOCKS);
constexpr size_t SCRATCH_DOUBLES = PARTIAL_DOUBLES + 32;  // + 256 bytes holding the error word

static __device__ __align__(256) double g_diag_scratch[SCRATCH_DOUBLES];

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mutex;
double* g_scratch_ptr[MAX_DEVICES] = {};

// Device address of the scratch array on the current device (set-up on first use).
cudaError_t scratch_on_current_device(double** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_diag_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

// Errors are returned as codes only (pf_strerror gives their text).
int reject(int code, const char*) { return code; }

}  // namespace

extern "C" {

int pf_diagnostics_static(const pf_params* p, int nx, int ny, int pitch, const float* phi, const float* c,
                          const float* rho, double* out_dev, int* err_dev, void* stream)
{
    if (!p || !phi || !c || !rho || !out_dev) return reject(PF_ERR_ARG, "null pointer");
    if (!(p->dx > 0.0)) return reject(PF_ERR_ARG, "dx must be positive");
    if (nx < 1 || ny < 1) return reject(PF_ERR_ARG, "empty grid");
    if (nx > (1 << 20) || ny > (1 << 20)) return reject(PF_ERR_ARG, "grid side above 1048576");
    if (pitch < nx || pitch % 4 != 0) return reject(PF_ERR_LAYOUT, "pitch must be >= nx and a multiple of 4");
    if (reinterpret_cast<uintptr_t>(out_dev) % 8 != 0) return reject(PF_ERR_LAYOUT, "out_dev must be 8-byte aligned");
    if (pf::diag_blocks(nx, ny) > PF_STATIC_DIAG_BLOCKS)
        return reject(PF_ERR_LAYOUT, "grid needs more reduction blocks than the static scratch holds");

    double* scratch = nullptr;
    cudaError_t e = scratch_on_current_device(&scratch);
    if (e != cudaSuccess) return reject(PF_ERR_CUDA, cudaGetErrorString(e));
    int* err_word = reinterpret_cast<int*>(scratch + PARTIAL_DOUBLES);
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    // The partials are fully rewritten by every call; only the error word must start at zero.
    e = cudaMemsetAsync(err_word, 0, sizeof(int), s);
    if (e != cudaSuccess) return reject(PF_ERR_CUDA, cudaGetErrorString(e));

    pf::DiagConst d{};
    d.nx = nx;
    d.ny = ny;
    d.pitch = pitch;
    d.Wc = float(p->W_c);
    d.Wf = float(p->W_phi);
    d.area = p->dx * p->dx;
    d.hkf = 0.5 * p->kappa_phi;
    d.hkc = 0.5 * p->kappa_c;
    e = pf::launch_diag(d, phi, c, rho, scratch, err_word, out_dev, nullptr, 0, s);
    if (e != cudaSuccess) return reject(PF_ERR_CUDA, cudaGetErrorString(e));
    if (err_dev) {
        e = cudaMemcpyAsync(err_dev, err_word, sizeof(int), cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return reject(PF_ERR_CUDA, cudaGetErrorString(e));
    }
    return PF_OK;
}

}  // extern "C"
