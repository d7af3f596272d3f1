// Two-point autocorrelation S2 of the solid A phase, the statistical error metric the paper
// judges the hybrid solver by ("Autocorrelations" in Results, "Error metrics" in Methods).
// A cell is solid A when phi > 0 and c > 0.5 (FP32 decisions); counts(r) = sum_x I(x) I(x + r)
// with periodic shifts, for |rx|, |ry| <= R.  Integer arithmetic: the counts are exact and the
// result does not depend on the summation order.
#include <cstdint>

#include "pf.h"

namespace {

__global__ void s2_indicator_kernel(const float* __restrict__ phi, const float* __restrict__ c, int nx, int ny,
                                    int pitch, uint8_t* __restrict__ ind)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nx * ny; i += gridDim.x * blockDim.x) {
        const size_t o = (size_t)(i / nx) * pitch + i % nx;
        ind[i] = (phi[o] > 0.0f && c[o] > 0.5f) ? 1 : 0;
    }
}

// Block ry + R: thread rx + R counts the pairs at offset (rx, ry).  The indicator is staged in
// shared memory when it fits (smem_ok), else read through L1.
__global__ void s2_count_kernel(const uint8_t* __restrict__ ind, int nx, int ny, int R, int smem_ok,
                                long long* __restrict__ counts)
{
    extern __shared__ uint8_t s[];
    const int n = nx * ny;
    const uint8_t* I = ind;
    if (smem_ok) {
        for (int i = threadIdx.x; i < n; i += blockDim.x) s[i] = ind[i];
        __syncthreads();
        I = s;
    }
    const int ry = (int)blockIdx.x - R, rx = (int)threadIdx.x - R;
    if (threadIdx.x > 2 * R) return;
    const int dy = ((ry % ny) + ny) % ny, dx = ((rx % nx) + nx) % nx;
    long long cnt = 0;
    for (int y = 0; y < ny; ++y) {
        const uint8_t* a = I + (size_t)y * nx;
        const uint8_t* b = I + (size_t)((y + dy) % ny) * nx;
        int x = 0;
        for (; x + dx < nx; ++x) cnt += a[x] & b[x + dx];
        for (; x < nx; ++x) cnt += a[x] & b[x + dx - nx];
    }
    counts[(size_t)blockIdx.x * (2 * R + 1) + threadIdx.x] = cnt;
}

}  // namespace

extern "C" int pf_s2_counts(const float* phi, const float* c, int nx, int ny, int pitch, int R,
                            unsigned char* scratch, long long* counts, void* stream)
{
    if (!phi || !c || !scratch || !counts) return PF_ERR_ARG;
    if (nx < 1 || ny < 1 || nx > (1 << 14) || ny > (1 << 14) || pitch < nx) return PF_ERR_ARG;
    if (R < 0 || R > 127 || 2 * R + 1 > nx || 2 * R + 1 > ny) return PF_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int n = nx * ny;
    s2_indicator_kernel<<<(n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024, 256, 0, s>>>(phi, c, nx, ny, pitch, scratch);
    const int smem_ok = n <= 200 * 1024;
    const size_t smem = smem_ok ? (size_t)n : 0;
    if (smem_ok && cudaFuncSetAttribute(s2_count_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
                       cudaSuccess)
        return PF_ERR_CUDA;
    const int threads = ((2 * R + 1 + 31) / 32) * 32;
    s2_count_kernel<<<2 * R + 1, threads, smem, s>>>(scratch, nx, ny, R, smem_ok, counts);
    return cudaGetLastError() == cudaSuccess ? PF_OK : PF_ERR_CUDA;
}
