// Mass and free-energy diagnostics of one state (dx^2 sum c, dx^2 sum phi,
// dx^2 sum rho, F_h) with a NaN/Inf check.
//
// F_h is the discrete free energy whose gradient the step's chemical
// potentials are (composition Cahn-Hilliard equation and order-parameter
// equation, Materials and Methods): dx^2 sum f(phi, c) + kappa_phi/2
// sum_faces (dphi)^2 + kappa_c/2 sum_faces (dc)^2, over every x face (periodic)
// and every interior y face.  Per-cell terms are FP32; every sum is FP64.
//
// Pass 1: a fixed grid of blocks, each summing a fixed grid-stride subset of
// cells, warp-shuffle butterfly then a fixed order across warps -> one FP64
// partial per block and quantity.  Pass 2: one block sums the partials in a
// fixed order.  The result is therefore bitwise reproducible run to run.
#include "pf_internal.h"

namespace pf {
namespace {

constexpr int DIAG_THREADS = 256;

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Deterministic block sum of 4 values; result valid in thread 0.
__device__ __forceinline__ void block_sum4(double v[4], double (*red)[DIAG_THREADS / 32])
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        v[q] = warp_sum(v[q]);
        if (lane == 0) red[q][w] = v[q];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            double s = 0.0;
            for (int i = 0; i < DIAG_THREADS / 32; ++i) s += red[q][i];
            v[q] = s;
        }
    }
}

__global__ void __launch_bounds__(DIAG_THREADS)
diag_partials(const DiagConst d, const float* __restrict__ phi, const float* __restrict__ c,
              const float* __restrict__ rho, double* __restrict__ partials, int* __restrict__ err)
{
    __shared__ double red[4][DIAG_THREADS / 32];
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    const long long n = (long long)d.nx * d.ny;
    bool bad = false;
    for (long long idx = (long long)blockIdx.x * DIAG_THREADS + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * DIAG_THREADS) {
        const int j = (int)(idx / d.nx), i = (int)(idx - (long long)j * d.nx);
        const size_t o = (size_t)j * d.pitch + i;
        const size_t oe = (size_t)j * d.pitch + (i + 1 == d.nx ? 0 : i + 1);
        const float f = phi[o], cc = c[o], r = rho[o];
        bad |= !(isfinite(f) && isfinite(cc) && isfinite(r));
        const float w = 1.f - f * f;
        const float q = cc * (1.f - cc);
        const float p = 0.25f * (2.f - f) * (1.f + f) * (1.f + f);
        const float dens = 0.25f * d.Wf * w * w + p * d.Wc * q * q;
        float dfe = phi[oe] - f, dce = c[oe] - cc;
        double grad_f = (double)(dfe * dfe), grad_c = (double)(dce * dce);
        if (j + 1 < d.ny) {
            const size_t on = o + d.pitch;
            const float dfn = phi[on] - f, dcn = c[on] - cc;
            grad_f += (double)(dfn * dfn);
            grad_c += (double)(dcn * dcn);
        }
        acc[0] += (double)cc;
        acc[1] += (double)f;
        acc[2] += (double)r;
        acc[3] += d.area * (double)dens + d.hkf * grad_f + d.hkc * grad_c;
    }
    if (bad) atomicOr(err, 1);
    block_sum4(acc, red);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < 4; ++q) partials[(size_t)q * gridDim.x + blockIdx.x] = acc[q];
    }
}

// hist: [0] = record count, [1] = step of the next record, [2] = capacity (as long long),
// followed by capacity records of 5 doubles. A NULL hist records nothing.
__global__ void __launch_bounds__(DIAG_THREADS)
diag_final(const double* __restrict__ partials, int nblocks, double area, int* __restrict__ err,
           double* __restrict__ out, long long* __restrict__ hist, long long step_stride)
{
    __shared__ double red[4][DIAG_THREADS / 32];
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblocks; b += DIAG_THREADS) {
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] += partials[(size_t)q * nblocks + b];
    }
    block_sum4(acc, red);
    if (threadIdx.x == 0) {
        const double v[4] = {area * acc[0], area * acc[1], area * acc[2], acc[3]};
        bool bad = false;
        for (int q = 0; q < 4; ++q) bad |= !isfinite(v[q]);
        if (bad) atomicOr(err, 1);
        if (out)
            for (int q = 0; q < 4; ++q) out[q] = v[q];
        if (hist) {
            const long long cnt = hist[0], cap = hist[2];
            double* rec = reinterpret_cast<double*>(hist + 3) + 5 * (cnt % cap);
            rec[0] = (double)hist[1];
            for (int q = 0; q < 4; ++q) rec[1 + q] = v[q];
            hist[0] = cnt + 1;
            hist[1] += step_stride;
        }
    }
}

__global__ void reset_kernel(long long* hist, long long capacity, long long next_step, int* err)
{
    if (hist) {
        hist[0] = 0;
        hist[1] = next_step;
        hist[2] = capacity;
    }
    if (err) *err = 0;
}

}  // namespace

cudaError_t launch_reset(long long* hist, long long capacity, long long next_step, int* err, cudaStream_t s)
{
    reset_kernel<<<1, 1, 0, s>>>(hist, capacity, next_step, err);
    return cudaGetLastError();
}

int diag_blocks(int nx, int ny)
{
    const long long n = (long long)nx * ny;
    long long b = (n + 4 * DIAG_THREADS - 1) / (4 * DIAG_THREADS);
    if (b < 1) b = 1;
    if (b > DIAG_MAX_BLOCKS) b = DIAG_MAX_BLOCKS;
    return (int)b;
}

cudaError_t launch_diag(const DiagConst& d, const float* phi, const float* c, const float* rho,
                        double* partials, int* err, double* out, long long* hist, long long step_stride,
                        cudaStream_t s)
{
    const int nb = diag_blocks(d.nx, d.ny);
    diag_partials<<<nb, DIAG_THREADS, 0, s>>>(d, phi, c, rho, partials, err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    diag_final<<<1, DIAG_THREADS, 0, s>>>(partials, nb, d.area, err, out, hist, step_stride);
    return cudaGetLastError();
}

}  // namespace pf
