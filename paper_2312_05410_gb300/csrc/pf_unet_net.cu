// CUDA-core kernels of the time-conditioned U-Net ("U-Net with temporal
// conditioning", Methods), around the tensor-core convolutions of
// pf_unet_conv.cu:
//
//   cond_kernel     the MLP basis f(dt) = w2 sin(w1 sin(w0 dt + b0) + b1) + b2 and the
//                   per-level conditioning factors W_p f(dt), in FP64, stored as BF16 values
//   in_conv_kernel  the first 3x3 convolution (4 -> 32 channels) straight from the DNS
//                   fields (phi, c, rho and a plane holding dt / dt_ref), with its group sums
//   out_conv_kernel the last 3x3 convolution (32 -> 3) as affine increments of the DNS fields
//   gn_stats_kernel group mean and 1/sqrt(var + eps) from the per-tile sums (FP64, fixed order),
//                   folded with gamma and beta into a per-channel affine a x + b
//   gn_apply_*      GN + GELU (+ conditioning product, + 2x2 max pooling) on stored BF16 values
//
// Storage follows the precision model of the reference: every stored activation is BF16
// (round to nearest even), sums are FP32 (FP64 for the statistics), products of BF16 values
// are exact in FP32.
#include <cstdint>

#include "pf_unet_internal.h"
#include "pf_unet_net.h"

namespace pf {
namespace {

constexpr int TPB = 128;  // one 128-pixel tile per block in the tile-shaped kernels

__device__ __forceinline__ float bf(uint16_t h) { return __uint_as_float((uint32_t)h << 16); }

__device__ __forceinline__ uint16_t to_bf(float f)
{
    uint32_t u = __float_as_uint(f);
    if ((u & 0x7f800000u) == 0x7f800000u && (u & 0x007fffffu)) return (uint16_t)((u >> 16) | 0x40);
    u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

__device__ __forceinline__ float rbf(float f) { return bf(to_bf(f)); }

// the paper's tanh form of GELU
__device__ __forceinline__ float gelu(float u)
{
    return 0.5f * u * (1.0f + tanhf(0.7978845608028654f * (u + 0.044715f * u * u * u)));
}

__global__ void cond_kernel(const double* __restrict__ mlp, const double* __restrict__ proj, double tau,
                            float* __restrict__ scales, int nscales)
{
    // mlp: w0[128], b0[128], w1[128][128], b1[128], w2[128][128], b2[128]; proj: [nscales][128]
    __shared__ double h0[UNET_FDIM], h1[UNET_FDIM], f[UNET_FDIM];
    const int k = threadIdx.x;
    const double* w0 = mlp;
    const double* b0 = w0 + UNET_FDIM;
    const double* w1 = b0 + UNET_FDIM;
    const double* b1 = w1 + UNET_FDIM * UNET_FDIM;
    const double* w2 = b1 + UNET_FDIM;
    const double* b2 = w2 + UNET_FDIM * UNET_FDIM;
    asm volatile("griddepcontrol.wait;" ::: "memory");
    h0[k] = sin(w0[k] * tau + b0[k]);
    __syncthreads();
    double s = b1[k];
    for (int j = 0; j < UNET_FDIM; ++j) s += w1[k * UNET_FDIM + j] * h0[j];
    h1[k] = sin(s);
    __syncthreads();
    s = b2[k];
    for (int j = 0; j < UNET_FDIM; ++j) s += w2[k * UNET_FDIM + j] * h1[j];
    f[k] = s;
    __syncthreads();
    for (int i = k; i < nscales; i += UNET_FDIM) {
        double v = 0.0;
        for (int j = 0; j < UNET_FDIM; ++j) v += proj[(size_t)i * UNET_FDIM + j] * f[j];
        scales[i] = rbf((float)v);  // FP64 -> FP32 -> BF16, as the reference stores it
    }
}

// First convolution: x = BF16(phi, c, rho, tau) with zero padding outside the image, 3x3, 4 -> 32.
// One thread per output pixel, one 128-pixel tile per block (neighbours come through L1: staging
// the halo in shared memory measured slower).  Group sums: one warp butterfly over all 16 values.
__global__ void __launch_bounds__(TPB)
in_conv_kernel(const float* const* __restrict__ phi, const float* const* __restrict__ c,
               const float* const* __restrict__ rho, int pitch, int h, int w, float tau,
               const float* __restrict__ wgt /* [36][32]: (ky,kx,ci) x co */, uint16_t* __restrict__ out,
               float* __restrict__ partials)
{
    __shared__ float ws[36 * 32];
    __shared__ float red[4][16];
    asm volatile("griddepcontrol.wait;" ::: "memory");
    for (int i = threadIdx.x; i < 36 * 32; i += TPB) ws[i] = wgt[i];
    __syncthreads();
    const int tpi = h * w / TPB;
    const int img = blockIdx.x / tpi, t = blockIdx.x % tpi;
    const int p = t * TPB + threadIdx.x, y = p / w, x = p % w;
    const float* F = phi[img];
    const float* C = c[img];
    const float* Rh = rho[img];
    const float tb = rbf(tau);
    float acc[32];
#pragma unroll
    for (int o = 0; o < 32; ++o) acc[o] = 0.f;
    for (int ky = 0; ky < 3; ++ky)
        for (int kx = 0; kx < 3; ++kx) {
            const int yy = y + ky - 1, xx = x + kx - 1;
            const bool in = yy >= 0 && yy < h && xx >= 0 && xx < w;
            const size_t o = in ? (size_t)yy * pitch + xx : 0;
            const float v0 = in ? rbf(F[o]) : 0.f;
            const float v1 = in ? rbf(C[o]) : 0.f;
            const float v2 = in ? rbf(Rh[o]) : 0.f;
            const float v3 = in ? tb : 0.f;
            const float* wk = ws + (ky * 3 + kx) * 4 * 32;
#pragma unroll
            for (int q = 0; q < 32; ++q)
                acc[q] = fmaf(v0, wk[q], fmaf(v1, wk[32 + q], fmaf(v2, wk[64 + q], fmaf(v3, wk[96 + q], acc[q]))));
        }
    uint4* dst = reinterpret_cast<uint4*>(out + ((size_t)img * h * w + p) * 32);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        uint32_t pk[4];
#pragma unroll
        for (int j = 0; j < 4; ++j)
            pk[j] = (uint32_t)to_bf(acc[8 * q + 2 * j]) | ((uint32_t)to_bf(acc[8 * q + 2 * j + 1]) << 16);
        dst[q] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    }
    // group sums (8 groups of 4 channels): per thread, then one butterfly per value, then 4 warps
    float sv[16];
#pragma unroll
    for (int g = 0; g < 8; ++g) {
        float s1 = 0.f, s2 = 0.f;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            s1 += acc[4 * g + j];
            s2 = fmaf(acc[4 * g + j], acc[4 * g + j], s2);
        }
        sv[2 * g] = s1;
        sv[2 * g + 1] = s2;
    }
#pragma unroll
    for (int k = 0; k < 16; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sv[k] += __shfl_xor_sync(0xffffffffu, sv[k], o);
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int k = 0; k < 16; ++k) red[threadIdx.x >> 5][k] = sv[k];
    __syncthreads();
    if (threadIdx.x < 16) {
        const int g = threadIdx.x >> 1, which = threadIdx.x & 1;
        partials[(((size_t)img * 8 + g) * tpi + t) * 2 + which] = red[0][threadIdx.x] + red[1][threadIdx.x] + red[2][threadIdx.x] + red[3][threadIdx.x];
    }
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Output: the last convolution (3x3, 32 -> 3) of BF16 NHWC [n][h][w][32], as per-channel affine
// increments added to the FP32 fields in place: u_k += gamma_k conv_k + beta_k for u = (phi, c, rho).
__global__ void __launch_bounds__(TPB)
out_conv_kernel(const uint16_t* __restrict__ in, int h, int w, const float* __restrict__ wgt /* [9][32][3] */,
                const float* __restrict__ gamma, const float* __restrict__ beta, float* const* __restrict__ phi,
                float* const* __restrict__ c, float* const* __restrict__ rho, int pitch)
{
    __shared__ float ws[9 * 32 * 3];
    asm volatile("griddepcontrol.wait;" ::: "memory");
    for (int i = threadIdx.x; i < 9 * 32 * 3; i += TPB) ws[i] = wgt[i];
    __syncthreads();
    const int tpi = h * w / TPB;
    const int img = blockIdx.x / tpi, t = blockIdx.x % tpi;
    const int p = t * TPB + threadIdx.x, y = p / w, x = p % w;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f;
    for (int ky = 0; ky < 3; ++ky)
        for (int kx = 0; kx < 3; ++kx) {
            const int yy = y + ky - 1, xx = x + kx - 1;
            if (yy < 0 || yy >= h || xx < 0 || xx >= w) continue;
            const uint4* src = reinterpret_cast<const uint4*>(in + ((size_t)img * h * w + (size_t)yy * w + xx) * 32);
            const float* wk = ws + (ky * 3 + kx) * 96;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint4 v = src[q];
                const uint32_t u[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int ci = 8 * q + 2 * j;
                    const float lo = bf((uint16_t)(u[j] & 0xffffu)), hi = bf((uint16_t)(u[j] >> 16));
                    a0 = fmaf(lo, wk[3 * ci], fmaf(hi, wk[3 * ci + 3], a0));
                    a1 = fmaf(lo, wk[3 * ci + 1], fmaf(hi, wk[3 * ci + 4], a1));
                    a2 = fmaf(lo, wk[3 * ci + 2], fmaf(hi, wk[3 * ci + 5], a2));
                }
            }
        }
    const size_t o = (size_t)y * pitch + x;
    phi[img][o] = phi[img][o] + fmaf(gamma[0], a0, beta[0]);
    c[img][o] = c[img][o] + fmaf(gamma[1], a1, beta[1]);
    rho[img][o] = rho[img][o] + fmaf(gamma[2], a2, beta[2]);
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Group statistics -> per-channel affine of the normalisation: block (image, group) sums its
// `entries` partial (sum, sum of squares) pairs in FP64 in a fixed order, and writes for every
// channel k of the group affine = (a, b) with a = gamma_k / sqrt(var + eps), b = beta_k - mean a,
// so that GN(x) = a x + b.
__global__ void gn_stats_kernel(const float* __restrict__ partials, int entries, double count, int C, int groups,
                                const float* __restrict__ gamma, const float* __restrict__ beta,
                                float* __restrict__ affine)
{
    __shared__ double r1[TPB], r2[TPB];
    __shared__ float mr[2];
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const float* p = partials + (size_t)blockIdx.x * entries * 2;
    double s1 = 0.0, s2 = 0.0;
    for (int t = threadIdx.x; t < entries; t += TPB) {
        s1 += (double)p[2 * t];
        s2 += (double)p[2 * t + 1];
    }
    r1[threadIdx.x] = s1;
    r2[threadIdx.x] = s2;
    __syncthreads();
    for (int o = TPB / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            r1[threadIdx.x] += r1[threadIdx.x + o];
            r2[threadIdx.x] += r2[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double mean = r1[0] / count;
        double var = r2[0] / count - mean * mean;
        var = var < 0.0 ? 0.0 : var;
        mr[0] = (float)mean;
        mr[1] = (float)(1.0 / sqrt(var + (double)UNET_EPS));
    }
    __syncthreads();
    const int img = blockIdx.x / groups, g = blockIdx.x % groups, cg = C / groups;
    for (int k = threadIdx.x; k < cg; k += TPB) {
        const int ch = g * cg + k;
        const float sc = mr[1] * gamma[ch];
        affine[((size_t)img * C + ch) * 2] = sc;
        affine[((size_t)img * C + ch) * 2 + 1] = fmaf(-mr[0], sc, beta[ch]);
    }
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// (a, b) of 8 consecutive channels: four 16-byte loads
struct Aff8 {
    float a[8], b[8];
};
__device__ __forceinline__ Aff8 aff8(const float* affine, int img, int C, int c0)
{
    Aff8 q;
    const float4* p = reinterpret_cast<const float4*>(affine + ((size_t)img * C + c0) * 2);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float4 v = p[k];
        q.a[2 * k] = v.x;
        q.b[2 * k] = v.y;
        q.a[2 * k + 1] = v.z;
        q.b[2 * k + 1] = v.w;
    }
    return q;
}

__device__ __forceinline__ void unpack8(const uint4 v, float* f)
{
    const uint32_t u[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        f[2 * j] = bf((uint16_t)(u[j] & 0xffffu));
        f[2 * j + 1] = bf((uint16_t)(u[j] >> 16));
    }
}

__device__ __forceinline__ uint4 pack8(const float* f)
{
    uint32_t u[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) u[j] = (uint32_t)to_bf(f[2 * j]) | ((uint32_t)to_bf(f[2 * j + 1]) << 16);
    return make_uint4(u[0], u[1], u[2], u[3]);
}

// Encoder level: z = BF16(GELU(GN(x))); zc = BF16(z * s) into the skip slice (channels [0, C) of a
// buffer with cat_stride channels); pool (if not NULL) = 2x2 max of z.  One thread per 8 channels
// of a 2x2 pixel block (pool) or of one pixel (no pool).
__global__ void gn_apply_enc_kernel(const uint16_t* __restrict__ x, int n, int h, int w, int C,
                                    const float* __restrict__ affine, const float* __restrict__ scale,
                                    uint16_t* __restrict__ cat, int cat_stride, uint16_t* __restrict__ pool)
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int c8 = C / 8;
    const int ph = pool ? h / 2 : h, pw = pool ? w / 2 : w;
    const long long total = (long long)n * ph * pw * c8;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int cb = (int)(i % c8);
        long long r = i / c8;
        const int px = (int)(r % pw);
        r /= pw;
        const int py = (int)(r % ph);
        const int img = (int)(r / ph);
        const Aff8 q = aff8(affine, img, C, cb * 8);
        float s[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) s[j] = scale[cb * 8 + j];
        float mx[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) mx[j] = -INFINITY;
        const int nsub = pool ? 4 : 1;
        for (int sidx = 0; sidx < nsub; ++sidx) {
            const int yy = pool ? 2 * py + (sidx >> 1) : py, xx = pool ? 2 * px + (sidx & 1) : px;
            const size_t pix = ((size_t)img * h + yy) * w + xx;
            float v[8], z[8], zc[8];
            unpack8(reinterpret_cast<const uint4*>(x + pix * C)[cb], v);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                z[j] = rbf(gelu(fmaf(v[j], q.a[j], q.b[j])));
                zc[j] = z[j] * s[j];
                mx[j] = fmaxf(mx[j], z[j]);
            }
            reinterpret_cast<uint4*>(cat + pix * cat_stride)[cb] = pack8(zc);
        }
        if (pool) reinterpret_cast<uint4*>(pool + (((size_t)img * ph + py) * pw + px) * C)[cb] = pack8(mx);
    }
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Decoder level: y = BF16(GELU(GN(x))), NHWC with C channels.
__global__ void gn_apply_dec_kernel(const uint16_t* __restrict__ x, long long pixels, int C, int hw,
                                    const float* __restrict__ affine, uint16_t* __restrict__ y)
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int c8 = C / 8;
    const long long total = pixels * c8;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int cb = (int)(i % c8);
        const long long pix = i / c8;
        const int img = (int)(pix / hw);
        const Aff8 q = aff8(affine, img, C, cb * 8);
        float v[8];
        unpack8(reinterpret_cast<const uint4*>(x + pix * C)[cb], v);
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = gelu(fmaf(v[j], q.a[j], q.b[j]));
        reinterpret_cast<uint4*>(y + pix * C)[cb] = pack8(v);
    }
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Plausibility of a predicted state: every phi, c and rho finite and inside its range; flags[img]
// is set to 1 on a violation (flags are cleared by the caller).
__global__ void check_kernel(const float* const* __restrict__ phi, const float* const* __restrict__ c,
                             const float* const* __restrict__ rho, int h, int w, int pitch, float phi_lo, float phi_hi,
                             float c_lo, float c_hi, float r_lo, float r_hi, int* __restrict__ flags)
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int img = blockIdx.y;
    const float* F = phi[img];
    const float* C = c[img];
    const float* Rh = rho[img];
    int bad = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < h * w; i += gridDim.x * blockDim.x) {
        const size_t o = (size_t)(i / w) * pitch + i % w;
        const float f = F[o], cc = C[o], r = Rh[o];
        // written so that NaN fails every comparison
        bad |= !(f >= phi_lo && f <= phi_hi && cc >= c_lo && cc <= c_hi && r >= r_lo && r <= r_hi);
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&flags[img], 1);
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

cudaLaunchConfig_t cfg_of(dim3 grid, int threads, cudaStream_t s, cudaLaunchAttribute* attr)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(threads);
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

unsigned grid_for(long long items, int threads)
{
    long long b = (items + threads - 1) / threads;
    return (unsigned)(b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : b));
}

}  // namespace

cudaError_t launch_cond(const double* mlp, const double* proj, double tau, float* scales, int nscales, cudaStream_t s)
{
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = cfg_of(dim3(1), UNET_FDIM, s, attr);
    return cudaLaunchKernelEx(&cfg, cond_kernel, mlp, proj, tau, scales, nscales);
}

cudaError_t launch_in_conv(const float* const* phi, const float* const* c, const float* const* rho, int pitch, int n,
                           int h, int w, float tau, const float* wgt, uint16_t* out, float* partials, cudaStream_t s)
{
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = cfg_of(dim3((unsigned)(n * (h * w / TPB))), TPB, s, attr);
    return cudaLaunchKernelEx(&cfg, in_conv_kernel, phi, c, rho, pitch, h, w, tau, wgt, out, partials);
}

cudaError_t launch_out_conv(const uint16_t* in, int n, int h, int w, const float* wgt, const float* gamma,
                            const float* beta, float* const* phi, float* const* c, float* const* rho, int pitch,
                            cudaStream_t s)
{
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = cfg_of(dim3((unsigned)(n * (h * w / TPB))), TPB, s, attr);
    return cudaLaunchKernelEx(&cfg, out_conv_kernel, in, h, w, wgt, gamma, beta, phi, c, rho, pitch);
}

cudaError_t launch_gn_stats(const float* partials, int n, int groups, int entries, double count, int C,
                            const float* gamma, const float* beta, float* affine, cudaStream_t s)
{
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = cfg_of(dim3((unsigned)(n * groups)), TPB, s, attr);
    return cudaLaunchKernelEx(&cfg, gn_stats_kernel, partials, entries, count, C, groups, gamma, beta, affine);
}

cudaError_t launch_gn_enc(const uint16_t* x, int n, int h, int w, int C, const float* affine, const float* scale,
                          uint16_t* cat, int cat_stride, uint16_t* pool, cudaStream_t s)
{
    const long long items = (long long)n * (pool ? (h / 2) * (w / 2) : h * w) * (C / 8);
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = cfg_of(dim3(grid_for(items, 256)), 256, s, attr);
    return cudaLaunchKernelEx(&cfg, gn_apply_enc_kernel, x, n, h, w, C, affine, scale, cat, cat_stride, pool);
}

cudaError_t launch_gn_dec(const uint16_t* x, int n, int h, int w, int C, const float* affine, uint16_t* y,
                          cudaStream_t s)
{
    const long long pixels = (long long)n * h * w;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = cfg_of(dim3(grid_for(pixels * (C / 8), 256)), 256, s, attr);
    return cudaLaunchKernelEx(&cfg, gn_apply_dec_kernel, x, pixels, C, h * w, affine, y);
}

cudaError_t launch_check(const float* const* phi, const float* const* c, const float* const* rho, int n, int h, int w,
                         int pitch, float phi_lo, float phi_hi, float c_lo, float c_hi, float r_lo, float r_hi,
                         int* flags, cudaStream_t s)
{
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = cfg_of(dim3(32, (unsigned)n), 256, s, attr);
    return cudaLaunchKernelEx(&cfg, check_kernel, phi, c, rho, h, w, pitch, phi_lo, phi_hi, c_lo, c_hi, r_lo, r_hi,
                              flags);
}

}  // namespace pf
