// CUDA-core kernels of the time-conditioned U-Net ("U-Net with temporal
// conditioning", Methods), around the tensor-core convolutions of
// pf_unet_conv.cu:
//
//   cond_kernel     the MLP basis f(dt) = w2 sin(w1 sin(w0 dt + b0) + b1) + b2 and the
//                   per-level conditioning factors W_p f(dt), in FP64, stored as BF16 values
//   in_conv_kernel  the first 3x3 convolution (4 -> 32 channels) straight from the DNS
//                   fields (phi, c, rho and a plane holding dt / dt_ref), with its group sums
//   gn_stats_kernel group mean and 1/sqrt(var + eps) from the per-tile sums (FP32, fixed order),
//                   folded with gamma and beta into a per-channel affine a x + b
//   gn_apply_*      GN + GELU (+ conditioning product, + 2x2 max pooling) on stored BF16 values
// (the last convolution, 32 -> 3, runs on the tensor cores: OUT3 mode of pf_unet_conv.cu)
//
// Storage follows the precision model of the reference: every stored activation is BF16
// (round to nearest even), sums are FP32, products of BF16 values are exact in FP32.
#include <cstdint>

#include "pf_unet_internal.h"
#include "pf_unet_net.h"

namespace pf {
namespace {

constexpr int TPB = 128;  // one 128-pixel tile per block in the tile-shaped kernels

__device__ __forceinline__ float bf(uint16_t h) { return __uint_as_float((uint32_t)h << 16); }

// FP32 -> BF16, round to nearest even: one conversion instruction each
__device__ __forceinline__ uint16_t to_bf(float f)
{
    uint16_t h;
    asm("cvt.rn.bf16.f32 %0, %1;" : "=h"(h) : "f"(f));
    return h;
}

__device__ __forceinline__ uint32_t to_bf2(float lo, float hi)
{
    uint32_t d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}

__device__ __forceinline__ float rbf(float f) { return bf(to_bf(f)); }

// the paper's tanh form of GELU, with the hardware tanh (tanh.approx.f32, relative error about
// 2^-11: a sixteenth of the BF16 spacing that every GELU output is rounded to)
__device__ __forceinline__ float tanh_hw(float x)
{
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float gelu(float u)
{
    return 0.5f * u * (1.0f + tanh_hw(0.7978845608028654f * (u + 0.044715f * u * u * u)));
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

// eight BF16 values (one 16-byte load) to FP32
__device__ __forceinline__ void unpack8(const uint4 v, float* f)
{
    const uint32_t u[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        f[2 * j] = bf((uint16_t)(u[j] & 0xffffu));
        f[2 * j + 1] = bf((uint16_t)(u[j] >> 16));
    }
}

// First convolution over the look-back input, 3x3, 10 -> 32, zero padding outside the image:
// x = (phi, c, rho) of the oldest frame, of the middle frame, of the current fields, then the tau
// plane, all in FP32 with FP32 weights (the composition fluctuations that seed the spinodal pattern
// are about 0.01 on c ~ 0.5, a few BF16 units: BF16 inputs would quantize them away).  The two
// older frames are FP32 planes [image][3][h][w] (old0, old1; either may be NULL: that frame is the
// current fields, the history of a run that has none yet).  The output is stored as BF16.
// A block covers two consecutive 128-pixel tiles of one image; thread t computes pixel t of each
// (neighbours come through L1: staging the halo in shared memory measured slower).  The 32 outputs
// are 16 pairs updated by packed FP32x2 FMAs, and each weight pair read from shared memory serves
// both pixels.  Group sums: one scatter-halving per warp and tile.
constexpr int IN_CH = UNET_IN;
static_assert(IN_CH == 10, "three frames of (phi, c, rho) and the tau plane");
__global__ void __launch_bounds__(TPB)
in_conv_kernel(const float* const* __restrict__ phi, const float* const* __restrict__ c,
               const float* const* __restrict__ rho, int pitch, const float* __restrict__ old0,
               const float* __restrict__ old1, int h, int w, float tau,
               const float* __restrict__ wgt /* [9 * IN_CH][32]: (ky,kx,ci) x co */, uint16_t* __restrict__ out,
               float* __restrict__ partials)
{
    __shared__ __align__(16) float ws[9 * IN_CH * 32];
    __shared__ float red[2][4][16];
    asm volatile("griddepcontrol.wait;" ::: "memory");
    for (int i = threadIdx.x; i < 9 * IN_CH * 32; i += TPB) ws[i] = wgt[i];
    __syncthreads();
    const int tpi = h * w / TPB, bpi = (tpi + 1) / 2;  // tiles and blocks per image
    const int img = blockIdx.x / bpi, t0 = 2 * (blockIdx.x % bpi);
    const bool two = t0 + 1 < tpi;
    const float* F = phi[img];
    const float* C = c[img];
    const float* Rh = rho[img];
    const size_t plane = (size_t)h * w;
    const float* O0 = old0 ? old0 + (size_t)img * 3 * plane : nullptr;
    const float* O1 = old1 ? old1 + (size_t)img * 3 * plane : nullptr;
    const float tb = tau;
    int y[2], x[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int p = (t0 + k) * TPB + threadIdx.x;
        y[k] = p / w;
        x[k] = p % w;
    }
    float2 acc[2][16];
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int o = 0; o < 16; ++o) acc[k][o] = make_float2(0.f, 0.f);
    for (int ky = 0; ky < 3; ++ky)
        for (int kx = 0; kx < 3; ++kx) {
            float v[2][IN_CH];
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const int yy = y[k] + ky - 1, xx = x[k] + kx - 1;
                const bool in = (k == 0 || two) && yy >= 0 && yy < h && xx >= 0 && xx < w;
                const size_t o = in ? (size_t)yy * pitch + xx : 0;
                const size_t ob = in ? (size_t)yy * w + xx : 0;
                const float f0 = in ? F[o] : 0.f, f1 = in ? C[o] : 0.f, f2 = in ? Rh[o] : 0.f;
                v[k][6] = f0;
                v[k][7] = f1;
                v[k][8] = f2;
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    v[k][q] = in ? (O0 ? O0[q * plane + ob] : v[k][6 + q]) : 0.f;
                    v[k][3 + q] = in ? (O1 ? O1[q * plane + ob] : v[k][6 + q]) : 0.f;
                }
                v[k][9] = in ? tb : 0.f;
            }
            const float4* wk = reinterpret_cast<const float4*>(ws + (ky * 3 + kx) * IN_CH * 32);
#pragma unroll
            for (int ci = 0; ci < IN_CH; ++ci) {
                const float2 b0 = make_float2(v[0][ci], v[0][ci]), b1 = make_float2(v[1][ci], v[1][ci]);
#pragma unroll
                for (int q2 = 0; q2 < 8; ++q2) {  // two output pairs per 16-byte weight load
                    const float4 wv = wk[ci * 8 + q2];
                    const float2 wa = make_float2(wv.x, wv.y), wb = make_float2(wv.z, wv.w);
                    acc[0][2 * q2] = __ffma2_rn(b0, wa, acc[0][2 * q2]);
                    acc[0][2 * q2 + 1] = __ffma2_rn(b0, wb, acc[0][2 * q2 + 1]);
                    acc[1][2 * q2] = __ffma2_rn(b1, wa, acc[1][2 * q2]);
                    acc[1][2 * q2 + 1] = __ffma2_rn(b1, wb, acc[1][2 * q2 + 1]);
                }
            }
        }
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        if (k == 1 && !two) break;
        uint4* dst = reinterpret_cast<uint4*>(out + ((size_t)img * h * w + (size_t)(t0 + k) * TPB + threadIdx.x) * 32);
#pragma unroll
        for (int q = 0; q < 4; ++q)
            dst[q] = make_uint4(to_bf2(acc[k][4 * q].x, acc[k][4 * q].y), to_bf2(acc[k][4 * q + 1].x, acc[k][4 * q + 1].y),
                                to_bf2(acc[k][4 * q + 2].x, acc[k][4 * q + 2].y),
                                to_bf2(acc[k][4 * q + 3].x, acc[k][4 * q + 3].y));
        // group sums (8 groups of 4 channels): value 2 g + j is the sum (j = 0) or the sum of squares (j = 1)
        float sv[16];
#pragma unroll
        for (int g = 0; g < 8; ++g) {
            const float2 a0 = acc[k][2 * g], a1 = acc[k][2 * g + 1];
            sv[2 * g] = (a0.x + a0.y) + (a1.x + a1.y);
            sv[2 * g + 1] = fmaf(a1.y, a1.y, fmaf(a1.x, a1.x, fmaf(a0.y, a0.y, a0.x * a0.x)));
        }
        const float tot = warp_sum_scatter<16>(sv, lane);  // even lane l: value l / 2
        if (!(lane & 1)) red[k][threadIdx.x >> 5][lane >> 1] = tot;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        const int k = threadIdx.x >> 4, i = threadIdx.x & 15;
        if (k == 0 || two) {
            const int g = i >> 1, which = i & 1;
            partials[(((size_t)img * 8 + g) * tpi + t0 + k) * 2 + which] =
                red[k][0][i] + red[k][1][i] + red[k][2][i] + red[k][3][i];
        }
    }
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// One look-back frame: the FP32 fields (row pitch `pitch`) of every image copied to dense FP32
// planes [image][3][h][w].
__global__ void frame_kernel(const float* const* __restrict__ phi, const float* const* __restrict__ c,
                             const float* const* __restrict__ rho, int pitch, int n, int h, int w,
                             float* __restrict__ dst)
{
    const size_t plane = (size_t)h * w, total = (size_t)n * 3 * plane;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int img = (int)(i / (3 * plane));
        const size_t r = i - (size_t)img * 3 * plane;
        const int q = (int)(r / plane);
        const size_t pix = r - (size_t)q * plane;
        const int yy = (int)(pix / w), xx = (int)(pix - (size_t)yy * w);
        const float* src = q == 0 ? phi[img] : (q == 1 ? c[img] : rho[img]);
        dst[i] = src[(size_t)yy * pitch + xx];
    }
}

// Group statistics -> per-channel affine of the normalisation: block (image, group) sums its
// `entries` partial (sum, sum of squares) pairs in a fixed order, and writes for every
// channel k of the group affine = (a, b) with a = gamma_k / sqrt(var + eps), b = beta_k - mean a,
// so that GN(x) = a x + b.
__global__ void gn_stats_kernel(const float* __restrict__ partials, int entries, double count, int C, int groups,
                                const float* __restrict__ gamma, const float* __restrict__ beta,
                                float* __restrict__ affine)
{
    // FP32 throughout, in a fixed order (strided per thread, warp butterfly, warps in order): the partial
    // sums are FP32 already, and the FP64 pipe of this part is slow enough to make the FP64 form the
    // latency of the whole kernel.  Relative error ~1e-6 in the moments, far below the BF16 output.
    __shared__ float r1[TPB / 32], r2[TPB / 32];
    __shared__ float mr[2];
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const float* p = partials + (size_t)blockIdx.x * entries * 2;
    float s1 = 0.f, s2 = 0.f;
    for (int t = threadIdx.x; t < entries; t += TPB) {
        const float2 v = reinterpret_cast<const float2*>(p)[t];
        s1 += v.x;
        s2 += v.y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        r1[threadIdx.x >> 5] = s1;
        r2[threadIdx.x >> 5] = s2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float t1 = 0.f, t2 = 0.f;
        for (int w = 0; w < TPB / 32; ++w) {
            t1 += r1[w];
            t2 += r2[w];
        }
        const float inv = (float)(1.0 / count);
        const float mean = t1 * inv;
        float var = fmaf(t2, inv, -mean * mean);
        var = var < 0.f ? 0.f : var;
        mr[0] = mean;
        mr[1] = 1.0f / sqrtf(var + UNET_EPS);
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

__device__ __forceinline__ uint4 pack8(const float* f)
{
    uint32_t u[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) u[j] = to_bf2(f[2 * j], f[2 * j + 1]);
    return make_uint4(u[0], u[1], u[2], u[3]);
}

// Encoder level: z = BF16(GELU(GN(x))); zc = BF16(z * s) into the skip slice (channels [0, C) of a
// buffer with cat_stride channels); pool (if not NULL) = 2x2 max of z.  One thread per 8 channels
// of a 2x2 pixel block (pool) or of one pixel (no pool).  Blocks in y walk the rows of (pooled)
// pixels, blocks in x the (pixel, 8-channel block) items of a row; C / 8 = 1 << lc8.
__global__ void gn_apply_enc_kernel(const uint16_t* __restrict__ x, int n, int h, int w, int C, int lc8,
                                    const float* __restrict__ affine, const float* __restrict__ scale,
                                    uint16_t* __restrict__ cat, int cat_stride, uint16_t* __restrict__ pool)
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int ph = pool ? h / 2 : h, pw = pool ? w / 2 : w;
    const int rows = n * ph, per_row = pw << lc8;
    for (int row = blockIdx.y; row < rows; row += gridDim.y)
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < per_row; i += gridDim.x * blockDim.x) {
        const int img = row / ph, py = row - img * ph;
        const int cb = i & ((1 << lc8) - 1), px = i >> lc8;
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

// Decoder level: y = BF16(GELU(GN(x))), NHWC with C channels; rows and items as in the encoder.
__global__ void gn_apply_dec_kernel(const uint16_t* __restrict__ x, int n, int h, int w, int C, int lc8,
                                    const float* __restrict__ affine, uint16_t* __restrict__ y)
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int rows = n * h, per_row = w << lc8;
    for (int row = blockIdx.y; row < rows; row += gridDim.y)
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < per_row; i += gridDim.x * blockDim.x) {
        const int img = row / h;
        const int cb = i & ((1 << lc8) - 1);
        const size_t pix = (size_t)row * w + (i >> lc8);
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

// Row-wise grid of the normalisation kernels: x covers one row's items, y the rows (at most 65535).
dim3 row_grid(int rows, long long per_row, int threads)
{
    const long long bx = (per_row + threads - 1) / threads;
    return dim3((unsigned)(bx < 1 ? 1 : (bx > 1024 ? 1024 : bx)), (unsigned)(rows < 65535 ? rows : 65535));
}

// log2 of C / 8, or -1 unless C / 8 is a power of two
int log2_c8(int C)
{
    if (C < 8 || C % 8) return -1;
    int l = 0;
    while ((8 << l) < C) ++l;
    return (8 << l) == C ? l : -1;
}

}  // namespace

cudaError_t launch_cond(const double* mlp, const double* proj, double tau, float* scales, int nscales, cudaStream_t s)
{
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = cfg_of(dim3(1), UNET_FDIM, s, attr);
    return cudaLaunchKernelEx(&cfg, cond_kernel, mlp, proj, tau, scales, nscales);
}

cudaError_t launch_in_conv(const float* const* phi, const float* const* c, const float* const* rho, int pitch,
                           const float* old0, const float* old1, int n, int h, int w, float tau,
                           const float* wgt, uint16_t* out, float* partials, cudaStream_t s)
{
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = cfg_of(dim3((unsigned)(n * ((h * w / TPB + 1) / 2))), TPB, s, attr);
    return cudaLaunchKernelEx(&cfg, in_conv_kernel, phi, c, rho, pitch, old0, old1, h, w, tau, wgt, out, partials);
}

cudaError_t launch_frame(const float* const* phi, const float* const* c, const float* const* rho, int pitch, int n,
                         int h, int w, float* dst, cudaStream_t s)
{
    const size_t total = (size_t)n * 3 * h * w;
    const unsigned blocks = (unsigned)((total + 255) / 256 < 152 * 16 ? (total + 255) / 256 : 152 * 16);
    frame_kernel<<<blocks, 256, 0, s>>>(phi, c, rho, pitch, n, h, w, dst);
    return cudaGetLastError();
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
    const int lc8 = log2_c8(C);
    if (lc8 < 0) return cudaErrorInvalidValue;
    const int rows = n * (pool ? h / 2 : h), per_row = (pool ? w / 2 : w) << lc8;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = cfg_of(row_grid(rows, per_row, 256), 256, s, attr);
    return cudaLaunchKernelEx(&cfg, gn_apply_enc_kernel, x, n, h, w, C, lc8, affine, scale, cat, cat_stride, pool);
}

cudaError_t launch_gn_dec(const uint16_t* x, int n, int h, int w, int C, const float* affine, uint16_t* y,
                          cudaStream_t s)
{
    const int lc8 = log2_c8(C);
    if (lc8 < 0) return cudaErrorInvalidValue;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = cfg_of(row_grid(n * h, (long long)w << lc8, 256), 256, s, attr);
    return cudaLaunchKernelEx(&cfg, gn_apply_dec_kernel, x, n, h, w, C, lc8, affine, y);
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
