// Implicit-GEMM convolutions of the time-conditioned U-Net on the tcgen05
// tensor cores ("U-Net with temporal conditioning": the 3x3 convolution of each
// conv_block and the stride-2 transposed convolution of the up-sampling path).
//
// GEMM view.  M = 128 output pixels of one image (a run of 128 pixels of a row,
// or 128/W whole rows when the image is narrower than 128), N = output channels
// (<= 256), K = taps x input channels.  Activations are NHWC BF16 and the weights
// are [tap][Cout][Cin] BF16, so both operands are K-major.  For each tap and each
// block of KC input channels, TMA copies one box of the activation tensor,
// shifted by the tap offset, into shared memory.  Its out-of-range rows and
// columns are zero-filled, and that zero fill is the convolution's zero padding.
// The weights of that tap and channel block come in a second box.  One thread
// issues KC/16 tcgen05.mma (kind::f16, BF16 x BF16 -> FP32) per stage into an
// accumulator of 128 lanes x N columns in tensor memory.  Four epilogue warps
// then read it back with tcgen05.ld.
//
// Pipeline: a persistent CTA per SM walks its tiles.  Warp 0 produces (TMA), warp
// 1 allocates tensor memory and issues the MMAs, warps 2-5 run the epilogue; ST
// shared-memory stages with full/empty mbarriers carry the stream across tiles
// without draining, and two accumulators (2 N columns of tensor memory) let the
// epilogue of one tile overlap the MMAs of the next.  Every wait is bounded: a wait
// that runs out sets the error word, and the CTA drains what it issued (bounded
// again) and frees its tensor memory.  The N tile is a template parameter, so the
// epilogue's loops unroll and its group indices are compile-time constants.
//
// Epilogues: CONV3 stores the raw convolution (BF16, into a channel slice of an
// NHWC buffer) and, per 32-pixel quarter of each tile, the sums of the FP32
// values and of their squares per normalisation group; TCONV scatters each input
// pixel's 4 x Cout outputs to the 2x2 block of output pixels it feeds.
#include <cstdint>
#include <cstring>

#include "pf_unet_internal.h"

namespace pf {
namespace {

constexpr int TM = 128;          // pixels per tile (MMA M)
constexpr int NTHREADS = 192;    // 6 warps
constexpr int MAX_ST = 8;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                 : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    return ok != 0;
}

// Bounded wait on a phase of an mbarrier; false if it ran out (or the CTA is aborting).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int cap, volatile int* abort_flag)
{
    for (int it = 0; it < cap; ++it) {
        if (mbar_try(bar, parity)) return true;
        if ((it & 255) == 255 && *abort_flag) return false;
    }
    return false;
}

// The same for waiters with nothing else to do (the epilogue between tiles): back off between
// polls so that they leave the issue slots to the producer and MMA threads of their schedulers.
__device__ __forceinline__ bool mbar_wait_sleep(uint32_t bar, uint32_t parity, int cap, volatile int* abort_flag)
{
    for (int it = 0; it < cap; ++it) {
        if (mbar_try(bar, parity)) return true;
        if ((it & 63) == 63 && *abort_flag) return false;
        __nanosleep(64);
    }
    return false;
}

// Shared-memory matrix descriptor of a K-major operand tile with 128-byte (KC = 64) or
// 64-byte (KC = 32) swizzling: rows of KC BF16, 8-row swizzle atoms SBO bytes apart.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, int kc)
{
    const uint64_t sbo = kc == 64 ? 1024 : 512;
    const uint64_t layout = kc == 64 ? 2 : 4;  // SWIZZLE_128B : SWIZZLE_64B
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)1 << 16;             // leading byte offset (unused for swizzled K-major)
    d |= (sbo >> 4) << 32;              // stride byte offset: next 8-row group
    d |= (uint64_t)1 << 46;             // descriptor version of this architecture
    d |= layout << 61;
    return d;
}

// Instruction descriptor: D FP32, A and B BF16, both K-major, M = 128, N = n.
__device__ __forceinline__ uint32_t umma_idesc(int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}


// Round to nearest even, as the oracle's format definition does.
__device__ __forceinline__ uint16_t f_to_bf16(float f)
{
    uint32_t u = __float_as_uint(f);
    if ((u & 0x7f800000u) == 0x7f800000u && (u & 0x007fffffu)) return (uint16_t)((u >> 16) | 0x40);  // NaN stays NaN
    u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

// Tile geometry: tile T of a launch -> image, first pixel (x0, y0) and first GEMM column n0.
struct TileGeo {
    int img, t, x0, y0, n0;
};

__device__ __forceinline__ TileGeo tile_geo(const ConvArgs& a, int T, int mtiles, int NT)
{
    TileGeo g;
    const int mt = T % mtiles, nt = T / mtiles;
    const int tpi = (a.h * a.w) / TM;
    const int BW = a.w < TM ? a.w : TM, BR = TM / BW, tiles_per_row = a.w / BW;
    g.img = mt / tpi;
    g.t = mt % tpi;
    g.y0 = (g.t / tiles_per_row) * BR;
    g.x0 = (g.t % tiles_per_row) * BW;
    g.n0 = nt * NT;
    return g;
}

// Persistent kernel: CTA b takes tiles b, b + gridDim.x, ...  The TMA / MMA stream runs through
// all of them without draining; two accumulators in tensor memory let the epilogue of one tile
// overlap the MMAs of the next.
template <int MODE, int NT>
__global__ void __launch_bounds__(NTHREADS, 1)
umma_conv_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, ConvArgs a)
{
    extern __shared__ __align__(1024) uint8_t smraw[];
    uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
    __shared__ __align__(8) uint64_t full_bar[MAX_ST], empty_bar[MAX_ST], accf_bar[2], acce_bar[2];
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int abort_flag;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int KC = a.kc, ST = a.stages;
    const uint32_t a_bytes = TM * KC * 2, b_bytes = NT * KC * 2, stage_bytes = a_bytes + b_bytes;
    const int kblocks = a.cin / KC, ntaps = MODE == CONV3 ? 9 : 1, iters = ntaps * kblocks;
    const int ncols = MODE == CONV3 ? a.cout : 4 * a.cout;
    const int mtiles = a.n * ((a.h * a.w) / TM), tiles = mtiles * (ncols / NT);
    const int tpi = (a.h * a.w) / TM;
    const int BW = a.w < TM ? a.w : TM;

    if (tid == 0) {
        abort_flag = 0;
        for (int s = 0; s < ST; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full_bar[s])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty_bar[s])) : "memory");
        }
        for (int b = 0; b < 2; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&accf_bar[b])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(smem_u32(&acce_bar[b])) : "memory");
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {  // the whole warp allocates both accumulators (2 NT columns)
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(&tmem_slot)), "r"(a.tmem_cols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    asm volatile("griddepcontrol.wait;" ::: "memory");

    if (warp == 0) {
        if (lane == 0) {  // ---- producer: a continuous stream of (tile, tap, channel block) stages
            int it = 0;  // stage counter over all tiles
            bool ok = true;
            for (int T = blockIdx.x; T < tiles && ok; T += gridDim.x) {
                const TileGeo g = tile_geo(a, T, mtiles, NT);
                for (int k = 0; k < iters && ok; ++k, ++it) {
                    const int s = it % ST;
                    ok = mbar_wait(smem_u32(&empty_bar[s]), ((uint32_t)(it / ST) & 1u) ^ 1u, a.wait_cap, &abort_flag);
                    if (!ok) break;
                    const int tap = k / kblocks, kb = k % kblocks;
                    const int dy = MODE == CONV3 ? tap / 3 - 1 : 0, dx = MODE == CONV3 ? tap % 3 - 1 : 0;
                    const uint32_t fb = smem_u32(&full_bar[s]);
                    const uint32_t sa = smem_u32(sm + (size_t)s * stage_bytes), sb = sa + a_bytes;
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(stage_bytes)
                                 : "memory");
                    asm volatile(
                        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(sa),
                        "l"(reinterpret_cast<uint64_t>(&tmA)), "r"(kb * KC), "r"(g.x0 + dx), "r"(g.y0 + dy),
                        "r"(g.img), "r"(fb)
                        : "memory");
                    asm volatile(
                        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(sb),
                        "l"(reinterpret_cast<uint64_t>(&tmB)), "r"(kb * KC), "r"(g.n0), "r"(tap), "r"(fb)
                        : "memory");
                }
            }
            if (!ok) {
                abort_flag = 1;
                atomicOr(a.err, UNET_ERR_TIMEOUT);
                // let the copies already issued land before the CTA leaves (bounded)
                for (int j = (it > ST ? it - ST : 0); j < it; ++j)
                    mbar_wait(smem_u32(&full_bar[j % ST]), (uint32_t)(j / ST) & 1u, a.wait_cap, &abort_flag);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {  // ---- MMA issuer
            const uint32_t idesc = umma_idesc(NT);
            int it = 0, local = 0;
            bool ok = true;
            for (int T = blockIdx.x; T < tiles && ok; T += gridDim.x, ++local) {
                const int b = local & 1;
                // the epilogue must have drained this accumulator (its previous use)
                ok = mbar_wait(smem_u32(&acce_bar[b]), ((uint32_t)(local >> 1) & 1u) ^ 1u, a.wait_cap, &abort_flag);
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t d = tmem + (uint32_t)(b * NT);
                for (int k = 0; k < iters && ok; ++k, ++it) {
                    const int s = it % ST;
                    ok = mbar_wait(smem_u32(&full_bar[s]), (uint32_t)(it / ST) & 1u, a.wait_cap, &abort_flag);
                    if (!ok) break;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t sa = smem_u32(sm + (size_t)s * stage_bytes), sb = sa + a_bytes;
                    for (int kk = 0; kk < KC / 16; ++kk) {
                        const uint64_t ad = umma_desc(sa + kk * 32, KC), bd = umma_desc(sb + kk * 32, KC);
                        const uint32_t acc = (k | kk) ? 1u : 0u;
                        asm volatile(
                            "{ .reg .pred p; setp.ne.b32 p, %4, 0;\n"
                            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(d),
                            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                            : "memory");
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                                 ::"r"(smem_u32(&empty_bar[s])) : "memory");
                }
                if (!ok) break;
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                             ::"r"(smem_u32(&accf_bar[b])) : "memory");
            }
            if (!ok) {
                abort_flag = 1;
                atomicOr(a.err, UNET_ERR_TIMEOUT);
            }
        }
    } else {  // ---- epilogue, warps 2..5: TMEM lanes 32 (warp % 4) ... + 31
        const int q = warp & 3;
        const int row = q * 32 + lane;  // pixel within the tile
        int local = 0;
        for (int T = blockIdx.x; T < tiles; T += gridDim.x, ++local) {
            const int b = local & 1;
            if (!mbar_wait_sleep(smem_u32(&accf_bar[b]), (uint32_t)(local >> 1) & 1u, a.wait_cap, &abort_flag)) {
                abort_flag = 1;
                if (lane == 0) atomicOr(a.err, UNET_ERR_TIMEOUT);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const TileGeo g = tile_geo(a, T, mtiles, NT);
            const int py = g.y0 + row / BW, px = g.x0 + row % BW;
            float s1[GN_MAX_GROUPS], s2[GN_MAX_GROUPS];
#pragma unroll
            for (int gg = 0; gg < GN_MAX_GROUPS; ++gg) s1[gg] = s2[gg] = 0.f;
#pragma unroll
            for (int c0 = 0; c0 < NT; c0 += 16) {
                uint32_t r[16];
                const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * NT + c0);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15},"
                    " [%16];"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                      "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                      "=r"(r[14]), "=r"(r[15])
                    : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                uint32_t pk[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float v0 = __uint_as_float(r[2 * j]), v1 = __uint_as_float(r[2 * j + 1]);
                    pk[j] = (uint32_t)f_to_bf16(v0) | ((uint32_t)f_to_bf16(v1) << 16);
                }
                uint16_t* dst;
                if (MODE == CONV3) {
                    constexpr int cg = NT / GN_MAX_GROUPS;  // channels per group (one N tile holds all Cout)
#pragma unroll
                    for (int j = 0; j < 16; ++j) {  // the group index is a compile-time constant
                        const float v = __uint_as_float(r[j]);
                        s1[(c0 + j) / cg] += v;
                        s2[(c0 + j) / cg] = fmaf(v, v, s2[(c0 + j) / cg]);
                    }
                    dst = a.out + ((size_t)(g.img * a.h + py) * a.w + px) * a.out_cstride + a.out_coff + c0;
                } else {  // TCONV: column n0 + c0 + j = sub-pixel s * cout + channel
                    const int col = g.n0 + c0, s = col / a.cout, co = col % a.cout;
                    const int oy = 2 * py + (s >> 1), ox = 2 * px + (s & 1);
                    dst = a.out + ((size_t)(g.img * 2 * a.h + oy) * (2 * a.w) + ox) * a.out_cstride + a.out_coff + co;
                }
                uint4* d4 = reinterpret_cast<uint4*>(dst);
                d4[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                d4[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
            }
            // the accumulator is drained: hand it back to the MMA issuer (one arrival per warp)
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0)
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acce_bar[b])) : "memory");
            if (MODE == CONV3 && a.partials) {
                // per warp: partials[((img * groups + g) * tpi + t) * 4 + q] = (sum, sum of squares)
#pragma unroll
                for (int gg = 0; gg < GN_MAX_GROUPS; ++gg) {
                    float v1 = s1[gg], v2 = s2[gg];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        v1 += __shfl_xor_sync(0xffffffffu, v1, o);
                        v2 += __shfl_xor_sync(0xffffffffu, v2, o);
                    }
                    if (lane == 0) {
                        float* pp = a.partials + ((((size_t)g.img * a.groups + gg) * tpi + g.t) * 4 + q) * 2;
                        pp[0] = v1;
                        pp[1] = v2;
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols)
                     : "memory");
    }
}

}  // namespace

namespace {

int conv_kc(int cin) { return cin % 64 == 0 ? 64 : 32; }

int sm_count()
{
    static int n = 0;
    if (!n) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
            n = 1;
    }
    return n;
}

int conv_nt(int mode, int cout) { return mode == CONV3 ? cout : (4 * cout < 256 ? 4 * cout : 256); }

int conv_stages(int kc, int nt)
{
    const int stage = TM * kc * 2 + nt * kc * 2;
    int st = (200 * 1024) / stage;
    return st < 2 ? 2 : (st > MAX_ST ? MAX_ST : st);
}

bool encode(CUtensorMap* m, const void* base, int rank, const cuuint64_t* dims, const cuuint64_t* strides,
            const cuuint32_t* box, int kc)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    cuuint32_t elem[4] = {1u, 1u, 1u, 1u};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, (cuuint32_t)rank, const_cast<void*>(base), dims, strides, box,
               elem, CU_TENSOR_MAP_INTERLEAVE_NONE,
               kc == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

size_t umma_conv_smem_bytes(int mode, int cin, int cout)
{
    const int kc = conv_kc(cin), nt = conv_nt(mode, cout);
    return (size_t)conv_stages(kc, nt) * (size_t)(TM * kc * 2 + nt * kc * 2) + 1024;
}

cudaError_t launch_umma_conv(int mode, const uint16_t* in, const uint16_t* wgt, ConvArgs a, cudaStream_t s)
{
    if (a.cin % 32 || a.cout % 16 || a.cout < 16 || a.n < 1 || a.h < 1 || a.w < 1) return cudaErrorInvalidValue;
    if ((a.w % TM) && (TM % a.w)) return cudaErrorInvalidValue;
    if (((long long)a.h * a.w) % TM) return cudaErrorInvalidValue;
    if (mode == CONV3 && ((a.cout != 32 && a.cout != 64 && a.cout != 128 && a.cout != 256) || a.groups != GN_MAX_GROUPS))
        return cudaErrorInvalidValue;
    if (mode == TCONV && a.cout != 16 && a.cout != 32 && a.cout != 64 && a.cout != 128) return cudaErrorInvalidValue;
    if (a.out_coff % 8 || a.out_cstride % 8) return cudaErrorInvalidValue;  // 16-byte vector stores
    const int ncols = mode == CONV3 ? a.cout : 4 * a.cout;
    a.kc = conv_kc(a.cin);
    a.nt = conv_nt(mode, a.cout);
    if (ncols % a.nt) return cudaErrorInvalidValue;
    a.stages = conv_stages(a.kc, a.nt);
    a.tmem_cols = 32;
    while (a.tmem_cols < 2 * a.nt) a.tmem_cols <<= 1;  // two accumulators
    const int BW = a.w < TM ? a.w : TM, BR = TM / BW;

    CUtensorMap mA, mB;
    const cuuint64_t dA[4] = {(cuuint64_t)a.cin, (cuuint64_t)a.w, (cuuint64_t)a.h, (cuuint64_t)a.n};
    const cuuint64_t sA[3] = {(cuuint64_t)a.cin * 2, (cuuint64_t)a.w * a.cin * 2, (cuuint64_t)a.h * a.w * a.cin * 2};
    const cuuint32_t bA[4] = {(cuuint32_t)a.kc, (cuuint32_t)BW, (cuuint32_t)BR, 1u};
    const int taps = mode == CONV3 ? 9 : 1;
    const cuuint64_t dB[3] = {(cuuint64_t)a.cin, (cuuint64_t)ncols, (cuuint64_t)taps};
    const cuuint64_t sB[2] = {(cuuint64_t)a.cin * 2, (cuuint64_t)ncols * a.cin * 2};
    const cuuint32_t bB[3] = {(cuuint32_t)a.kc, (cuuint32_t)a.nt, 1u};
    if (!encode(&mA, in, 4, dA, sA, bA, a.kc) || !encode(&mB, wgt, 3, dB, sB, bB, a.kc))
        return cudaErrorInvalidValue;

    const size_t smem = umma_conv_smem_bytes(mode, a.cin, a.cout);
    cudaLaunchConfig_t cfg = {};
    const long long tiles = (long long)a.n * a.h * a.w / TM * (ncols / a.nt);
    int per_sm = (int)((227 * 1024) / (smem + 2048));  // CTAs that fit next to each other on an SM
    per_sm = per_sm < 1 ? 1 : (per_sm > 2 ? 2 : per_sm);
    if (per_sm * a.tmem_cols > 512) per_sm = 512 / a.tmem_cols;
    const long long slots = (long long)sm_count() * per_sm;
    cfg.gridDim = dim3((unsigned)(tiles < slots ? tiles : slots));
    cfg.blockDim = dim3(NTHREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    auto go = [&](auto kern) -> cudaError_t {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        return cudaLaunchKernelEx(&cfg, kern, mA, mB, a);
    };
    if (mode == CONV3) {
        if (a.nt == 32) return go(umma_conv_kernel<CONV3, 32>);
        if (a.nt == 64) return go(umma_conv_kernel<CONV3, 64>);
        if (a.nt == 128) return go(umma_conv_kernel<CONV3, 128>);
        if (a.nt == 256) return go(umma_conv_kernel<CONV3, 256>);
        return cudaErrorInvalidValue;
    }
    if (a.nt == 64) return go(umma_conv_kernel<TCONV, 64>);
    if (a.nt == 128) return go(umma_conv_kernel<TCONV, 128>);
    if (a.nt == 256) return go(umma_conv_kernel<TCONV, 256>);
    return cudaErrorInvalidValue;
}

}  // namespace pf
