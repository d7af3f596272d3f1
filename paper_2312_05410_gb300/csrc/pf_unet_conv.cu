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
// Halo form (3x3 convolutions of 32, 64 or 128 channels on rows that are whole tiles): one box of
// 3 rows x 130 pixels per channel block serves all nine taps as shifted windows, and the weights
// of the CTA's column tile stay resident for the whole launch (see halo_box below).
//
// Epilogues: CONV3 stores the raw convolution (BF16, into a channel slice of an
// NHWC buffer) and, per 32-pixel quarter of each tile, the sums of the FP32
// values and of their squares per normalisation group; TCONV scatters each input
// pixel's 4 x Cout outputs to the 2x2 block of output pixels it feeds; OUT3 adds
// gamma x (its first three columns) + beta to three FP32 fields in place.
#include <cstdint>
#include <cstring>

#include "pf_unet_internal.h"

namespace pf {
namespace {

constexpr int TM = 128;          // pixels per tile (MMA M)
constexpr int EPI_WARPS = 4;     // epilogue warps: EPI_WARPS / 4 per TMEM lane quarter, each on a share of the N columns
constexpr int NTHREADS = 64 + 32 * EPI_WARPS;  // producer warp, MMA warp, epilogue warps
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

// Halo form (3x3, 32, 64 or 128 input channels, rows that are whole 128-pixel tiles): per channel
// block, a tile's three input rows of 130 pixels (the 128 of the tile and one on each side) arrive
// in ONE box; tap (dy, dx) is the 128-row window starting at row (dy + 1) * 130 + dx + 1 of it.
// TMA and the MMA both apply the 128- or 64-byte swizzle as a function of the absolute shared-
// memory address (the copy starts on a 1024-byte boundary), so a window that starts at any row
// takes a plain descriptor with base offset 0.  The weights of the CTA's column tile, all taps,
// stay resident in shared memory for the whole launch.
constexpr int HALO_W = TM + 2;
// Bytes of a tile's box with channel blocks of kc (rows of 2 kc bytes), and the stage stride
// (1024-byte aligned, a whole number of swizzle atoms of either width).
__host__ __device__ constexpr uint32_t halo_box(int kc) { return 3u * HALO_W * 2u * (uint32_t)kc; }
__host__ __device__ constexpr uint32_t halo_stage(int kc) { return (halo_box(kc) + 1023u) & ~1023u; }

// Instruction descriptor: D FP32, A and B BF16, both K-major, M = 128, N = n.
__device__ __forceinline__ uint32_t umma_idesc(int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}


// Round to nearest even, as the oracle's format definition does.
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi)
{
    uint32_t d;  // one conversion instruction: hi to bits 16-31, lo to bits 0-15, both rounded to nearest even
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}

// Quotient and remainder of a non-negative int x < 2^22 by a positive divisor through an FP32
// reciprocal computed once: x and 1/d are exact to 2^-24 relative, so the product is within 1/2 of
// x / d and the truncated quotient is off by at most one; one correction step makes it exact.
// (The GPU's FP64 rate is too low for this to be done in double precision on the hot path.)
struct FastDiv {
    int d;
    float inv;
};

__device__ __forceinline__ FastDiv make_fastdiv(int d) { return {d, 1.0f / (float)d}; }

__device__ __forceinline__ int fast_divmod(int x, const FastDiv& f, int& r)
{
    int q = __float2int_rz(__int2float_rn(x) * f.inv);
    r = x - q * f.d;
    if (r < 0) {
        --q;
        r += f.d;
    } else if (r >= f.d) {
        ++q;
        r -= f.d;
    }
    return q;
}

static_assert(EPI_WARPS == 4 || EPI_WARPS == 8, "one or two epilogue warps per TMEM lane quarter");
static_assert(GN_MAX_GROUPS % (EPI_WARPS / 4) == 0, "the column shares split the normalisation groups");

// Tile geometry: tile T of a launch -> image, first pixel (x0, y0) and first GEMM column n0.
struct TileGeo {
    int img, t, x0, y0, n0;
};

// Tiles are numbered column-tile-major (T = nt mtiles + mt), or, with `inter` (the halo form, whose
// CTAs keep the weights of one column tile), column-tile-minor (T = mt nsplit + nt): there a grid
// that is a multiple of nsplit gives every CTA a single column tile.
struct TileDivs {
    FastDiv mtiles, nsplit, tpi, tiles_per_row;
    int BW, BR;
    bool inter;
};

__device__ __forceinline__ TileDivs tile_divs(const ConvArgs& a, int mtiles, int nsplit, bool inter)
{
    const int BW = a.w < TM ? a.w : TM;
    return {make_fastdiv(mtiles), make_fastdiv(nsplit), make_fastdiv((a.h * a.w) / TM), make_fastdiv(a.w / BW),
            BW, TM / BW, inter};
}

__device__ __forceinline__ TileGeo tile_geo(const TileDivs& v, int T, int NT)
{
    TileGeo g;
    int mt, nt, r;
    if (v.inter)
        mt = fast_divmod(T, v.nsplit, nt);
    else
        nt = fast_divmod(T, v.mtiles, mt);
    g.img = fast_divmod(mt, v.tpi, g.t);
    g.y0 = fast_divmod(g.t, v.tiles_per_row, r) * v.BR;
    g.x0 = r * v.BW;
    g.n0 = nt * NT;
    return g;
}

// Persistent kernel: CTA b takes tiles b, b + gridDim.x, ...  The TMA / MMA stream runs through
// all of them without draining; two accumulators in tensor memory let the epilogue of one tile
// overlap the MMAs of the next.
// Position in a stage ring: stage, phase parity and stages passed, advanced without divisions.
struct Ring {
    int s = 0, it = 0;
    uint32_t ph = 0;
    __device__ __forceinline__ void next(int st)
    {
        ++it;
        if (++s == st) {
            s = 0;
            ph ^= 1u;
        }
    }
};

// GPT: normalisation groups per column tile (all 8 unless the halo form splits Cout over two tiles);
// HKB, HKC: channel blocks per tile in the halo form, and channels per block (64: 128-byte swizzle,
// 32: 64-byte swizzle).
template <int MODE, int NT, bool HALO = false, int GPT = GN_MAX_GROUPS, int HKB = 1, int HKC = 64>
__global__ void __launch_bounds__(NTHREADS, 1)
umma_conv_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, ConvArgs a)
{
    static_assert(GPT >= EPI_WARPS / 4 && GPT % (EPI_WARPS / 4) == 0 && NT % GPT == 0, "group split");
    extern __shared__ __align__(1024) uint8_t smraw[];
    uint8_t* const sm0 = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
    // halo mode: resident weights ([channel block][9 taps][NT rows][128 bytes]) first, then the stage ring
    constexpr uint32_t RB = 2u * HKC;  // halo form: bytes per pixel row of a channel block
    constexpr uint32_t bres = HALO ? (uint32_t)HKB * 9u * NT * RB : 0u;
    uint8_t* const sm = sm0 + bres;
    __shared__ __align__(8) uint64_t full_bar[MAX_ST], empty_bar[MAX_ST], accf_bar[2], acce_bar[2], bres_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int abort_flag;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int KC = a.kc, ST = a.stages;
    const uint32_t a_bytes = HALO ? halo_stage(HKC) : TM * KC * 2, b_bytes = HALO ? 0u : NT * KC * 2;
    const uint32_t stage_bytes = a_bytes + b_bytes;
    const int kblocks = HALO ? HKB : a.cin / KC, ntaps = MODE == TCONV ? 1 : 9, iters = HALO ? HKB : ntaps * kblocks;
    const int ncols = MODE == TCONV ? 4 * a.cout : a.cout;
    const int nsplit = ncols / NT;
    const int mtiles = a.n * ((a.h * a.w) / TM), tiles = mtiles * nsplit;
    const int tpi = (a.h * a.w) / TM;
    const int BW = a.w < TM ? a.w : TM;
    const TileDivs divs = tile_divs(a, mtiles, nsplit, HALO);

    if (tid == 0) {
        abort_flag = 0;
        for (int s = 0; s < ST; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full_bar[s])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty_bar[s])) : "memory");
        }
        for (int b = 0; b < 2; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&accf_bar[b])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&acce_bar[b])), "n"(EPI_WARPS)
                         : "memory");
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bres_bar)) : "memory");
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
            Ring r;
            bool ok = true;
            if constexpr (HALO) {  // this CTA's column tile, all 9 taps, once: one 64 x NT x 9 box per channel block
                const uint32_t bb = smem_u32(&bres_bar);
                const int ntc = (int)blockIdx.x % nsplit;  // the grid is a multiple of nsplit
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bb), "r"(bres) : "memory");
#pragma unroll
                for (int kb = 0; kb < HKB; ++kb)
                    asm volatile(
                        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(sm0 + (size_t)kb * 9 * NT * RB)),
                        "l"(reinterpret_cast<uint64_t>(&tmB)), "r"(kb * HKC), "r"(ntc * NT), "r"(0), "r"(bb)
                        : "memory");
            }
            for (int T = blockIdx.x; T < tiles && ok; T += gridDim.x) {
                const TileGeo g = tile_geo(divs, T, NT);
                for (int tap = 0; tap < (HALO ? 1 : ntaps) && ok; ++tap)
                    for (int kb = 0; kb < kblocks && ok; ++kb, r.next(ST)) {
                        ok = mbar_wait(smem_u32(&empty_bar[r.s]), r.ph ^ 1u, a.wait_cap, &abort_flag);
                        if (!ok) break;
                        const uint32_t fb = smem_u32(&full_bar[r.s]);
                        const uint32_t sa = smem_u32(sm + (size_t)r.s * stage_bytes), sb = sa + a_bytes;
                        if constexpr (HALO) {  // rows y0-1 .. y0+1, columns x0-1 .. x0+128 of channel block kb
                            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb),
                                         "r"(halo_box(HKC)) : "memory");
                            asm volatile(
                                "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                                " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(sa),
                                "l"(reinterpret_cast<uint64_t>(&tmA)), "r"(kb * HKC), "r"(g.x0 - 1), "r"(g.y0 - 1),
                                "r"(g.img), "r"(fb)
                                : "memory");
                        } else {
                            const int dy = MODE == TCONV ? 0 : tap / 3 - 1, dx = MODE == TCONV ? 0 : tap % 3 - 1;
                            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb),
                                         "r"(stage_bytes) : "memory");
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
            }
            if (!ok) {
                abort_flag = 1;
                atomicOr(a.err, UNET_ERR_TIMEOUT);
                // let the copies already issued land before the CTA leaves (bounded)
                const int it = r.it;
                for (int j = (it > ST ? it - ST : 0); j < it; ++j)
                    mbar_wait(smem_u32(&full_bar[j % ST]), (uint32_t)(j / ST) & 1u, a.wait_cap, &abort_flag);
                if constexpr (HALO) mbar_wait(smem_u32(&bres_bar), 0u, a.wait_cap, &abort_flag);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {  // ---- MMA issuer
            const uint32_t idesc = umma_idesc(NT);
            Ring r;
            int local = 0;
            bool ok = true;
            if constexpr (HALO) ok = mbar_wait(smem_u32(&bres_bar), 0u, a.wait_cap, &abort_flag);
            for (int T = blockIdx.x; T < tiles && ok; T += gridDim.x, ++local) {
                const int b = local & 1;
                // the epilogue must have drained this accumulator (its previous use)
                ok = mbar_wait(smem_u32(&acce_bar[b]), ((uint32_t)(local >> 1) & 1u) ^ 1u, a.wait_cap, &abort_flag);
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t d = tmem + (uint32_t)(b * NT);
                if constexpr (HALO) {
                    // all channel blocks of the tile first, then tap by tap: the per-tap form's order of sums
                    int ss[HKB];
#pragma unroll
                    for (int kb = 0; kb < HKB; ++kb, r.next(ST)) {
                        ss[kb] = r.s;
                        if (ok) ok = mbar_wait(smem_u32(&full_bar[r.s]), r.ph, a.wait_cap, &abort_flag);
                    }
                    if (!ok) break;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    // descriptors of the stage and weight bases; a window or K step adds its byte offset / 16
                    // to the start-address field (every address stays below 2^18)
                    uint64_t adesc[HKB];
#pragma unroll
                    for (int kb = 0; kb < HKB; ++kb) adesc[kb] = umma_desc(smem_u32(sm + (size_t)ss[kb] * stage_bytes), HKC);
                    const uint64_t bdesc = umma_desc(smem_u32(sm0), HKC);
#pragma unroll
                    for (int tap = 0; tap < 9; ++tap)
#pragma unroll
                        for (int kb = 0; kb < HKB; ++kb)
#pragma unroll
                            for (int kk = 0; kk < HKC / 16; ++kk) {
                                const uint64_t ad = adesc[kb] + (uint64_t)((((tap / 3) * HALO_W + tap % 3) * RB + kk * 32) >> 4);
                                const uint64_t bd = bdesc + (uint64_t)(((kb * 9 + tap) * NT * RB + kk * 32) >> 4);
                                const uint32_t acc = (tap | kb | kk) ? 1u : 0u;
                                asm volatile(
                                    "{ .reg .pred p; setp.ne.b32 p, %4, 0;\n"
                                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(d),
                                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                                    : "memory");
                            }
#pragma unroll
                    for (int kb = 0; kb < HKB; ++kb)
                        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                                     ::"r"(smem_u32(&empty_bar[ss[kb]])) : "memory");
                } else {
                    for (int k = 0; k < iters && ok; ++k, r.next(ST)) {
                        ok = mbar_wait(smem_u32(&full_bar[r.s]), r.ph, a.wait_cap, &abort_flag);
                        if (!ok) break;
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        const uint32_t sa = smem_u32(sm + (size_t)r.s * stage_bytes), sb = sa + a_bytes;
                        const uint64_t ad0 = umma_desc(sa, KC), bd0 = umma_desc(sb, KC);
                        for (int kk = 0; kk < KC / 16; ++kk) {
                            const uint64_t ad = ad0 + (uint64_t)(2 * kk), bd = bd0 + (uint64_t)(2 * kk);  // + 32 B
                            const uint32_t acc = (k | kk) ? 1u : 0u;
                            asm volatile(
                                "{ .reg .pred p; setp.ne.b32 p, %4, 0;\n"
                                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(d),
                                "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                                : "memory");
                        }
                        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                                     ::"r"(smem_u32(&empty_bar[r.s])) : "memory");
                    }
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
    } else {  // ---- epilogue, warps 2 .. 2 + EPI_WARPS - 1: TMEM lanes 32 (warp % 4) ... + 31
        constexpr int SHARES = EPI_WARPS / 4;      // warps per lane quarter
        constexpr int NS = NT / SHARES;            // columns per warp
        const int q = warp & 3;
        const int half = (warp - 2) / 4;           // columns [half NS, (half + 1) NS)
        const int row = q * 32 + lane;             // pixel within the tile
        constexpr int HG = GPT / SHARES;           // groups per warp (CONV3: GPT groups per column tile)
        static_assert(MODE != OUT3 || (NT == 16 && SHARES == 1), "the output layer is one 16-column tile");
        if constexpr (MODE == OUT3) {
            // u += gamma conv + beta for u = phi, c, rho.  The fields of the next PD tiles are loaded
            // ahead, so that the read-modify-write of a tile does not wait for its loads.
            constexpr int PD = 4;
            float og[3], ob[3];
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                og[f] = a.ogamma[f];
                ob[f] = a.obeta[f];
            }
            float pv[PD][3];
            float* pp[PD][3];
            auto fetch = [&](int T, int d) {
                if (T < tiles) {
                    const TileGeo g = tile_geo(divs, T, NT);
                    const size_t o = (size_t)(g.y0 + row / BW) * a.fpitch + g.x0 + row % BW;
#pragma unroll
                    for (int f = 0; f < 3; ++f) {
                        pp[d][f] = a.fields[f * a.n + g.img] + o;
                        pv[d][f] = *pp[d][f];
                    }
                }
            };
#pragma unroll
            for (int d = 0; d < PD; ++d) fetch((int)blockIdx.x + d * (int)gridDim.x, d);
            int local = 0;
            for (int T = blockIdx.x; T < tiles; T += gridDim.x, ++local) {
                const int b = local & 1;
                if (!mbar_wait_sleep(smem_u32(&accf_bar[b]), (uint32_t)(local >> 1) & 1u, a.wait_cap, &abort_flag)) {
                    abort_flag = 1;
                    if (lane == 0) atomicOr(a.err, UNET_ERR_TIMEOUT);
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                uint32_t r[4];
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                             : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                             : "r"(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * NT)));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0)
                    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acce_bar[b])) : "memory");
#pragma unroll
                for (int f = 0; f < 3; ++f) *pp[0][f] = pv[0][f] + fmaf(og[f], __uint_as_float(r[f]), ob[f]);
#pragma unroll
                for (int d = 0; d + 1 < PD; ++d)
#pragma unroll
                    for (int f = 0; f < 3; ++f) {
                        pv[d][f] = pv[d + 1][f];
                        pp[d][f] = pp[d + 1][f];
                    }
                fetch(T + PD * (int)gridDim.x, PD - 1);
            }
        } else {
        int local = 0;
        for (int T = blockIdx.x; T < tiles; T += gridDim.x, ++local) {
            const int b = local & 1;
            if (!mbar_wait_sleep(smem_u32(&accf_bar[b]), (uint32_t)(local >> 1) & 1u, a.wait_cap, &abort_flag)) {
                abort_flag = 1;
                if (lane == 0) atomicOr(a.err, UNET_ERR_TIMEOUT);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const TileGeo g = tile_geo(divs, T, NT);
            const int py = g.y0 + row / BW, px = g.x0 + row % BW;
            float s1[HG], s2[HG];
#pragma unroll
            for (int gg = 0; gg < HG; ++gg) s1[gg] = s2[gg] = 0.f;
#pragma unroll
            for (int k0 = 0; k0 < NS; k0 += 16) {
                const int c0 = half * NS + k0;
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
                {
                    uint32_t pk[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const float v0 = __uint_as_float(r[2 * j]), v1 = __uint_as_float(r[2 * j + 1]);
                        pk[j] = pack_bf16x2(v0, v1);
                    }
                    uint16_t* dst;
                    if (MODE == CONV3) {
                        constexpr int cg = NT / GPT;  // channels per group; NS = HG groups
#pragma unroll
                        for (int j = 0; j < 16; ++j) {  // the group index within the share is a compile-time constant
                            const float v = __uint_as_float(r[j]);
                            s1[(k0 + j) / cg] += v;
                            s2[(k0 + j) / cg] = fmaf(v, v, s2[(k0 + j) / cg]);
                        }
                        dst = a.out + ((size_t)(g.img * a.h + py) * a.w + px) * a.out_cstride + a.out_coff + g.n0 + c0;
                    } else {  // TCONV: column n0 + c0 + j = sub-pixel s * cout + channel
                        const int col = g.n0 + c0, s = col / a.cout, co = col % a.cout;
                        const int oy = 2 * py + (s >> 1), ox = 2 * px + (s & 1);
                        dst = a.out + ((size_t)(g.img * 2 * a.h + oy) * (2 * a.w) + ox) * a.out_cstride + a.out_coff + co;
                    }
                    uint4* d4 = reinterpret_cast<uint4*>(dst);
                    d4[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                    d4[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
                }
            }
            // the accumulator is drained: hand it back to the MMA issuer (one arrival per warp)
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0)
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acce_bar[b])) : "memory");
            if (MODE == CONV3 && a.partials) {
                // per warp: partials[((img * groups + g) * tpi + t) * 4 + q] = (sum, sum of squares) of its
                // HG groups; lane (32 / 2 HG) i holds value i: statistic i / HG of group half HG + i % HG
                float v[2 * HG];
#pragma unroll
                for (int gg = 0; gg < HG; ++gg) {
                    v[gg] = s1[gg];
                    v[HG + gg] = s2[gg];
                }
                const float tot = warp_sum_scatter<2 * HG>(v, lane);
                constexpr int LS = 32 / (2 * HG);
                if (lane % LS == 0) {
                    const int i = lane / LS, gg = (g.n0 / NT) * GPT + half * HG + i % HG, st = i / HG;
                    a.partials[((((size_t)g.img * a.groups + gg) * tpi + g.t) * 4 + q) * 2 + st] = tot;
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

bool g_halo_enabled = true;

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

int conv_nt(int mode, int cout) { return mode == TCONV ? (4 * cout < 256 ? 4 * cout : 256) : cout; }

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

// Column tile of the halo form, or 0 where it does not apply: 3x3 convolutions of 32, 64 or 128
// channels into at most 64, on rows that are whole 128-pixel tiles.  The weights of a column tile
// must fit next to the stages: 32 or 64 -> N keeps all N columns, 128 -> N keeps 32 (two column
// tiles for N = 64).  Channel blocks: one of 32 or 64 channels, or two of 64.
int halo_nt(int mode, const ConvArgs& a)
{
    if (!g_halo_enabled || mode == TCONV || a.w % TM || a.cout > 64) return 0;
    if (mode == OUT3) return a.cin == 32 ? a.cout : 0;
    return (a.cin == 32 || a.cin == 64) ? a.cout : (a.cin == 128 ? 32 : 0);
}

int halo_kc(int cin) { return cin == 32 ? 32 : 64; }

constexpr size_t HALO_SMEM = 225 * 1024;  // weights + stage ring (plus 1 KB of alignment slack)

int halo_stages(int cin, int nt)
{
    const int kc = halo_kc(cin);
    const int st = (int)((HALO_SMEM - (size_t)cin * 2 * 9 * nt) / halo_stage(kc));
    return st > MAX_ST ? MAX_ST : st;
}

size_t conv_smem_bytes(int mode, int cin, int nt, bool halo, int stages)
{
    if (halo) return (size_t)cin * 2 * 9 * nt + (size_t)stages * halo_stage(halo_kc(cin)) + 1024;
    const int kc = conv_kc(cin);
    return (size_t)stages * (size_t)(TM * kc * 2 + nt * kc * 2) + 1024;
}

}  // namespace

int set_conv_halo(int on)
{
    const int prev = g_halo_enabled ? 1 : 0;
    g_halo_enabled = on != 0;
    return prev;
}

cudaError_t launch_umma_conv(int mode, const uint16_t* in, const uint16_t* wgt, ConvArgs a, cudaStream_t s)
{
    if (a.cin % 32 || a.cout % 16 || a.cout < 16 || a.n < 1 || a.h < 1 || a.w < 1) return cudaErrorInvalidValue;
    if ((a.w % TM) && (TM % a.w)) return cudaErrorInvalidValue;
    if (((long long)a.h * a.w) % TM) return cudaErrorInvalidValue;
    if (mode == CONV3 && ((a.cout != 32 && a.cout != 64 && a.cout != 128 && a.cout != 256) || a.groups != GN_MAX_GROUPS))
        return cudaErrorInvalidValue;
    if (mode == TCONV && a.cout != 16 && a.cout != 32 && a.cout != 64 && a.cout != 128) return cudaErrorInvalidValue;
    if (mode == OUT3 && (a.cout != 16 || a.cin != 32 || !a.fields || !a.ogamma || !a.obeta || a.fpitch < a.w))
        return cudaErrorInvalidValue;
    if (mode == OUT3) a.partials = nullptr;
    if (a.out_coff % 8 || a.out_cstride % 8) return cudaErrorInvalidValue;  // 16-byte vector stores
    const int ncols = mode == TCONV ? 4 * a.cout : a.cout;
    a.kc = conv_kc(a.cin);
    const int hnt = halo_nt(mode, a);
    const bool halo = hnt > 0 && halo_stages(a.cin, hnt) >= 2;
    a.nt = halo ? hnt : conv_nt(mode, a.cout);
    if (ncols % a.nt) return cudaErrorInvalidValue;
    const int nsplit = ncols / a.nt;
    // tile indices (pixel tiles x at most 2 column tiles) stay below 2^22, the range of the FP32 divisions
    if ((long long)a.n * a.h * a.w / TM >= (1LL << 20) || nsplit > 2) return cudaErrorInvalidValue;
    a.stages = halo ? halo_stages(a.cin, a.nt) : conv_stages(a.kc, a.nt);
    if (halo && a.stages < a.cin / a.kc) return cudaErrorInvalidValue;  // a tile's channel blocks are resident together
    a.tmem_cols = 32;
    while (a.tmem_cols < 2 * a.nt) a.tmem_cols <<= 1;  // two accumulators
    const int BW = a.w < TM ? a.w : TM, BR = TM / BW;

    CUtensorMap mA, mB;
    const cuuint64_t dA[4] = {(cuuint64_t)a.cin, (cuuint64_t)a.w, (cuuint64_t)a.h, (cuuint64_t)a.n};
    const cuuint64_t sA[3] = {(cuuint64_t)a.cin * 2, (cuuint64_t)a.w * a.cin * 2, (cuuint64_t)a.h * a.w * a.cin * 2};
    // halo mode: three rows of 130 pixels per box, and all nine taps of the weights in one box
    const cuuint32_t bA[4] = {(cuuint32_t)a.kc, (cuuint32_t)(halo ? HALO_W : BW), (cuuint32_t)(halo ? 3 : BR), 1u};
    const int taps = mode == TCONV ? 1 : 9;
    const cuuint64_t dB[3] = {(cuuint64_t)a.cin, (cuuint64_t)ncols, (cuuint64_t)taps};
    const cuuint64_t sB[2] = {(cuuint64_t)a.cin * 2, (cuuint64_t)ncols * a.cin * 2};
    const cuuint32_t bB[3] = {(cuuint32_t)a.kc, (cuuint32_t)a.nt, halo ? 9u : 1u};
    if (!encode(&mA, in, 4, dA, sA, bA, a.kc) || !encode(&mB, wgt, 3, dB, sB, bB, a.kc))
        return cudaErrorInvalidValue;

    const size_t smem = conv_smem_bytes(mode, a.cin, a.nt, halo, a.stages);
    cudaLaunchConfig_t cfg = {};
    const long long tiles = (long long)a.n * a.h * a.w / TM * (ncols / a.nt);
    int per_sm = (int)((227 * 1024) / (smem + 2048));  // CTAs that fit next to each other on an SM
    per_sm = per_sm < 1 ? 1 : (per_sm > 2 ? 2 : per_sm);
    if (per_sm * a.tmem_cols > 512) per_sm = 512 / a.tmem_cols;
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
        // two CTAs of a small-stage configuration share an SM: ask for the largest shared-memory carveout,
        // and cap the CTAs per SM by their registers as well
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        if (e != cudaSuccess) return e;
        cudaFuncAttributes fa;
        e = cudaFuncGetAttributes(&fa, kern);
        if (e != cudaSuccess) return e;
        const int regs_cta = NTHREADS * ((fa.numRegs + 7) & ~7);
        const int by_regs = regs_cta > 0 ? 65536 / regs_cta : 1;
        const int ps = by_regs < 1 ? 1 : (by_regs < per_sm ? by_regs : per_sm);
        const long long slots = (long long)sm_count() * ps;
        long long grid = tiles < slots ? tiles : slots;
        if (halo) grid = grid < nsplit ? nsplit : grid - grid % nsplit;  // each CTA keeps one column tile's weights
        cfg.gridDim = dim3((unsigned)grid);
        return cudaLaunchKernelEx(&cfg, kern, mA, mB, a);
    };
    if (mode == OUT3) {
        if (halo) return go(umma_conv_kernel<OUT3, 16, true, GN_MAX_GROUPS, 1, 32>);
        return go(umma_conv_kernel<OUT3, 16>);
    }
    if (halo && a.cin == 32) {
        if (a.nt == 32) return go(umma_conv_kernel<CONV3, 32, true, GN_MAX_GROUPS, 1, 32>);
        if (a.nt == 64) return go(umma_conv_kernel<CONV3, 64, true, GN_MAX_GROUPS, 1, 32>);
        return cudaErrorInvalidValue;
    }
    if (halo) {
        const int kb = a.cin / 64;
        if (a.nt == 32 && nsplit == 1 && kb == 1) return go(umma_conv_kernel<CONV3, 32, true, GN_MAX_GROUPS, 1>);
        if (a.nt == 32 && nsplit == 1 && kb == 2) return go(umma_conv_kernel<CONV3, 32, true, GN_MAX_GROUPS, 2>);
        if (a.nt == 32 && nsplit == 2 && kb == 2) return go(umma_conv_kernel<CONV3, 32, true, GN_MAX_GROUPS / 2, 2>);
        if (a.nt == 64 && nsplit == 1 && kb == 1) return go(umma_conv_kernel<CONV3, 64, true, GN_MAX_GROUPS, 1>);
        return cudaErrorInvalidValue;
    }
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
