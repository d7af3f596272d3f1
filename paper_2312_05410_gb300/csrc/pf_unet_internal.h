// Internal interface of the U-Net kernels (not part of the C ABI).
#pragma once

#include <cstdint>

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

namespace pf {

// cuTensorMapEncodeTiled through the runtime's driver entry point (NULL if unavailable).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();

// CONV3: 3x3 convolution into BF16 channels (with group sums); TCONV: 2x2 stride-2 transposed
// convolution; OUT3: 3x3 convolution whose first three output columns are added, through a
// per-output affine (gamma, beta), to three FP32 fields in place (the U-Net's output layer).
enum ConvMode { CONV3 = 0, TCONV = 1, OUT3 = 2 };
constexpr int GN_MAX_GROUPS = 8;        // group normalisation groups of the hidden layers
constexpr int UNET_ERR_TIMEOUT = 2;     // error-word bit: a bounded wait of a tensor-core kernel ran out

#ifdef __CUDACC__
// Sum over the warp of V values per lane (V = 2^b <= 32) by recursive halving: each exchange
// step, with offsets 16, 8, ... down to 32 / V, sends half of the remaining values to the partner
// lane and keeps the other half, so that lane l ends with value (l >> (5 - b)) & (V - 1) summed
// over the lanes that agree with l in their low 5 - b bits; full exchanges at the remaining
// offsets complete the sum over all 32 lanes.  V + 4 - b shuffles instead of 5 V.
template <int V>
__device__ __forceinline__ float warp_sum_scatter(float (&v)[V], int lane)
{
    static_assert(V >= 1 && V <= 32 && (V & (V - 1)) == 0, "V must be a power of two <= 32");
#pragma unroll
    for (int h = V / 2, o = 16; h >= 1; h >>= 1, o >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int j = 0; j < h; ++j) {
            const float send = up ? v[j] : v[j + h];
            const float keep = up ? v[j + h] : v[j];
            v[j] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    float s = v[0];
#pragma unroll
    for (int o = 16 / V; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}
#endif

// Arguments of one implicit-GEMM convolution launch (see pf_unet_conv.cu).
struct ConvArgs {
    int n, h, w;           // images and input size
    int cin, cout;         // channels (TCONV: GEMM N = 4 cout)
    int kc, nt, stages;    // K block (32 or 64 channels), N tile (<= 256), pipeline depth
    int tmem_cols;         // accumulator columns allocated (power of 2, >= nt, >= 32)
    int groups;            // CONV3: normalisation groups of cout
    uint16_t* out;         // BF16 NHWC output (CONV3: n x h x w; TCONV: n x 2h x 2w)
    int out_cstride;       // channels per output pixel (the output is a slice of a wider buffer)
    int out_coff;          // first channel of the slice
    float* partials;       // CONV3: per-tile group sums [n][groups][h*w/128][2], or NULL
    int* err;              // error word (UNET_ERR_TIMEOUT)
    int wait_cap;          // polls of a bounded mbarrier wait
    float* const* fields;  // OUT3: device table of 3 n field pointers (phi of each image, then c, then rho)
    int fpitch;            // OUT3: row pitch of the fields (floats)
    const float* ogamma;   // OUT3: device, 3 values
    const float* obeta;    // OUT3: device, 3 values
};

// Encode the tensor maps and launch.  in: BF16 NHWC [n][h][w][cin]; wgt: BF16
// [taps][ncols][cin] with taps = 9 (CONV3, ncols = cout) or 1 (TCONV, ncols = 4 cout,
// row s * cout + co for output sub-pixel s = 2 dy + dx).  Requires cin % 32 == 0,
// cout % 16 == 0, and (h * w) % 128 == 0 with w % 128 == 0 or 128 % w == 0.
// Returns cudaErrorInvalidValue for shapes outside these rules.
cudaError_t launch_umma_conv(int mode, const uint16_t* in, const uint16_t* wgt, ConvArgs a, cudaStream_t s);
// Enables (1) or disables (0) the halo form of the 3x3 convolution; returns the previous setting.
int set_conv_halo(int on);

}  // namespace pf
