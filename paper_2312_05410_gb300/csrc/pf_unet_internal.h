// Internal interface of the U-Net kernels (not part of the C ABI).
#pragma once

#include <cstdint>

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

namespace pf {

// cuTensorMapEncodeTiled through the runtime's driver entry point (NULL if unavailable).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();

enum ConvMode { CONV3 = 0, TCONV = 1 };
constexpr int GN_MAX_GROUPS = 8;        // group normalisation groups of the hidden layers
constexpr int UNET_ERR_TIMEOUT = 2;     // error-word bit: a bounded wait of a tensor-core kernel ran out

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
};

// Encode the tensor maps and launch.  in: BF16 NHWC [n][h][w][cin]; wgt: BF16
// [taps][ncols][cin] with taps = 9 (CONV3, ncols = cout) or 1 (TCONV, ncols = 4 cout,
// row s * cout + co for output sub-pixel s = 2 dy + dx).  Requires cin % 32 == 0,
// cout % 16 == 0, and (h * w) % 128 == 0 with w % 128 == 0 or 128 % w == 0.
// Returns cudaErrorInvalidValue for shapes outside these rules.
cudaError_t launch_umma_conv(int mode, const uint16_t* in, const uint16_t* wgt, ConvArgs a, cudaStream_t s);
size_t umma_conv_smem_bytes(int mode, int cin, int cout);

}  // namespace pf
