// Launchers of the CUDA-core kernels of the U-Net (pf_unet_net.cu); internal.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace pf {

constexpr int UNET_FDIM = 128;       // MLP hidden width and basis size
constexpr float UNET_EPS = 1e-5f;    // group-normalisation epsilon

cudaError_t launch_cond(const double* mlp, const double* proj, double tau, float* scales, int nscales, cudaStream_t s);
// Look-back input: the two older frames are FP32 planes [image][3][h][w] (NULL: use the current fields).
constexpr int UNET_LB = 3;                 // frames fed to the network
constexpr int UNET_IN = 3 * UNET_LB + 1;   // input planes: the frames' (phi, c, rho), oldest first, then tau
cudaError_t launch_in_conv(const float* const* phi, const float* const* c, const float* const* rho, int pitch,
                           const float* old0, const float* old1, int n, int h, int w, float tau,
                           const float* wgt, uint16_t* out, float* partials, cudaStream_t s);
cudaError_t launch_frame(const float* const* phi, const float* const* c, const float* const* rho, int pitch, int n,
                         int h, int w, float* dst, cudaStream_t s);
cudaError_t launch_gn_stats(const float* partials, int n, int groups, int entries, double count, int C,
                            const float* gamma, const float* beta, float* affine, cudaStream_t s);
cudaError_t launch_gn_enc(const uint16_t* x, int n, int h, int w, int C, const float* affine, const float* scale,
                          uint16_t* cat, int cat_stride, uint16_t* pool, cudaStream_t s);
cudaError_t launch_gn_dec(const uint16_t* x, int n, int h, int w, int C, const float* affine, uint16_t* y,
                          cudaStream_t s);
cudaError_t launch_check(const float* const* phi, const float* const* c, const float* const* rho, int n, int h, int w,
                         int pitch, float phi_lo, float phi_hi, float c_lo, float c_hi, float r_lo, float r_hi,
                         int* flags, cudaStream_t s);

}  // namespace pf
