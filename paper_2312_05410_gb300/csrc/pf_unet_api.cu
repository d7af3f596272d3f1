// C-ABI layer of the U-Net path (declarations in include/pf.h): the two tensor-core
// convolution primitives, and (below) the time-conditioned U-Net jump of the
// hybrid DNS / U-Net solver ("U-Net with temporal conditioning", Methods;
// "Hybrid" in Results: the surrogate leaps over a stretch of DNS steps).
#include <cstdarg>
#include <cstdio>
#include <string>

#include "pf.h"
#include "pf_unet_internal.h"

namespace {

thread_local std::string g_unet_error;

int ufail(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_unet_error = buf;
    return code;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

int conv_common(int mode, const void* in, int n, int h, int w, int cin, const void* wgt, int cout, void* out,
                int out_cstride, int out_coff, int groups, float* partials, int* err_dev, void* stream)
{
    if (!in || !wgt || !out || !err_dev) return ufail(PF_ERR_ARG, "null pointer");
    if (n < 1 || h < 1 || w < 1 || n > (1 << 16) || h > (1 << 14) || w > (1 << 14))
        return ufail(PF_ERR_ARG, "bad image size %d x %d x %d", n, h, w);
    if (cin < 32 || cin > 1024 || cin % 32 || cout < 16 || cout % 16)
        return ufail(PF_ERR_ARG, "channels cin=%d cout=%d unsupported (cin %% 32, cout %% 16)", cin, cout);
    if (mode == pf::CONV3 && (cout > 256 || groups < 1 || groups > pf::GN_MAX_GROUPS || cout % groups))
        return ufail(PF_ERR_ARG, "cout=%d / groups=%d unsupported", cout, groups);
    if ((w % 128) && (128 % w)) return ufail(PF_ERR_ARG, "width %d: must divide or be a multiple of 128", w);
    if (((long long)h * w) % 128) return ufail(PF_ERR_ARG, "h*w must be a multiple of 128");
    if (out_cstride < out_coff + cout || out_coff % 8 || out_cstride % 8)
        return ufail(PF_ERR_LAYOUT, "output slice [%d, %d) of %d channels", out_coff, out_coff + cout, out_cstride);
    if (!aligned16(in) || !aligned16(wgt) || !aligned16(out)) return ufail(PF_ERR_LAYOUT, "16-byte alignment");
    pf::ConvArgs a = {};
    a.n = n;
    a.h = h;
    a.w = w;
    a.cin = cin;
    a.cout = cout;
    a.groups = groups;
    a.out = static_cast<uint16_t*>(out);
    a.out_cstride = out_cstride;
    a.out_coff = out_coff;
    a.partials = partials;
    a.err = err_dev;
    a.wait_cap = 1 << 22;
    cudaError_t e = pf::launch_umma_conv(mode, static_cast<const uint16_t*>(in), static_cast<const uint16_t*>(wgt),
                                         a, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return ufail(PF_ERR_CUDA, "convolution launch: %s", cudaGetErrorString(e));
    return PF_OK;
}

}  // namespace

extern "C" {

int pf_conv3x3_bf16(const void* in, int n, int h, int w, int cin, const void* wgt, int cout, void* out,
                    int out_cstride, int out_coff, int groups, float* partials, int* err_dev, void* stream)
{
    return conv_common(pf::CONV3, in, n, h, w, cin, wgt, cout, out, out_cstride, out_coff, groups, partials,
                       err_dev, stream);
}

int pf_tconv2x2_bf16(const void* in, int n, int h, int w, int cin, const void* wgt, int cout, void* out,
                     int out_cstride, int out_coff, int* err_dev, void* stream)
{
    return conv_common(pf::TCONV, in, n, h, w, cin, wgt, cout, out, out_cstride, out_coff, 1, nullptr, err_dev,
                       stream);
}

const char* pf_unet_last_error(void) { return g_unet_error.c_str(); }

}  // extern "C"
