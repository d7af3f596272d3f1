// C-ABI layer of the U-Net path (declarations in include/pf.h): the two tensor-core
// convolution primitives, and (below) the time-conditioned U-Net jump of the
// hybrid DNS / U-Net solver ("U-Net with temporal conditioning", Methods;
// "Hybrid" in Results: the surrogate leaps over a stretch of DNS steps).
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "pf.h"
#include "pf_internal.h"
#include "pf_unet_internal.h"
#include "pf_unet_net.h"

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
    if (mode == pf::CONV3 && ((cout != 32 && cout != 64 && cout != 128 && cout != 256) || groups != pf::GN_MAX_GROUPS))
        return ufail(PF_ERR_ARG, "cout=%d / groups=%d unsupported (cout 32, 64, 128 or 256; 8 groups)", cout, groups);
    if (mode == pf::TCONV && cout != 16 && cout != 32 && cout != 64 && cout != 128)
        return ufail(PF_ERR_ARG, "cout=%d unsupported (16, 32, 64 or 128)", cout);
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


// ---------------------------------------------------------------------------------------------
// The network: weights, activations and the jump.

namespace {

constexpr int NW = 40;  // weight arrays, in the order documented in pf.h
static_assert(pf::UNET_LB == 3, "the look-back ring holds two frames (slots 0 and 1)");
const int CH[4] = {32, 64, 128, 256};

// host BF16 rounding (nearest, ties to even) from the format definition
uint16_t host_bf16(float f)
{
    uint32_t u;
    std::memcpy(&u, &f, 4);
    if ((u & 0x7f800000u) == 0x7f800000u && (u & 0x007fffffu)) return (uint16_t)((u >> 16) | 0x40);
    u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

struct UnetLayout {
    size_t mlp, proj, win, wout, wc[7], wt[3], gb[9][2];
    size_t act[16];  // see ACT_* below
    size_t partials, stats, scales, err, ptrs, flags, ring, fptrs, total;
};
enum { A_PRE1, A_CAT1, A_P1, A_PRE2, A_CAT2, A_P2, A_PRE3, A_CAT3, A_P3, A_PRE4, A_ZC4, A_H4, A_H3, A_H2, A_H1, A_PREO };

bool shape_ok(int n, int h, int w)
{
    if (n < 1 || n > 4096 || h < 128 || w < 128 || h > 8192 || w > 8192 || h % 8 || w % 8) return false;
    if ((long long)n * h * w >= (1LL << 27)) return false;  // the convolutions' tile-index range
    const int w8 = w / 8;
    if ((w8 % 128) && (128 % w8)) return false;
    return ((long long)(h / 8) * w8) % 128 == 0;
}

UnetLayout unet_layout(int n, int h, int w)
{
    UnetLayout L;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = al256(off + bytes);
        return o;
    };
    L.mlp = take(sizeof(double) * (3 * 128 + 2 * 128 * 128 + 128));
    L.proj = take(sizeof(double) * 480 * 128);
    L.win = take(sizeof(float) * 9 * pf::UNET_IN * 32);
    L.wout = take(2 * 9 * 16 * 32);  // output conv as one 16-column tensor-core tile: [tap][16][32] BF16, rows 3.. zero
    const int conv_io[7][2] = {{32, 64}, {64, 128}, {128, 256}, {256, 256}, {256, 128}, {128, 64}, {64, 32}};
    for (int k = 0; k < 7; ++k) L.wc[k] = take(2 * 9 * (size_t)conv_io[k][0] * conv_io[k][1]);
    const int tc_io[3][2] = {{256, 128}, {128, 64}, {64, 32}};
    for (int k = 0; k < 3; ++k) L.wt[k] = take(2 * 4 * (size_t)tc_io[k][0] * tc_io[k][1]);
    const int gbc[9] = {32, 64, 128, 256, 256, 128, 64, 32, 3};
    for (int k = 0; k < 9; ++k)
        for (int q = 0; q < 2; ++q) L.gb[k][q] = take(sizeof(float) * gbc[k]);
    const size_t P0 = (size_t)n * h * w, P1 = P0 / 4, P2 = P0 / 16, P3 = P0 / 64;
    const size_t elems[16] = {P0 * 32, P0 * 64, P1 * 32, P1 * 64, P1 * 128, P2 * 64, P2 * 128, P2 * 256,
                              P3 * 128, P3 * 256, P3 * 256, P3 * 256, P2 * 128, P1 * 64, P0 * 32, 0};
    for (int k = 0; k < 16; ++k) L.act[k] = take(2 * elems[k]);
    L.partials = take(sizeof(float) * (size_t)n * 8 * (h * (size_t)w / 128) * 4 * 2);
    L.stats = take(sizeof(float) * (size_t)n * 256 * 2);  // per-channel GN affine (a, b) of the current layer
    L.scales = take(sizeof(float) * 480);
    L.err = take(sizeof(int));
    L.ptrs = take(sizeof(float*) * 3 * (size_t)n);
    L.flags = take(sizeof(int) * (size_t)n);
    L.ring = take(sizeof(float) * (pf::UNET_LB - 1) * (size_t)n * 3 * h * w);  // look-back frames, FP32 [slot][n][3][h][w]
    L.fptrs = take(sizeof(float*) * 3 * (size_t)n);
    L.total = off;
    return L;
}

}  // namespace

struct pf_unet {
    int n, h, w;
    char* base;
    UnetLayout L;
    cudaStream_t stream;
    std::vector<float*> ptrs;  // host copy of the run pointer table (phi[n], c[n], rho[n])
    double cond_tau;           // jump length the stored conditioning factors belong to
    int last_pitch;            // row pitch of the fields of the last jump
    bool cond_valid;
    int frames;                // look-back frames held (0 .. UNET_LB - 1)
    int newest;                // ring slot of the newest frame
    std::vector<const float*> fptrs;  // host copy of the pointer table of the last pushed frame
    template <class T>
    T* at(size_t off) const { return reinterpret_cast<T*>(base + off); }
};

namespace pf {

void unet_shape(const pf_unet* u, int* batch, int* nx, int* ny)
{
    *batch = u->n;
    *nx = u->w;
    *ny = u->h;
}

cudaStream_t unet_stream(const pf_unet* u) { return u->stream; }

}  // namespace pf

namespace {

int upload(pf_unet* u, size_t off, const void* src, size_t bytes)
{
    cudaError_t e = cudaMemcpyAsync(u->base + off, src, bytes, cudaMemcpyHostToDevice, u->stream);
    if (e != cudaSuccess) return ufail(PF_ERR_CUDA, "weight upload: %s", cudaGetErrorString(e));
    return PF_OK;
}

// One tensor-core convolution; with gamma/beta, also its group statistics folded into the
// per-channel affine of the normalisation that follows (in the stats buffer).
int conv_tc(pf_unet* u, int mode, const uint16_t* in, int h, int w, int cin, const uint16_t* wgt, int cout,
            uint16_t* out, int cstride, int coff, const float* gamma = nullptr, const float* beta = nullptr)
{
    pf::ConvArgs a = {};
    a.n = u->n;
    a.h = h;
    a.w = w;
    a.cin = cin;
    a.cout = cout;
    a.groups = pf::GN_MAX_GROUPS;
    a.out = out;
    a.out_cstride = cstride;
    a.out_coff = coff;
    const bool stats_too = gamma != nullptr;
    a.partials = stats_too ? u->at<float>(u->L.partials) : nullptr;
    a.err = u->at<int>(u->L.err);
    a.wait_cap = 1 << 22;
    cudaError_t e = pf::launch_umma_conv(mode, in, wgt, a, u->stream);
    if (e != cudaSuccess) return ufail(PF_ERR_CUDA, "tensor-core convolution: %s", cudaGetErrorString(e));
    if (!stats_too) return PF_OK;
    e = pf::launch_gn_stats(u->at<float>(u->L.partials), u->n, pf::GN_MAX_GROUPS, h * w / 128 * 4,
                            (double)(cout / pf::GN_MAX_GROUPS) * h * w, cout, gamma, beta, u->at<float>(u->L.stats),
                            u->stream);
    if (e != cudaSuccess) return ufail(PF_ERR_CUDA, "group statistics: %s", cudaGetErrorString(e));
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

int pf_conv_halo(int on) { return pf::set_conv_halo(on); }

size_t pf_unet_workspace_size(int batch, int nx, int ny)
{
    if (!shape_ok(batch, ny, nx)) return 0;
    return unet_layout(batch, ny, nx).total;
}

int pf_unet_init(const float* const* weights, int nweights, int batch, int nx, int ny, void* work, size_t work_bytes,
                 void* stream, pf_unet** out)
{
    if (!out) return ufail(PF_ERR_ARG, "null output handle pointer");
    *out = nullptr;
    if (!weights || nweights != NW) return ufail(PF_ERR_ARG, "expected %d weight arrays", NW);
    for (int k = 0; k < NW; ++k)
        if (!weights[k]) return ufail(PF_ERR_ARG, "weight array %d is null", k);
    if (!shape_ok(batch, ny, nx))
        return ufail(PF_ERR_ARG, "batch %d of %d x %d unsupported (sides >= 128, multiples of 8, nx/8 dividing "
                     "or a multiple of 128, nx*ny %% 8192 == 0)", batch, nx, ny);
    if (!work || reinterpret_cast<uintptr_t>(work) % 256) return ufail(PF_ERR_LAYOUT, "workspace must be 256-byte aligned");
    const UnetLayout L = unet_layout(batch, ny, nx);
    if (work_bytes < L.total) return ufail(PF_ERR_LAYOUT, "workspace of %zu bytes, %zu needed", work_bytes, L.total);
    pf_unet* u = new (std::nothrow) pf_unet();
    if (!u) return ufail(PF_ERR_ARG, "out of host memory");
    u->n = batch;
    u->h = ny;
    u->w = nx;
    u->base = static_cast<char*>(work);
    u->L = L;
    u->stream = static_cast<cudaStream_t>(stream);
    u->ptrs.assign(3 * (size_t)batch, nullptr);
    u->cond_valid = false;
    u->last_pitch = nx;
    u->cond_tau = 0.0;
    u->frames = 0;
    u->newest = 0;
    u->fptrs.assign(3 * (size_t)batch, nullptr);
    // ---- host-side conversion into the device layouts (once)
    std::vector<double> mlp;
    for (int k = 0; k < 6; ++k) {
        const size_t cnt = (k == 2 || k == 4) ? 128 * 128 : 128;
        mlp.insert(mlp.end(), weights[k], weights[k] + cnt);
    }
    std::vector<double> proj;
    for (int p = 0; p < 4; ++p) proj.insert(proj.end(), weights[6 + p], weights[6 + p] + (size_t)CH[p] * 128);
    // first conv [32][UNET_IN][3][3] -> [(ky,kx,ci)][co], FP32 (this layer runs in FP32 on the CUDA cores)
    constexpr int CI = pf::UNET_IN;
    std::vector<float> win(9 * CI * 32);
    for (int co = 0; co < 32; ++co)
        for (int ci = 0; ci < CI; ++ci)
            for (int t = 0; t < 9; ++t) win[(t * CI + ci) * 32 + co] = weights[10][((co * CI + ci) * 9) + t];
    // last conv [3][32][3][3] -> [tap][16][32] BF16 (output columns 3..15 zero)
    std::vector<uint16_t> wout(9 * 16 * 32, 0);
    for (int co = 0; co < 3; ++co)
        for (int ci = 0; ci < 32; ++ci)
            for (int t = 0; t < 9; ++t) wout[(t * 16 + co) * 32 + ci] = host_bf16(weights[21][((co * 32 + ci) * 9) + t]);
    // tensor-core convs [Cout][Cin][3][3] -> [tap][Cout][Cin] BF16: enc2..4 (11..13), dec4..1 (14..17)
    const int conv_io[7][2] = {{32, 64}, {64, 128}, {128, 256}, {256, 256}, {256, 128}, {128, 64}, {64, 32}};
    const int conv_src[7] = {11, 12, 13, 14, 15, 16, 17};
    int rc = PF_OK;
    std::vector<std::vector<uint16_t>> keep;
    for (int k = 0; k < 7 && rc == PF_OK; ++k) {
        const int ci_n = conv_io[k][0], co_n = conv_io[k][1];
        std::vector<uint16_t> v((size_t)9 * co_n * ci_n);
        for (int co = 0; co < co_n; ++co)
            for (int ci = 0; ci < ci_n; ++ci)
                for (int t = 0; t < 9; ++t)
                    v[((size_t)t * co_n + co) * ci_n + ci] = host_bf16(weights[conv_src[k]][((size_t)co * ci_n + ci) * 9 + t]);
        keep.push_back(std::move(v));
        rc = upload(u, L.wc[k], keep.back().data(), keep.back().size() * 2);
    }
    // transposed convs [Cin][Cout][2][2] -> [(2 dy + dx) Cout + co][Cin]: up4, up3, up2 (18..20)
    const int tc_io[3][2] = {{256, 128}, {128, 64}, {64, 32}};
    for (int k = 0; k < 3 && rc == PF_OK; ++k) {
        const int ci_n = tc_io[k][0], co_n = tc_io[k][1];
        std::vector<uint16_t> v((size_t)4 * co_n * ci_n);
        for (int ci = 0; ci < ci_n; ++ci)
            for (int co = 0; co < co_n; ++co)
                for (int s = 0; s < 4; ++s)
                    v[((size_t)s * co_n + co) * ci_n + ci] = host_bf16(weights[18 + k][((size_t)ci * co_n + co) * 4 + s]);
        keep.push_back(std::move(v));
        rc = upload(u, L.wt[k], keep.back().data(), keep.back().size() * 2);
    }
    const int gbc[9] = {32, 64, 128, 256, 256, 128, 64, 32, 3};
    if (rc == PF_OK) rc = upload(u, L.mlp, mlp.data(), mlp.size() * sizeof(double));
    if (rc == PF_OK) rc = upload(u, L.proj, proj.data(), proj.size() * sizeof(double));
    if (rc == PF_OK) rc = upload(u, L.win, win.data(), win.size() * sizeof(float));
    if (rc == PF_OK) rc = upload(u, L.wout, wout.data(), wout.size() * sizeof(uint16_t));
    for (int k = 0; k < 9 && rc == PF_OK; ++k)
        for (int q = 0; q < 2 && rc == PF_OK; ++q) rc = upload(u, L.gb[k][q], weights[22 + 2 * k + q], gbc[k] * sizeof(float));
    if (rc == PF_OK) {
        cudaError_t e = cudaMemsetAsync(u->base + L.err, 0, sizeof(int), u->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(u->stream);  // host staging vectors go out of scope
        if (e != cudaSuccess) rc = ufail(PF_ERR_CUDA, "U-Net init: %s", cudaGetErrorString(e));
    }
    if (rc != PF_OK) {
        delete u;
        return rc;
    }
    *out = u;
    return PF_OK;
}

int pf_unet_jump(pf_unet* u, int n, float* const* phi, float* const* c, float* const* rho, int pitch, double tau)
{
    pf::TraceRange trace("pf_unet_jump");
    if (!u || !phi || !c || !rho) return ufail(PF_ERR_ARG, "null pointer");
    if (n != u->n) return ufail(PF_ERR_ARG, "batch %d, the handle was built for %d", n, u->n);
    if (pitch < u->w) return ufail(PF_ERR_LAYOUT, "pitch %d < nx %d", pitch, u->w);
    if (!std::isfinite(tau)) return ufail(PF_ERR_ARG, "jump length is not finite");
    for (int i = 0; i < n; ++i) {
        if (!phi[i] || !c[i] || !rho[i]) return ufail(PF_ERR_ARG, "run %d: null field", i);
        u->ptrs[i] = phi[i];
        u->ptrs[n + i] = c[i];
        u->ptrs[2 * n + i] = rho[i];
    }
    cudaStream_t s = u->stream;
    u->last_pitch = pitch;
    cudaError_t e = cudaMemcpyAsync(u->base + u->L.ptrs, u->ptrs.data(), sizeof(float*) * 3 * n,
                                    cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return ufail(PF_ERR_CUDA, "pointer table: %s", cudaGetErrorString(e));
    float** dp = u->at<float*>(u->L.ptrs);
    const UnetLayout& L = u->L;
    const int H = u->h, W = u->w;
    auto act = [&](int k) { return u->at<uint16_t>(L.act[k]); };
    float* part = u->at<float>(L.partials);
    float* stats = u->at<float>(L.stats);
    float* sc = u->at<float>(L.scales);
    auto gam = [&](int k) { return u->at<float>(L.gb[k][0]); };
    auto bet = [&](int k) { return u->at<float>(L.gb[k][1]); };
    const int G = pf::GN_MAX_GROUPS;
    int rc = PF_OK;  // G: the 8 groups of the first block's statistics
    auto ck = [&](cudaError_t ce, const char* what) {
        if (rc == PF_OK && ce != cudaSuccess) rc = ufail(PF_ERR_CUDA, "%s: %s", what, cudaGetErrorString(ce));
    };
    // conditioning factors of the four levels (kept while the jump length stays the same)
    if (!u->cond_valid || u->cond_tau != tau) {
        ck(pf::launch_cond(u->at<double>(L.mlp), u->at<double>(L.proj), tau, sc, 480, s), "conditioning");
        u->cond_valid = rc == PF_OK;
        u->cond_tau = tau;
    }
    // ---- encoder
    // look-back frames: the oldest and the middle one (a missing frame is the oldest one held, or the
    // current fields when none is)
    const size_t frame_elems = (size_t)n * 3 * H * W;
    const float* ring = u->at<float>(L.ring);
    const float* newest = u->frames > 0 ? ring + (size_t)u->newest * frame_elems : nullptr;
    const float* older = u->frames > 1 ? ring + (size_t)(1 - u->newest) * frame_elems : newest;
    ck(pf::launch_in_conv(dp, dp + n, dp + 2 * n, pitch, older, newest, n, H, W, (float)tau, u->at<float>(L.win),
                          act(A_PRE1), part, s),
       "input conv");
    ck(pf::launch_gn_stats(part, n, G, H * W / 128, 4.0 * H * W, 32, gam(0), bet(0), stats, s), "statistics");
    ck(pf::launch_gn_enc(act(A_PRE1), n, H, W, 32, stats, sc, act(A_CAT1), 64, act(A_P1), s), "level 1");
    if (rc == PF_OK)
        rc = conv_tc(u, pf::CONV3, act(A_P1), H / 2, W / 2, 32, u->at<uint16_t>(L.wc[0]), 64, act(A_PRE2), 64, 0, gam(1), bet(1));
    ck(pf::launch_gn_enc(act(A_PRE2), n, H / 2, W / 2, 64, stats, sc + 32, act(A_CAT2), 128, act(A_P2), s), "level 2");
    if (rc == PF_OK)
        rc = conv_tc(u, pf::CONV3, act(A_P2), H / 4, W / 4, 64, u->at<uint16_t>(L.wc[1]), 128, act(A_PRE3), 128, 0, gam(2), bet(2));
    ck(pf::launch_gn_enc(act(A_PRE3), n, H / 4, W / 4, 128, stats, sc + 96, act(A_CAT3), 256, act(A_P3), s), "level 3");
    if (rc == PF_OK)
        rc = conv_tc(u, pf::CONV3, act(A_P3), H / 8, W / 8, 128, u->at<uint16_t>(L.wc[2]), 256, act(A_PRE4), 256, 0, gam(3), bet(3));
    ck(pf::launch_gn_enc(act(A_PRE4), n, H / 8, W / 8, 256, stats, sc + 224, act(A_ZC4), 256, nullptr, s), "level 4");
    // ---- decoder
    if (rc == PF_OK)
        rc = conv_tc(u, pf::CONV3, act(A_ZC4), H / 8, W / 8, 256, u->at<uint16_t>(L.wc[3]), 256, act(A_PRE4), 256, 0, gam(4), bet(4));
    ck(pf::launch_gn_dec(act(A_PRE4), n, H / 8, W / 8, 256, stats, act(A_H4), s), "decoder 4");
    if (rc == PF_OK) rc = conv_tc(u, pf::TCONV, act(A_H4), H / 8, W / 8, 256, u->at<uint16_t>(L.wt[0]), 128, act(A_CAT3), 256, 128);
    if (rc == PF_OK)
        rc = conv_tc(u, pf::CONV3, act(A_CAT3), H / 4, W / 4, 256, u->at<uint16_t>(L.wc[4]), 128, act(A_PRE3), 128, 0, gam(5), bet(5));
    ck(pf::launch_gn_dec(act(A_PRE3), n, H / 4, W / 4, 128, stats, act(A_H3), s), "decoder 3");
    if (rc == PF_OK) rc = conv_tc(u, pf::TCONV, act(A_H3), H / 4, W / 4, 128, u->at<uint16_t>(L.wt[1]), 64, act(A_CAT2), 128, 64);
    if (rc == PF_OK)
        rc = conv_tc(u, pf::CONV3, act(A_CAT2), H / 2, W / 2, 128, u->at<uint16_t>(L.wc[5]), 64, act(A_PRE2), 64, 0, gam(6), bet(6));
    ck(pf::launch_gn_dec(act(A_PRE2), n, H / 2, W / 2, 64, stats, act(A_H2), s), "decoder 2");
    if (rc == PF_OK) rc = conv_tc(u, pf::TCONV, act(A_H2), H / 2, W / 2, 64, u->at<uint16_t>(L.wt[2]), 32, act(A_CAT1), 64, 32);
    if (rc == PF_OK)
        rc = conv_tc(u, pf::CONV3, act(A_CAT1), H, W, 64, u->at<uint16_t>(L.wc[6]), 32, act(A_PRE1), 32, 0, gam(7), bet(7));
    ck(pf::launch_gn_dec(act(A_PRE1), n, H, W, 32, stats, act(A_H1), s), "decoder 1");
    // ---- output: conv 32 -> 3 on the tensor cores, added as affine increments to the DNS fields
    if (rc == PF_OK) {
        pf::ConvArgs a = {};
        a.n = n;
        a.h = H;
        a.w = W;
        a.cin = 32;
        a.cout = 16;
        a.groups = G;
        a.err = u->at<int>(L.err);
        a.wait_cap = 1 << 22;
        a.fields = dp;
        a.fpitch = pitch;
        a.ogamma = gam(8);
        a.obeta = bet(8);
        ck(pf::launch_umma_conv(pf::OUT3, act(A_H1), u->at<uint16_t>(L.wout), a, s), "output");
    }
    return rc;
}

int pf_unet_frame(pf_unet* u, int n, const float* const* phi, const float* const* c, const float* const* rho,
                  int pitch)
{
    if (!u || !phi || !c || !rho) return ufail(PF_ERR_ARG, "null pointer");
    if (n != u->n) return ufail(PF_ERR_ARG, "batch %d, the handle was built for %d", n, u->n);
    if (pitch < u->w) return ufail(PF_ERR_LAYOUT, "pitch %d < nx %d", pitch, u->w);
    for (int i = 0; i < n; ++i) {
        if (!phi[i] || !c[i] || !rho[i]) return ufail(PF_ERR_ARG, "run %d: null field", i);
        u->fptrs[i] = phi[i];
        u->fptrs[n + i] = c[i];
        u->fptrs[2 * n + i] = rho[i];
    }
    cudaError_t e = cudaMemcpyAsync(u->base + u->L.fptrs, u->fptrs.data(), sizeof(float*) * 3 * n,
                                    cudaMemcpyHostToDevice, u->stream);
    if (e != cudaSuccess) return ufail(PF_ERR_CUDA, "frame pointer table: %s", cudaGetErrorString(e));
    const float** dp = u->at<const float*>(u->L.fptrs);
    const int slot = u->frames == 0 ? 0 : 1 - u->newest;  // overwrite the oldest frame held
    const size_t frame_elems = (size_t)n * 3 * u->h * u->w;
    e = pf::launch_frame(dp, dp + n, dp + 2 * n, pitch, n, u->h, u->w,
                         u->at<float>(u->L.ring) + (size_t)slot * frame_elems, u->stream);
    if (e != cudaSuccess) return ufail(PF_ERR_CUDA, "frame: %s", cudaGetErrorString(e));
    u->newest = slot;
    if (u->frames < pf::UNET_LB - 1) ++u->frames;
    return PF_OK;
}

int pf_unet_reset_frames(pf_unet* u)
{
    if (!u) return ufail(PF_ERR_ARG, "null handle");
    u->frames = 0;
    u->newest = 0;
    return PF_OK;
}

int pf_unet_sync(pf_unet* u)
{
    if (!u) return ufail(PF_ERR_ARG, "null handle");
    int err = 0;
    cudaError_t e = cudaStreamSynchronize(u->stream);
    if (e == cudaSuccess) e = cudaMemcpy(&err, u->base + u->L.err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return ufail(PF_ERR_CUDA, "U-Net sync: %s", cudaGetErrorString(e));
    if (err & pf::UNET_ERR_TIMEOUT) return ufail(PF_ERR_TIMEOUT, "a bounded tensor-core pipeline wait ran out");
    return PF_OK;
}

int pf_unet_check(pf_unet* u, double phi_lo, double phi_hi, double c_lo, double c_hi, double rho_lo, double rho_hi,
                  int* ok)
{
    if (!u || !ok) return ufail(PF_ERR_ARG, "null pointer");
    const int n = u->n;
    int* flags = u->at<int>(u->L.flags);
    cudaError_t e = cudaMemsetAsync(flags, 0, sizeof(int) * n, u->stream);
    float** dp = u->at<float*>(u->L.ptrs);  // the fields of the last jump
    if (e == cudaSuccess)
        e = pf::launch_check(dp, dp + n, dp + 2 * n, n, u->h, u->w, u->last_pitch, (float)phi_lo, (float)phi_hi,
                             (float)c_lo, (float)c_hi, (float)rho_lo, (float)rho_hi, flags, u->stream);
    std::vector<int> f(n, 1);
    if (e == cudaSuccess) e = cudaMemcpyAsync(f.data(), flags, sizeof(int) * n, cudaMemcpyDeviceToHost, u->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(u->stream);
    if (e != cudaSuccess) return ufail(PF_ERR_CUDA, "plausibility check: %s", cudaGetErrorString(e));
    for (int i = 0; i < n; ++i) ok[i] = f[i] ? 0 : 1;
    return PF_OK;
}

int pf_unet_buffer(const pf_unet* u, int which, void** ptr, int* channels)
{
    if (!u || !ptr || !channels || which < 0 || which > 14) return ufail(PF_ERR_ARG, "bad buffer query");
    const int ch[16] = {32, 64, 32, 64, 128, 64, 128, 256, 128, 256, 256, 256, 128, 64, 32, 2};
    *ptr = u->base + u->L.act[which];
    *channels = ch[which];
    return PF_OK;
}

int pf_unet_destroy(pf_unet* u)
{
    if (!u) return PF_OK;
    cudaError_t e = cudaStreamSynchronize(u->stream);
    delete u;
    if (e != cudaSuccess) return ufail(PF_ERR_CUDA, "stream synchronize: %s", cudaGetErrorString(e));
    return PF_OK;
}

const char* pf_unet_last_error(void) { return g_unet_error.c_str(); }

}  // extern "C"
