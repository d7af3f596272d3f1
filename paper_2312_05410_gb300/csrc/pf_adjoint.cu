// Hand-written discrete adjoint of the explicit midpoint step (declarations in
// include/pf.h: pf_adjoint).  It gives the exact gradient, through every time
// step of the scheme the forward kernel runs (Materials and Methods equations,
// "Dataset": central differences, explicit midpoint), of a linear functional
// of the final state, L = sum(w . u_N), with respect to the initial fields
// and to three parameters: the incident speed V (deposition rate), a factor on
// the composition mobility (M_c -> s M_c, at s = 1) and kappa_c.  dt is fixed.
//
// For one step u' = u + dt R(u*), u* = u + dt/2 R(u), with w' the cotangent of u':
//   w* = dt J_R(u*)^T w'
//   w  = w' + w* + dt/2 J_R(u)^T w*
//   theta_bar += dt (dR/dtheta)(u*)^T w' + dt/2 (dR/dtheta)(u)^T w*.
// J_R(v)^T x is evaluated by two gather kernels.  Pass A, per cell: the
// cotangents of the chemical potentials, of the mobility and of the source,
//   mu_c_bar = div_M(x_c) (the flux operator is self-adjoint),
//   M_bar = -1/(2dx^2) sum_faces (mu_nb - mu)(x_nb - x),
//   mu_phi_bar = M_phi L(x_phi) (Allen-Cahn form: -L_phi x_phi), s_bar = x_phi - x_rho,
// and the parameter partials.  Pass B, per cell: the cotangents of phi, c, rho
// from the pointwise derivatives and the transposed stencils.
// Boundary rules of the transposes (the forward copies boundary values into
// ghost rows): operands of symmetric stencils (Laplacians, flux divergence)
// take mirrored ghosts; weights of the central y-difference take negated
// ghosts (mirror fields) or zero (rho's fixed reservoir value above the top);
// rho's Laplacian takes a zero ghost above the top.
//
// Checkpointing: the forward stores the state every K steps; the backward
// recomputes each segment's K states from its checkpoint with the fused step
// kernel, then walks them in reverse.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <string>
#include <vector>

#include "pf.h"
#include "pf_internal.h"

namespace pf {
namespace {

constexpr int ADJ_THREADS = 256;
constexpr int ADJ_MAX_BLOCKS = 8192;

struct AdjConst {
    StepConst k;
    float idx2;            // 1 / dx^2
    float cx, cy;          // dR/dV scaling: (cos a, -sin a) / (2 dx), zero without deposition
    float MAb, MBb, MAs, MBs, isig2;
    int phi_mode;
};

// Field access with the forward's ghost rules: x periodic; phi and c reflected
// (mirror); rho mirrored at the bottom, rho_top above the top.
// (Offsets are at most 2 cells, so one correction suffices unless the grid is tinier than that.)
__device__ __forceinline__ int wrapx(int i, int nx)
{
    if (nx > 2) return i < 0 ? i + nx : (i >= nx ? i - nx : i);
    i %= nx;
    return i < 0 ? i + nx : i;
}
__device__ __forceinline__ int refl(int j, int ny)
{
    if (ny > 2) return j < 0 ? -1 - j : (j >= ny ? 2 * ny - 1 - j : j);
    for (int it = 0; it < 4 && (j < 0 || j >= ny); ++it) j = j < 0 ? -1 - j : 2 * ny - 1 - j;
    return j < 0 ? 0 : (j >= ny ? ny - 1 : j);
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// The passes work on tiles of ATX x ATY cells.  Each block stages, for its tile and a one-cell
// halo, every operand the stencils read into shared memory.  A halo cell (gj, gi) holds the value
// at the reflected row and wrapped column, exactly what the forward's ghost rules read there.
// The rules that are not copies (rho_top above the top, the negated or zero ghosts of the
// transposes) are applied where the value is used, from the neighbour's global row.
constexpr int ATX = 32, ATY = ADJ_THREADS / ATX;
constexpr int AW = ATX + 2, AH = ATY + 2;

// Fill the staged tile of `nf` fields (rows j0-1 .. j0+ATY, columns i0-1 .. i0+ATX); cells
// beyond the first halo ring outside the grid are never read and hold 0.
template <int NF>
__device__ __forceinline__ void stage_tile(float (*S)[AH][AW], const float* const* f, int j0, int i0, int nx, int ny,
                                           int pitch)
{
    for (int e = threadIdx.x; e < AH * AW; e += ADJ_THREADS) {
        const int r = e / AW, cc = e - r * AW;
        const int gj = j0 - 1 + r, gi = i0 - 1 + cc;
        const bool ok = gj >= -1 && gj <= ny && gi >= -1 && gi <= nx;
        const size_t src = ok ? (size_t)refl(gj, ny) * pitch + wrapx(gi, nx) : 0;
#pragma unroll
        for (int q = 0; q < NF; ++q) S[q][r][cc] = ok ? f[q][src] : 0.f;
    }
}

// Pass A. x: cotangent (phi, c, rho); v: state. Writes mu_c_bar, M_bar, mu_phi_bar, s_bar and
// adds the block's parameter partials {V, m_scale, kappa_c} (FP64, fixed order) to its slot.
// The chemical potential and mobility of the state are computed here for the tile and its
// one-cell halo, from phi and c staged with a two-cell halo: a halo cell beyond the top or
// bottom takes the value of the cell it mirrors (computed there, with the same stencil and
// summation order), and one beyond the left or right edge is the periodic translate.
constexpr int BW2 = ATX + 4, BH2 = ATY + 4;
__global__ void __launch_bounds__(ADJ_THREADS)
vjp_a_kernel(const AdjConst a, const float* __restrict__ vphi, const float* __restrict__ vc,
             const float* __restrict__ vrho, const float* __restrict__ xphi, const float* __restrict__ xc,
             const float* __restrict__ xrho, float* __restrict__ muc_bar, float* __restrict__ M_bar,
             float* __restrict__ muf_bar, float* __restrict__ s_bar, double* __restrict__ partials, double pscale)
{
    __shared__ float S2[2][BH2][BW2];  // vphi, vc with a two-cell halo
    __shared__ float S[5][AH][AW];     // muc, Mc (computed), xc, xphi, vrho
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int nx = a.k.nx, ny = a.k.ny, pitch = a.k.pitch;
    const int ntx = (nx + ATX - 1) / ATX, ntiles = ntx * ((ny + ATY - 1) / ATY);
    const int tx = threadIdx.x % ATX, ty = threadIdx.x / ATX;
    const float* const fl[3] = {xc, xphi, vrho};
    double accV = 0.0, accM = 0.0, accK = 0.0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int j0 = (tile / ntx) * ATY, i0 = (tile % ntx) * ATX;
        __syncthreads();  // the previous tile's readers are done
        for (int e = threadIdx.x; e < BH2 * BW2; e += ADJ_THREADS) {
            const int r = e / BW2, cc = e - r * BW2;
            const int gj = j0 - 2 + r, gi = i0 - 2 + cc;
            const bool ok = gj >= -2 && gj <= ny + 1 && gi >= -2 && gi <= nx + 1;
            const size_t src = ok ? (size_t)refl(gj, ny) * pitch + wrapx(gi, nx) : 0;
            S2[0][r][cc] = ok ? vphi[src] : 0.f;
            S2[1][r][cc] = ok ? vc[src] : 0.f;
        }
        {
            float (*Sx)[AH][AW] = &S[2];
            stage_tile<3>(Sx, fl, j0, i0, nx, ny, pitch);
        }
        __syncthreads();
        // mu_c and M_c on the tile and its halo (rows j0-1 .. j0+ATY, columns i0-1 .. i0+ATX)
        for (int e = threadIdx.x; e < AH * AW; e += ADJ_THREADS) {
            const int r = e / AW, cc = e - r * AW;
            const int gj = j0 - 1 + r, gi = i0 - 1 + cc;
            float muc = 0.f, Mc = 0.f;
            if (gj >= -1 && gj <= ny && gi >= -1 && gi <= nx) {
                const int y2 = refl(gj, ny) - (j0 - 2), x2 = cc + 1;  // stencil centre in S2
                const float f = S2[0][y2][x2], c0 = S2[1][y2][x2];
                const float sc = S2[1][y2][x2 + 1] + S2[1][y2][x2 - 1] + S2[1][y2 + 1][x2] + S2[1][y2 - 1][x2];
                const float P = 0.25f * (2.f - f) * (1.f + f) * (1.f + f);
                const float dg = 2.f * c0 * (1.f - c0) * (1.f - 2.f * c0);
                muc = P * a.k.Wc * dg - a.k.kc * (sc - 4.f * c0);
                const float h = c0 * c0 * (3.f - 2.f * c0);
                Mc = P * (h * a.MAb + (1.f - h) * a.MBb);
                if (a.MAs != 0.f || a.MBs != 0.f) Mc += expf(-f * f * a.isig2) * (h * a.MAs + (1.f - h) * a.MBs);
            }
            S[0][r][cc] = muc;
            S[1][r][cc] = Mc;
        }
        __syncthreads();
        const int j = j0 + ty, i = i0 + tx;
        if (j >= ny || i >= nx) continue;
        const size_t o = (size_t)j * pitch + i;
        const int y = ty + 1, x = tx + 1;  // staged position of (j, i)
        auto at = [&](int q, int dj, int di) { return S[q][y + dj][x + di]; };
        auto at2 = [&](int q, int dj, int di) { return S2[q][y + 1 + dj][x + 1 + di]; };
        const int dj4[4] = {0, 0, 1, -1}, di4[4] = {1, -1, 0, 0};
        const float m0 = at(0, 0, 0), M0 = at(1, 0, 0);
        const float wc = at(2, 0, 0);
        float mub = 0.f, Mb = 0.f, Rc = 0.f;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            // a ghost neighbour is the mirror copy: its mu and M equal the boundary cell's
            const float mn = at(0, dj4[q], di4[q]), Mn = at(1, dj4[q], di4[q]);
            const float dw = at(2, dj4[q], di4[q]) - wc;
            mub += (M0 + Mn) * dw;
            Mb -= (mn - m0) * dw;
            Rc += (M0 + Mn) * (mn - m0);
        }
        mub *= a.k.cR;
        Mb *= a.k.cR;
        Rc *= a.k.cR;
        const float wf = at(3, 0, 0), wr = xrho[o];
        float mfb;
        if (a.phi_mode == 0) {
            const float s = at(3, 0, 1) + at(3, 0, -1) + at(3, 1, 0) + at(3, -1, 0);
            mfb = a.k.cF * (s - 4.f * wf);
        } else {
            mfb = a.k.cF * wf;
        }
        const float sb = wf - wr;
        muc_bar[o] = mub;
        M_bar[o] = Mb;
        muf_bar[o] = mfb;
        s_bar[o] = sb;
        // parameter partials
        const float c0 = at2(1, 0, 0), r0 = at(4, 0, 0);
        const float Lc = at2(1, 0, 1) + at2(1, 0, -1) + at2(1, 1, 0) + at2(1, -1, 0) - 4.f * c0;
        accK -= (double)mub * (double)(Lc * a.idx2);  // d mu_c / d kappa_c = -L(c)
        accM += (double)wc * (double)Rc;
        const float dfx = at2(0, 0, 1) - at2(0, 0, -1);
        const float dfy = at2(0, 1, 0) - at2(0, -1, 0);
        // rho above the top is the reservoir value
        auto rh = [&](int dj, int di) { return j + dj >= ny ? a.k.rho_top : at(4, dj, di); };
        const float drx = rh(0, 1) - rh(0, -1);
        const float dry = rh(1, 0) - rh(-1, 0);
        accV += (double)(sb * r0 * (a.cx * dfx + a.cy * dfy)) - (double)(wr * (a.cx * drx + a.cy * dry));
    }
    // Block sum in a fixed order, added (scaled) to this block's own accumulator slot: the slots
    // collect every call of the adjoint in the same order whatever the checkpoint interval, and
    // are summed once, in a fixed order, at the end (adj_sum_kernel).
    __shared__ double red[3][ADJ_THREADS / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    accV = warp_sum(accV);
    accM = warp_sum(accM);
    accK = warp_sum(accK);
    if (lane == 0) {
        red[0][w] = accV;
        red[1][w] = accM;
        red[2][w] = accK;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        const int q = threadIdx.x;
        double s = 0.0;
        for (int t = 0; t < ADJ_THREADS / 32; ++t) s += red[q][t];
        partials[(size_t)q * gridDim.x + blockIdx.x] += pscale * s;
    }
}

// acc[q] = sum over the blocks' accumulator slots (fixed order: strided per thread, then the
// warp butterfly, then the warps in order).  One block.
__global__ void __launch_bounds__(ADJ_THREADS) adj_sum_kernel(const double* __restrict__ partials, int nb,
                                                               double* __restrict__ acc)
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    __shared__ double red[3][ADJ_THREADS / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int q = 0; q < 3; ++q) {
        double t = 0.0;
        for (int b = threadIdx.x; b < nb; b += ADJ_THREADS) t += partials[(size_t)q * nb + b];
        t = warp_sum(t);
        if (lane == 0) red[q][w] = t;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double t = 0.0;
        for (int i = 0; i < ADJ_THREADS / 32; ++i) t += red[threadIdx.x][i];
        acc[threadIdx.x] = t;
    }
}

// Pass B. out = base1 + base2 + scale * J_R(v)^T x, from pass A's fields; base1/base2 may be NULL.
__global__ void __launch_bounds__(ADJ_THREADS)
vjp_b_kernel(const AdjConst a, const float* __restrict__ vphi, const float* __restrict__ vc,
             const float* __restrict__ vrho, const float* __restrict__ xrho, const float* __restrict__ muc_bar,
             const float* __restrict__ M_bar, const float* __restrict__ muf_bar, const float* __restrict__ s_bar,
             float scale, const float* __restrict__ b1phi, const float* __restrict__ b1c,
             const float* __restrict__ b1rho, const float* __restrict__ b2phi, const float* __restrict__ b2c,
             const float* __restrict__ b2rho, float* __restrict__ ophi, float* __restrict__ oc,
             float* __restrict__ orho)
{
    __shared__ float S[6][AH][AW];  // muc_bar, muf_bar, vrho, s_bar, vphi, xrho
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int nx = a.k.nx, ny = a.k.ny, pitch = a.k.pitch;
    const int ntx = (nx + ATX - 1) / ATX, ntiles = ntx * ((ny + ATY - 1) / ATY);
    const int tx = threadIdx.x % ATX, ty = threadIdx.x / ATX;
    const float* const fl[6] = {muc_bar, muf_bar, vrho, s_bar, vphi, xrho};
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int j0 = (tile / ntx) * ATY, i0 = (tile % ntx) * ATX;
        __syncthreads();  // the previous tile's readers are done
        stage_tile<6>(S, fl, j0, i0, nx, ny, pitch);
        __syncthreads();
        const int j = j0 + ty, i = i0 + tx;
        if (j >= ny || i >= nx) continue;
        const size_t o = (size_t)j * pitch + i;
        const int y = ty + 1, x = tx + 1;
        auto at = [&](int q, int dj, int di) { return S[q][y + dj][x + di]; };
        const float f = at(4, 0, 0), cc = vc[o];
        const float P = 0.25f * (2.f - f) * (1.f + f) * (1.f + f);
        const float dP = 0.75f * (1.f - f * f);
        const float d2P = -1.5f * f;
        const float g = cc * cc * (1.f - cc) * (1.f - cc);
        const float dg = 2.f * cc * (1.f - cc) * (1.f - 2.f * cc);
        const float d2g = 2.f - 12.f * cc + 12.f * cc * cc;
        const float h = cc * cc * (3.f - 2.f * cc);
        const float dh = 6.f * cc * (1.f - cc);
        float dMdf = dP * (h * a.MAb + (1.f - h) * a.MBb);
        float dMdc = P * (a.MAb - a.MBb) * dh;
        if (a.MAs != 0.f || a.MBs != 0.f) {
            const float e = expf(-f * f * a.isig2);
            dMdf += -2.f * f * a.isig2 * e * (h * a.MAs + (1.f - h) * a.MBs);
            dMdc += e * (a.MAs - a.MBs) * dh;
        }
        const float mub = at(0, 0, 0), mfb = at(1, 0, 0), Mb = M_bar[o];
        // neighbour sums of the mirrored cotangents (symmetric Laplacians)
        const float Lmub = at(0, 0, 1) + at(0, 0, -1) + at(0, 1, 0) + at(0, -1, 0) - 4.f * mub;
        const float Lmfb = at(1, 0, 1) + at(1, 0, -1) + at(1, 1, 0) + at(1, -1, 0) - 4.f * mfb;
        float cb = a.k.Wc * P * d2g * mub - a.k.kc * Lmub + dP * a.k.Wc * dg * mfb + dMdc * Mb;
        const float fpp = a.k.Wf * (3.f * f * f - 1.f) + d2P * a.k.Wc * g;
        float fb = a.k.Wc * dP * dg * mub + fpp * mfb - a.k.kf * Lmfb + dMdf * Mb;
        // transposed central differences of phi in the source: weights a = (ax, ay) rho s_bar
        auto aw = [&](int dj, int di) {  // weight at a neighbour; y-ghosts negated (mirror field)
            const float sgn = (j + dj < 0 || j + dj >= ny) ? -1.f : 1.f;
            return sgn * at(2, dj, di) * at(3, dj, di);
        };
        fb += a.k.ax * (aw(0, -1) - aw(0, 1)) + a.k.ay * (aw(-1, 0) - aw(1, 0));
        // rho: source factor, diffusion with the transposed boundary rules, transposed advection
        const float sb = at(3, 0, 0);
        const float dfx = at(4, 0, 1) - at(4, 0, -1);
        const float dfy = at(4, 1, 0) - at(4, -1, 0);
        float rb = sb * (a.k.ax * dfx + a.k.ay * dfy);
        auto wr_lap = [&](int dj, int di) {  // mirrored below, zero above the top
            if (j + dj >= ny) return 0.f;
            return at(5, dj, di);
        };
        auto wr_dy = [&](int dj, int di) {  // negated below, zero above the top
            if (j + dj >= ny) return 0.f;
            const float v = at(5, dj, di);
            return j + dj < 0 ? -v : v;
        };
        const float wr0 = at(5, 0, 0);
        rb += a.k.cD * (wr_lap(0, 1) + wr_lap(0, -1) + wr_lap(1, 0) + wr_lap(-1, 0) - 4.f * wr0);
        rb -= a.k.ax * (wr_lap(0, -1) - wr_lap(0, 1)) + a.k.ay * (wr_dy(-1, 0) - wr_dy(1, 0));
        float of = scale * fb, oc_ = scale * cb, orr = scale * rb;
        if (b1phi) {
            of += b1phi[o];
            oc_ += b1c[o];
            orr += b1rho[o];
        }
        if (b2phi) {
            of += b2phi[o];
            oc_ += b2c[o];
            orr += b2rho[o];
        }
        ophi[o] = of;
        oc[o] = oc_;
        orho[o] = orr;
    }
}

int adj_blocks(int nx, int ny)
{
    // one block per ATX x ATY tile (one thread per cell) up to the cap
    long long b = (long long)((nx + ATX - 1) / ATX) * ((ny + ATY - 1) / ATY);
    return (int)(b < 1 ? 1 : (b > ADJ_MAX_BLOCKS ? ADJ_MAX_BLOCKS : b));
}

}  // namespace
}  // namespace pf

namespace {

thread_local std::string g_adj_error;

int afail(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_adj_error = buf;
    return code;
}

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

struct AdjLayout {
    size_t plane;   // bytes of one field plane
    size_t pp;      // ping-pong (2 x 3 planes)
    size_t ckpt;    // (nseg + 1) x 3 planes
    size_t seg;     // K x 3 planes
    size_t lam;     // 3 cotangents x 3 planes
    size_t ustar;   // 3 planes
    size_t scratch; // 4 planes (the pass-A fields mu_c_bar, M_bar, mu_phi_bar, s_bar)
    size_t partials, acc, total;
};

bool adj_layout(int nx, int ny, int pitch, long nsteps, int K, AdjLayout& L)
{
    if (nx < 1 || ny < 1 || pitch < nx || nsteps < 0 || K < 1) return false;
    const long nseg = (nsteps + K - 1) / K;
    L.plane = a256(size_t(ny) * size_t(pitch) * sizeof(float));
    size_t off = 0;
    L.pp = off;
    off += 6 * L.plane;
    L.ckpt = off;
    off += size_t(nseg + 1) * 3 * L.plane;
    L.seg = off;
    off += size_t(K) * 3 * L.plane;
    L.lam = off;
    off += 9 * L.plane;
    L.ustar = off;
    off += 3 * L.plane;
    L.scratch = off;
    off += 4 * L.plane;
    L.partials = off;
    off = a256(off + 3 * size_t(pf::adj_blocks(nx, ny)) * sizeof(double));
    L.acc = off;
    off = a256(off + 3 * sizeof(double) + sizeof(unsigned));  // the three parameter gradients (+ padding)
    L.total = off;
    return true;
}

}  // namespace

extern "C" {

size_t pf_adjoint_workspace_size(int nx, int ny, int pitch, long nsteps, int K)
{
    AdjLayout L;
    return adj_layout(nx, ny, pitch, nsteps, K, L) ? L.total : 0;
}

int pf_adjoint(const pf_params* p, int nx, int ny, int pitch, const float* phi0, const float* c0, const float* rho0,
               long nsteps, int K, const float* w_phi, const float* w_c, const float* w_rho, float* g_phi0,
               float* g_c0, float* g_rho0, double* g_params, float* final_phi, float* final_c, float* final_rho,
               void* work, size_t work_bytes, void* stream)
{
    pf::TraceRange trace("pf_adjoint");
    using namespace pf;
    if (!p || !phi0 || !c0 || !rho0 || !w_phi || !w_c || !g_phi0 || !g_c0 || !g_rho0 || !g_params || !work)
        return afail(PF_ERR_ARG, "null pointer");
    if (nx < 1 || ny < 1 || nx > (1 << 20) || ny > (1 << 20)) return afail(PF_ERR_ARG, "bad grid size");
    if (pitch < nx || pitch % 4) return afail(PF_ERR_LAYOUT, "bad pitch");
    if (nsteps < 0 || K < 1) return afail(PF_ERR_ARG, "need nsteps >= 0 and K >= 1");
    if (reinterpret_cast<uintptr_t>(work) % 256) return afail(PF_ERR_LAYOUT, "workspace must be 256-byte aligned");
    if (!(p->dx > 0.0) || (p->phi_mode != 0 && p->phi_mode != 1)) return afail(PF_ERR_ARG, "bad dx or phi_mode");
    if ((p->MA_surf != 0.0 || p->MB_surf != 0.0) && !(p->sigma_surf > 0.0))
        return afail(PF_ERR_ARG, "sigma_surf must be positive");
    double lim[4];
    pf_dt_limit(p, lim);
    if (!(p->dt > 0.0) || p->dt > lim[0] * (1.0 + 1e-12)) return afail(PF_ERR_UNSTABLE, "dt outside the limit");
    AdjLayout L;
    if (!adj_layout(nx, ny, pitch, nsteps, K, L)) return afail(PF_ERR_ARG, "bad sizes");
    if (work_bytes < L.total) return afail(PF_ERR_LAYOUT, "workspace of %zu bytes, %zu needed", work_bytes, L.total);

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char* w = static_cast<char*>(work);
    auto planes = [&](size_t off) {
        float* b = reinterpret_cast<float*>(w + off);
        const size_t pl = L.plane / sizeof(float);
        return std::vector<float*>{b, b + pl, b + 2 * pl};
    };
    const size_t pl = L.plane / sizeof(float);
    const StepConst k = step_const_of(*p, nx, ny, pitch);
    StepConst khalf = k;
    khalf.dt = float(0.5 * p->dt);
    const int mob = mob_kind_of(*p), tile = choose_tile(nx, ny);
    AdjConst ac{};
    ac.k = k;
    ac.idx2 = float(1.0 / (p->dx * p->dx));
    double vxu = 0.0, vyu = 0.0;
    if (p->deposition) {
        const double ang = p->v_angle_deg * (M_PI / 180.0);
        vxu = std::cos(ang);
        vyu = -std::sin(ang);
    }
    ac.cx = float(vxu / (2.0 * p->dx));
    ac.cy = float(vyu / (2.0 * p->dx));
    ac.MAb = float(p->MA_bulk);
    ac.MBb = float(p->MB_bulk);
    ac.MAs = float(p->MA_surf);
    ac.MBs = float(p->MB_surf);
    ac.isig2 = p->sigma_surf > 0.0 ? float(1.0 / (p->sigma_surf * p->sigma_surf)) : 0.f;
    ac.phi_mode = p->phi_mode;
    const int nb = adj_blocks(nx, ny);
    double* partials = reinterpret_cast<double*>(w + L.partials);
    double* acc = reinterpret_cast<double*>(w + L.acc);
    const long nseg = (nsteps + K - 1) / K;

    cudaError_t e = cudaSuccess;
    // field copies move the nx model columns only (padding columns are left as they are)
    auto copy3 = [&](float* const* dst, const float* const* src) {
        for (int q = 0; q < 3 && e == cudaSuccess; ++q)
            e = cudaMemcpy2DAsync(dst[q], size_t(pitch) * sizeof(float), src[q], size_t(pitch) * sizeof(float),
                                  size_t(nx) * sizeof(float), size_t(ny), cudaMemcpyDeviceToDevice, s);
    };
    auto ckpt = [&](long i) { return planes(L.ckpt + size_t(i) * 3 * L.plane); };
    auto segst = [&](long i) { return planes(L.seg + size_t(i) * 3 * L.plane); };
    auto step = [&](const std::vector<float*>& a, const std::vector<float*>& b) {
        if (e == cudaSuccess) e = launch_step(k, tile, p->phi_mode, mob, a[0], a[1], a[2], b[0], b[1], b[2], s);
    };
    // ---- forward: checkpoints at multiples of K, final state
    {
        const float* init[3] = {phi0, c0, rho0};
        std::vector<float*> c0v = ckpt(0);
        copy3(c0v.data(), init);
        std::vector<float*> A = planes(L.pp), B = {A[0] + 3 * pl, A[1] + 3 * pl, A[2] + 3 * pl};
        std::vector<float*> cur = c0v;
        for (long t = 0; t < nsteps && e == cudaSuccess; ++t) {
            std::vector<float*> dst = ((t + 1) % K == 0) ? ckpt((t + 1) / K) : ((cur == A) ? B : A);
            step(cur, dst);
            cur = dst;
        }
        if (final_phi && final_c && final_rho && e == cudaSuccess) {
            float* fin[3] = {final_phi, final_c, final_rho};
            const float* src[3] = {cur[0], cur[1], cur[2]};
            copy3(fin, src);
        }
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(acc, 0, 3 * sizeof(double) + sizeof(unsigned), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(partials, 0, 3 * size_t(nb) * sizeof(double), s);
    // ---- backward
    std::vector<float*> lamA = planes(L.lam), lamB = planes(L.lam + 3 * L.plane), lamS = planes(L.lam + 6 * L.plane);
    std::vector<float*> us = planes(L.ustar);
    float* sc = reinterpret_cast<float*>(w + L.scratch);
    float *muc_b = sc, *M_b = sc + pl, *muf_b = sc + 2 * pl, *s_b = sc + 3 * pl;
    // cotangent buffers start at zero (also a zero rho cotangent when none is given)
    if (e == cudaSuccess) e = cudaMemsetAsync(lamA[0], 0, 9 * L.plane, s);
    {
        const float* wsrc[3] = {w_phi, w_c, w_rho};
        for (int q = 0; q < 3 && e == cudaSuccess; ++q)
            if (wsrc[q])
                e = cudaMemcpy2DAsync(lamA[q], size_t(pitch) * sizeof(float), wsrc[q], size_t(pitch) * sizeof(float),
                                      size_t(nx) * sizeof(float), size_t(ny), cudaMemcpyDeviceToDevice, s);
    }
    std::vector<float*> lam = lamA;
    auto vjp = [&](const std::vector<float*>& v, const std::vector<float*>& x, double pscale, float scale,
                   const std::vector<float*>* b1, const std::vector<float*>* b2, const std::vector<float*>& out) {
        if (e != cudaSuccess) return;
        // programmatic dependent launch: each kernel waits for its predecessor before reading
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(nb);
        cfg.blockDim = dim3(ADJ_THREADS);
        cfg.stream = s;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        const float* nil = nullptr;
        e = cudaLaunchKernelEx(&cfg, vjp_a_kernel, ac, (const float*)v[0], (const float*)v[1], (const float*)v[2],
                               (const float*)x[0], (const float*)x[1], (const float*)x[2], muc_b, M_b, muf_b, s_b,
                               partials, pscale);
        if (e == cudaSuccess)
            e = cudaLaunchKernelEx(&cfg, vjp_b_kernel, ac, (const float*)v[0], (const float*)v[1],
                                   (const float*)v[2], (const float*)x[2], (const float*)muc_b, (const float*)M_b,
                                   (const float*)muf_b, (const float*)s_b, scale, b1 ? (const float*)(*b1)[0] : nil,
                                   b1 ? (const float*)(*b1)[1] : nil, b1 ? (const float*)(*b1)[2] : nil,
                                   b2 ? (const float*)(*b2)[0] : nil, b2 ? (const float*)(*b2)[1] : nil,
                                   b2 ? (const float*)(*b2)[2] : nil, out[0], out[1], out[2]);
    };
    const double dt = p->dt;
    // One segment: recompute its states from segst(0), then walk them backwards.  The cotangent
    // starts and ends in lamA (an odd length ends with a copy), so a full segment has fixed
    // pointers and is captured once as a CUDA graph and replayed for every full segment.
    auto segment_body = [&](long len) {
        for (long i = 1; i < len && e == cudaSuccess; ++i) step(segst(i - 1), segst(i));
        std::vector<float*> l = lamA, ln = lamB;
        for (long i = len - 1; i >= 0 && e == cudaSuccess; --i) {
            const std::vector<float*> u = segst(i);
            // u* = u + dt/2 R(u)
            e = launch_euler(khalf, p->phi_mode, mob, u[0], u[1], u[2], us[0], us[1], us[2], s);
            // w* = dt J(u*)^T w'
            vjp(us, l, dt, float(dt), nullptr, nullptr, lamS);
            // w = w' + w* + dt/2 J(u)^T w*
            vjp(u, lamS, 0.5 * dt, float(0.5 * dt), &l, &lamS, ln);
            std::swap(l, ln);
        }
        if (l != lamA) {
            const float* src[3] = {l[0], l[1], l[2]};
            copy3(lamA.data(), src);
        }
    };
    cudaGraphExec_t gseg = nullptr;
    const long full = nsteps / K;  // segments of exactly K steps
    if (full >= 2 && e == cudaSuccess) {
        cudaStream_t real = s;
        cudaStream_t cap;
        e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        if (e == cudaSuccess) {
            s = cap;
            e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                segment_body(K);
                cudaGraph_t g = nullptr;
                cudaError_t e2 = cudaStreamEndCapture(cap, &g);
                if (e == cudaSuccess) e = e2;
                if (e == cudaSuccess) e = cudaGraphInstantiate(&gseg, g, 0);
                if (g) cudaGraphDestroy(g);
            }
            s = real;
            cudaStreamDestroy(cap);
        }
    }
    for (long sg = nseg - 1; sg >= 0 && e == cudaSuccess; --sg) {
        const long t0 = sg * K, len = std::min<long>(K, nsteps - t0);
        {
            std::vector<float*> c = ckpt(sg), s0 = segst(0);
            const float* src[3] = {c[0], c[1], c[2]};
            copy3(s0.data(), src);
        }
        if (gseg && len == K)
            e = cudaGraphLaunch(gseg, s);
        else
            segment_body(len);
    }
    if (gseg) cudaGraphExecDestroy(gseg);
    lam = lamA;
    if (e == cudaSuccess) {
        float* g[3] = {g_phi0, g_c0, g_rho0};
        const float* src[3] = {lam[0], lam[1], lam[2]};
        copy3(g, src);
    }
    if (e == cudaSuccess) {
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(1);
        cfg.blockDim = dim3(ADJ_THREADS);
        cfg.stream = s;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        e = cudaLaunchKernelEx(&cfg, adj_sum_kernel, (const double*)partials, nb, acc);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(g_params, acc, 3 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return afail(PF_ERR_CUDA, "adjoint: %s", cudaGetErrorString(e));
    return PF_OK;
}

const char* pf_adjoint_last_error(void) { return g_adj_error.c_str(); }

}  // extern "C"
