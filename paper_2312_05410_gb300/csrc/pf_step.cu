// Fused explicit-midpoint step of the phase-field PVD model (arXiv 2312.05410,
// Materials and Methods: composition Cahn-Hilliard equation with mobility
// M^Bulk + M^Surf, order-parameter equation with deposition source
// S = grad(phi).(rho v), vapor convection-diffusion; "Dataset": second-order
// central differences, explicit midpoint in time).
//
// One CTA owns a 56 x TY block of output cells.  It stages 64 x (TY+8) cells of
// phi, c, rho (4-cell halo, periodic wrap in x) in shared memory, then runs the
// two Runge-Kutta stages as two streaming passes:
//   stage 1  u* = u^n + dt/2 R(u^n)   -> shared memory
//   stage 2  u^{n+1} = u^n + dt R(u*) -> global memory
// so a step is one launch with 24 B of algorithmic HBM traffic per cell.
//
// Work layout: a warp's 32 lanes own the 32 column pairs of the 64 staged
// columns, and each warp streams down a segment of rows.  In one pass a lane
// keeps a few rows of phi, c, rho and of the chemical potentials and mobility
// in registers: per row it computes mu_c, mu_phi, M_c (5-point Laplacians),
// and one row behind it the right-hand side (conserved flux divergences,
// Allen-Cahn variant, deposition source, vapor transport).  Vertical
// neighbours are registers, west/east neighbours come from the adjacent lane
// by warp shuffle, so shared memory is touched only to read each input row
// once and to write the stage result.  A pair is computed with packed FP32x2
// arithmetic (fma/add/mul .f32x2).  The outer two columns on each side see a
// shuffled value of their own lane instead of the true neighbour; they lie in
// the halo, which the two stages consume.
//
// Boundary rules live in ghost rows of the staged state: x is periodic; below
// the bottom and above the top row, phi and c are reflected two rows deep
// (mirror), which makes the computed mu and M of the first ghost row equal to
// those of the boundary row, as the no-flux rule requires; rho is reflected
// one row at the bottom and holds the reservoir value rho_top above the top.
// After stage 1, CTAs that touch a boundary write the same ghost rows of u*.
#include "pf_internal.h"

// Tile heights TY and warps S of the three tile kinds (overridable for sweeps), and the
// register budget of the short tile (resident CTAs per SM).
#ifndef PF_MINB_SMALL
#define PF_MINB_SMALL 5
#endif
#ifndef PF_SMALL_TY
#define PF_SMALL_TY 8
#define PF_SMALL_S 4
#endif
#ifndef PF_MEDIUM_TY
#define PF_MEDIUM_TY 16
#define PF_MEDIUM_S 4
#endif
#ifndef PF_LARGE_TY
#define PF_LARGE_TY 24
#define PF_LARGE_S 4
#endif
#ifndef PF_MINB_LARGE
#define PF_MINB_LARGE 4
#endif
// Single runs: TMA staging of the bottom and top tiles and of the x-wrap tiles as well (1), or of
// interior tiles only (0).
#ifndef PF_SINGLE_TMA_EDGES
#define PF_SINGLE_TMA_EDGES 1
#endif

namespace pf {
namespace {

// Pair arithmetic: packed .f32x2 instructions, or (PF_PACKED=0) two scalar FP32 operations.
// Operations with a constant operand (the *K helpers) can instead be issued as two scalar
// operations reading the constant directly (PF_CONST_SCALAR=1): a packed operation needs the
// constant broadcast into a register pair.
#ifndef PF_PACKED
#define PF_PACKED 1
#endif
#ifndef PF_CONST_SCALAR
#define PF_CONST_SCALAR 0
#endif
typedef float2 f2;
__device__ __forceinline__ f2 F2(float a) { return make_float2(a, a); }
#if PF_PACKED
__device__ __forceinline__ f2 add2(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 mul2(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }
#if PF_CONST_SCALAR
__device__ __forceinline__ f2 sub2(f2 a, f2 b) { return make_float2(a.x - b.x, a.y - b.y); }
#else
__device__ __forceinline__ f2 sub2(f2 a, f2 b) { return __ffma2_rn(b, F2(-1.f), a); }
#endif
#else
__device__ __forceinline__ f2 add2(f2 a, f2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ f2 mul2(f2 a, f2 b) { return make_float2(a.x * b.x, a.y * b.y); }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return make_float2(fmaf(a.x, b.x, c.x), fmaf(a.y, b.y, c.y)); }
__device__ __forceinline__ f2 sub2(f2 a, f2 b) { return make_float2(a.x - b.x, a.y - b.y); }
#endif
#if PF_CONST_SCALAR || !PF_PACKED
__device__ __forceinline__ f2 mulK(f2 x, float a) { return make_float2(x.x * a, x.y * a); }
__device__ __forceinline__ f2 fmaKV(float a, f2 x, f2 y) { return make_float2(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y)); }
__device__ __forceinline__ f2 fmaVK(f2 x, float a, float b) { return make_float2(fmaf(x.x, a, b), fmaf(x.y, a, b)); }
__device__ __forceinline__ f2 fmaVVK(f2 x, f2 y, float c) { return make_float2(fmaf(x.x, y.x, c), fmaf(x.y, y.y, c)); }
#else
__device__ __forceinline__ f2 mulK(f2 x, float a) { return mul2(x, F2(a)); }
__device__ __forceinline__ f2 fmaKV(float a, f2 x, f2 y) { return fma2(F2(a), x, y); }
__device__ __forceinline__ f2 fmaVK(f2 x, float a, float b) { return fma2(x, F2(a), F2(b)); }
__device__ __forceinline__ f2 fmaVVK(f2 x, f2 y, float c) { return fma2(x, y, F2(c)); }
#endif
__device__ __forceinline__ f2 ld2(const float* p) { return *reinterpret_cast<const f2*>(p); }
__device__ __forceinline__ void st2(float* p, f2 v) { *reinterpret_cast<f2*>(p) = v; }

constexpr unsigned FULL = 0xffffffffu;
constexpr int HALO = 4;
constexpr int TXO = 56;  // output columns per CTA
constexpr int LX = 64;   // staged columns = 32 lanes x 2

template <int TY, int S>
struct Geo {
    static constexpr int LY = TY + 2 * HALO;  // staged rows
    static constexpr int PX = LX;             // row pitch (floats)
    static constexpr int PLANE = LY * PX;
    static constexpr int THREADS = 32 * S;    // S warps = S row segments
    // resident CTAs per SM the register budget is sized for: 5 for the short tile of small grids
    // (102 registers; the TMA-staged kernel there runs best at that cap), else 4 (4 warps) or 3
    static constexpr int MINB = (TY == PF_SMALL_TY && S == PF_SMALL_S) ? PF_MINB_SMALL
                              : (TY == PF_LARGE_TY && S == PF_LARGE_S) ? PF_MINB_LARGE
                                                                       : (S <= 4 ? 4 : 3);
    static constexpr int cdiv(int a, int b) { return (a + b - 1) / b; }
    static constexpr int L1 = cdiv(TY + 4, S);  // longest stage-1 segment (u* rows)
    static constexpr int L2 = cdiv(TY, S);      // longest stage-2 segment (output rows)
    static constexpr int GUARD = (L1 + 4) * PX; // rows read past a plane by the last segment's tail
    static constexpr size_t BYTES = (size_t(6) * PLANE + GUARD) * sizeof(float);
    static constexpr size_t TMA_BYTES = BYTES + 128;  // + slack to align the TMA destinations to 128 bytes
};

// Every tile kind's staged window (TMA alignment slack included) fits one CTA's shared memory.
static_assert(Geo<PF_SMALL_TY, PF_SMALL_S>::TMA_BYTES <= 227 * 1024 &&
                  Geo<PF_MEDIUM_TY, PF_MEDIUM_S>::TMA_BYTES <= 227 * 1024 &&
                  Geo<PF_LARGE_TY, PF_LARGE_S>::TMA_BYTES <= 227 * 1024,
              "a tile's shared memory exceeds the per-CTA limit");

// West and east neighbours of the lane's pair (x, x+1): x-1 from the lane below, x+2 from the lane above.
__device__ __forceinline__ float west(f2 C) { return __shfl_up_sync(FULL, C.y, 1); }
__device__ __forceinline__ float east(f2 C) { return __shfl_down_sync(FULL, C.x, 1); }
// Horizontal neighbour sums (u[x-1] + u[x+1], u[x] + u[x+2]) and central differences.
__device__ __forceinline__ f2 hsum(float W, f2 C, float E) { return make_float2(W + C.y, C.x + E); }
__device__ __forceinline__ f2 hdiff(float W, f2 C, float E) { return make_float2(C.y - W, E - C.x); }

// Reflect a row index into [0, ny) (mirror about -1/2 and ny - 1/2).
__device__ __forceinline__ int reflect(int gy, int ny)
{
    for (int it = 0; it < 4 && (gy < 0 || gy >= ny); ++it) gy = gy < 0 ? -1 - gy : 2 * ny - 1 - gy;
    return gy < 0 ? 0 : (gy >= ny ? ny - 1 : gy);
}

// Source row of window row gy for field fld under the staging rules: the row itself inside the
// domain, phi and c mirrored two rows deep at the bottom and top, rho mirrored two rows deep at the
// bottom and the reservoir value at row ny (-2), mirrored at ny + 1; -1: zero (rows farther out).
__device__ __forceinline__ int staged_src_row(int fld, int gy, int ny)
{
    if (gy < -2 || gy > ny + 1) return -1;
    if (fld == 2 && gy == ny) return -2;
    return reflect(gy, ny);
}

// First output column of tile column bx.  In a grid whose width is a multiple of 4 the last tile
// column starts at nx - 56 (overlapping its neighbour, whose cells it recomputes bit for bit), so
// its window reaches only 4 columns past the edge, as the first column's does.
__device__ __forceinline__ int tile_x0(int bx, int nx)
{
    const int x0 = bx * TXO;
    return ((nx & 3) == 0 && nx >= TXO && x0 + TXO > nx) ? nx - TXO : x0;
}

// Chemical potentials and mobility of one pair, from its phi and c and their
// four-neighbour sums (f: phi, c: composition, sf / sc: neighbour sums).
template <int MOB>
__device__ __forceinline__ void chem(const StepConst& k, f2 f, f2 c, f2 sf, f2 sc, f2& muc, f2& muf, f2& M)
{
    const f2 ff = mul2(f, f);
    const f2 p = fmaVVK(fmaVK(ff, -0.25f, 0.75f), f, 0.5f);  // p = 1/4 (2-phi)(1+phi)^2
    const f2 q = mul2(c, fmaVK(c, -1.f, 1.f));                  // c (1 - c)
    const f2 g = mul2(q, q);                                           // g(c) = c^2 (1-c)^2
    const f2 Wdg = mul2(q, fmaVK(c, -4.f * k.Wc, 2.f * k.Wc));  // W_c g'(c)
    // mu_c = p W_c g' - kappa_c L(c)
    muc = fmaKV(-k.kc, sc, fmaKV(4.f * k.kc, c, mul2(p, Wdg)));
    // mu_phi = -W_phi phi (1 - phi^2) + p'(phi) W_c g - kappa_phi L(phi),  p' = 3/4 (1 - phi^2)
    f2 m = mul2(fmaVK(ff, k.Wf, -k.Wf), f);
    m = fma2(fmaVK(ff, -0.75f * k.Wc, 0.75f * k.Wc), g, m);
    m = fmaKV(4.f * k.kf, f, m);
    muf = fmaKV(-k.kf, sf, m);
    // M_c = p (MB + h dM) [+ exp(-(phi/sigma)^2)(MBs + h dMs)],  h = c^2 (3 - 2c)
    if (MOB == MOB_UNIFORM) {
        M = mulK(p, k.MBb);
    } else {
        const f2 h = mul2(mul2(c, c), fmaVK(c, -2.f, 3.f));
        M = mul2(p, fmaVK(h, k.dMb, k.MBb));
        if (MOB == MOB_SURF) {
            const f2 t = mulK(ff, k.nisig2);
            M = fma2(make_float2(exp2f(t.x), exp2f(t.y)), fmaVK(h, k.dMs, k.MBs), M);
        }
    }
}

// One Runge-Kutta stage for the rows [r0, r0+n) of the lane's column pair.
// In: staged planes (phi, c, rho) at I, I+PLANE, I+2 PLANE, already offset to the lane's pair.
// Base: the state the update starts from (the input itself for stage 1, u^n for stage 2).
// MODE 0: u* = in + dt/2 R(in) into the planes at Out; MODE 1: u^{n+1} = base + dt R(in) to
// global memory; MODE 2: the same u^{n+1} into the planes at Out (the first of two steps in one
// launch); MODE 3: as MODE 1, with the base u^n read from global memory at the output cell (b_phi,
// b_c, b_rho; the staged window is then free while this stage runs).  Every lane runs all L + 2
// iterations (shuffles need the whole warp); rows past n are computed from guard/halo data and not
// stored.
template <int L, int PX, int PLANE, int PHI_MODE, int MOB, int MODE>
__device__ __forceinline__ void stage(const StepConst& k, const float* __restrict__ I,
                                      const float* __restrict__ Base, float* __restrict__ Out, int r0, int n,
                                      float* __restrict__ g_phi, float* __restrict__ g_c, float* __restrict__ g_rho,
                                      size_t g_off, int pitch, bool store_x, bool pair_full,
                                      const float* __restrict__ b_phi = nullptr, const float* __restrict__ b_c = nullptr,
                                      const float* __restrict__ b_rho = nullptr)
{
    const float* Fi = I;
    const float* Ci = I + PLANE;
    const float* Ri = I + 2 * PLANE;
    // Windows. phi and c rows are numbered t = row - (r0 - 2); rho rows t' = row - (r0 - 3).
    f2 fw[4], cw[3], rw[3], mcw[3], mfw[3], Mw[3];
    float fWw[2], fEw[2];  // west/east neighbours of phi at the last two mu rows
    fw[0] = ld2(Fi + (r0 - 2) * PX);
    fw[1] = ld2(Fi + (r0 - 1) * PX);
    cw[0] = ld2(Ci + (r0 - 2) * PX);
    cw[1] = ld2(Ci + (r0 - 1) * PX);
    constexpr bool FINAL = MODE != 0;  // a full-dt update from the base state
    const float hdt = FINAL ? k.dt : 0.5f * k.dt;
#pragma unroll
    for (int j = 0; j < L + 2; ++j) {
        // rows entering the window: phi, c at r0 + j (t = j + 2); rho at r0 - 1 + j (t' = j + 2)
        fw[(j + 2) % 4] = ld2(Fi + (r0 + j) * PX);
        cw[(j + 2) % 3] = ld2(Ci + (r0 + j) * PX);
        rw[(j + 2) % 3] = ld2(Ri + (r0 - 1 + j) * PX);

        // mu_c, mu_phi, M at row r0 - 1 + j (phi, c rows t = j .. j + 2)
        {
            const f2 f = fw[(j + 1) % 4], c = cw[(j + 1) % 3];
            fWw[j % 2] = west(f);
            fEw[j % 2] = east(f);
            const f2 sf = add2(hsum(fWw[j % 2], f, fEw[j % 2]), add2(fw[j % 4], fw[(j + 2) % 4]));
            const f2 sc = add2(hsum(west(c), c, east(c)), add2(cw[j % 3], cw[(j + 2) % 3]));
            chem<MOB>(k, f, c, sf, sc, mcw[j % 3], mfw[j % 3], Mw[j % 3]);
        }
        if (j < 2) continue;

        // right-hand side at row r0 - 2 + j: mu/M rows j-2, j-1, j (window slots), phi t = j-1..j+1,
        // rho t' = j .. j + 2, c t = j
        const int iS = (j - 2) % 3, iC = (j - 1) % 3, iN = j % 3;
        // conserved composition flux: sum_faces (M + M_nb)(mu_nb - mu) / (2 dx^2)
        const f2 m = mcw[iC], M = Mw[iC];
        const float mE = east(m), ME = east(M);
        const float Fb = (M.x + M.y) * (m.y - m.x);  // face (x | x+1)
        const float Fc = (M.y + ME) * (mE - m.y);    // face (x+1 | x+2)
        const float Fa = __shfl_up_sync(FULL, Fc, 1);  // face (x-1 | x) = the west lane's east face
        f2 rc = make_float2(Fb - Fa, Fc - Fb);
        rc = fma2(add2(M, Mw[iN]), sub2(mcw[iN], m), rc);
        rc = fma2(add2(M, Mw[iS]), sub2(mcw[iS], m), rc);

        // deposition source S = grad(phi) . (rho v), central differences
        const f2 f = fw[j % 4], fN = fw[(j + 1) % 4], fS = fw[(j + 3) % 4];
        const f2 r = rw[(j + 1) % 3], rN = rw[(j + 2) % 3], rS = rw[j % 3];
        const float rW = west(r), rE = east(r);
        // phi at this row is the centre of the mu row computed one iteration earlier
        const f2 Src = mul2(r, fmaKV(k.ax, hdiff(fWw[(j + 1) % 2], f, fEw[(j + 1) % 2]), mulK(sub2(fN, fS), k.ay)));

        f2 Rf;
        if (PHI_MODE == 0) {
            const f2 u = mfw[iC];
            const f2 su = add2(hsum(west(u), u, east(u)), add2(mfw[iN], mfw[iS]));
            Rf = fmaKV(k.cF, fmaKV(-4.f, u, su), Src);
        } else {
            Rf = fmaKV(k.cF, mfw[iC], Src);
        }
        // vapor: D L(rho) - div(rho v) - S
        const f2 lap = fmaKV(-4.f, r, add2(hsum(rW, r, rE), add2(rN, rS)));
        const f2 nadv = fmaKV(-k.ax, hdiff(rW, r, rE), mulK(sub2(rN, rS), -k.ay));  // -div(rho v)
        const f2 Rr = sub2(fmaKV(k.cD, lap, nadv), Src);

        const int i = j - 2;  // output row r0 + i
        f2 bf, bc, br;
        if (MODE == 3) {  // only stored cells need their base
            bf = bc = br = F2(0.f);
            if (store_x && i < n) {
                const size_t g = g_off + size_t(i) * pitch;
                if (pair_full) {
                    bf = __ldg(reinterpret_cast<const f2*>(b_phi + g));
                    bc = __ldg(reinterpret_cast<const f2*>(b_c + g));
                    br = __ldg(reinterpret_cast<const f2*>(b_rho + g));
                } else {
                    bf.x = __ldg(b_phi + g);
                    bc.x = __ldg(b_c + g);
                    br.x = __ldg(b_rho + g);
                }
            }
        } else if (FINAL) {
            const int o = (r0 + i) * PX;
            bf = ld2(Base + o);
            bc = ld2(Base + PLANE + o);
            br = ld2(Base + 2 * PLANE + o);
        } else {
            bf = f;
            bc = cw[j % 3];
            br = r;
        }
        const f2 of = fmaKV(hdt, Rf, bf);
        const f2 oc = fmaKV(hdt, mulK(rc, k.cR), bc);
        const f2 orr = fmaKV(hdt, Rr, br);
        if (i < n) {
            if (MODE == 0 || MODE == 2) {
                const int o = (r0 + i) * PX;
                st2(Out + o, of);
                st2(Out + PLANE + o, oc);
                st2(Out + 2 * PLANE + o, orr);
            } else if (store_x) {
                const size_t g = g_off + size_t(i) * pitch;
                if (pair_full) {
                    st2(g_phi + g, of);
                    st2(g_c + g, oc);
                    st2(g_rho + g, orr);
                } else {
                    g_phi[g] = of.x;
                    g_c[g] = oc.x;
                    g_rho[g] = orr.x;
                }
            }
        }
    }
}

// Rows [lo, hi) split into S near-equal segments; segment s of them.
__device__ __forceinline__ void segment(int lo, int hi, int S, int s, int& r0, int& n)
{
    const int H = hi > lo ? hi - lo : 0;
    r0 = lo + (s * H) / S;
    n = lo + ((s + 1) * H) / S - r0;
}

// Stage 1 of one staged tile (window corner (gx0, gy0), u^n in U): u* on the staged rows [2, LY-2)
// inside the domain into B, then the ghost rows of u* where the tile touches the bottom or top.
// Ends with a barrier: U is no longer read after it.
template <int TY, int S, int PHI_MODE, int MOB>
__device__ __forceinline__ void tile_stage1(const StepConst& k, int gx0, int gy0, const float* __restrict__ U,
                                            float* __restrict__ B)
{
    using G = Geo<TY, S>;
    constexpr int PX = G::PX, PLANE = G::PLANE, LY = G::LY;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ny = k.ny;
    const int dlo = -gy0 > 0 ? -gy0 : 0;  // staged rows holding domain rows: [dlo, dhi)
    const int dhi = ny - gy0 < LY ? ny - gy0 : LY;
    const int lo2 = 2 * lane;
    int r0, n;
    segment(dlo > 2 ? dlo : 2, dhi < LY - 2 ? dhi : LY - 2, S, warp, r0, n);
    stage<G::L1, PX, PLANE, PHI_MODE, MOB, 0>(k, U + lo2, nullptr, B + lo2, r0, n, nullptr, nullptr, nullptr, 0, 0,
                                              false, false);
    __syncthreads();
    const bool bottom = dlo > 0, top = dhi <= LY - 3;
    if (bottom || top) {
        for (int idx = tid; idx < 3 * 2 * LX; idx += G::THREADS) {
            const int fld = idx / (2 * LX), rem = idx - fld * (2 * LX);
            const int d = rem / LX, x = rem - d * LX;  // ghost depth d + 1
            float* P = B + fld * PLANE + x;
            if (bottom) {
                const int gy = -1 - d;
                if (fld < 2 || d == 0) P[(gy - gy0) * PX] = P[(reflect(gy, ny) - gy0) * PX];
            }
            if (top) {
                const int gy = ny + d, ly = gy - gy0;
                if (ly < LY) {
                    if (fld == 2)
                        P[ly * PX] = (d == 0) ? k.rho_top : 0.f;
                    else
                        P[ly * PX] = P[(reflect(gy, ny) - gy0) * PX];
                }
            }
        }
        __syncthreads();
    }
}

// Stage 2 of one tile: u^{n+1} on the output rows [4, 4+TY) inside the domain, from u* in B and the
// base u^n staged in U (MODE 1) or read from global memory at the output cells (MODE 3: b_*).
template <int TY, int S, int PHI_MODE, int MOB, int MODE = 1>
__device__ __forceinline__ void tile_stage2(const StepConst& k, int gx0, int gy0, const float* __restrict__ U,
                                            const float* __restrict__ B, float* __restrict__ phi1,
                                            float* __restrict__ c1, float* __restrict__ rho1,
                                            const float* b_phi = nullptr, const float* b_c = nullptr,
                                            const float* b_rho = nullptr)
{
    using G = Geo<TY, S>;
    constexpr int PX = G::PX, PLANE = G::PLANE, LY = G::LY;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nx = k.nx, ny = k.ny, pitch = k.pitch;
    const int dlo = -gy0 > 0 ? -gy0 : 0;
    const int dhi = ny - gy0 < LY ? ny - gy0 : LY;
    const int lo2 = 2 * lane;
    int r0, n;
    segment(dlo > HALO ? dlo : HALO, dhi < HALO + TY ? dhi : HALO + TY, S, warp, r0, n);
    const int gx = gx0 + lo2;  // global column of the pair's first cell
    const bool store_x = (lo2 >= HALO) && (lo2 < HALO + TXO) && gx < nx;
    const bool pair_full = gx + 1 < nx;
    const size_t g_off = (size_t)(gy0 + r0) * pitch + (gx < 0 ? 0 : gx);
    stage<G::L2, PX, PLANE, PHI_MODE, MOB, MODE>(k, B + lo2, U + lo2, nullptr, r0, n, phi1, c1, rho1, g_off, pitch,
                                                 store_x, pair_full, b_phi, b_c, b_rho);
}

// The two Runge-Kutta stages of one staged tile (window corner (gx0, gy0), u^n in U, u* in B):
// stage 1 into B, the ghost rows of u* where the tile touches the bottom or top, stage 2 to global
// memory.  STAGES = 1: one forward-Euler update u + dt R(u) straight to global memory.
template <int TY, int S, int PHI_MODE, int MOB, int STAGES = 2>
__device__ __forceinline__ void compute_tile(const StepConst& k, int gx0, int gy0, const float* __restrict__ U,
                                             float* __restrict__ B, float* __restrict__ phi1,
                                             float* __restrict__ c1, float* __restrict__ rho1)
{
    using G = Geo<TY, S>;
    constexpr int PX = G::PX, PLANE = G::PLANE, LY = G::LY;
    if (STAGES == 1) {  // u + dt R(u) on the output rows, straight to global memory
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const int nx = k.nx, ny = k.ny, pitch = k.pitch;
        const int dlo = -gy0 > 0 ? -gy0 : 0;
        const int dhi = ny - gy0 < LY ? ny - gy0 : LY;
        const int lo2 = 2 * lane;
        int r0, n;
        segment(dlo > HALO ? dlo : HALO, dhi < HALO + TY ? dhi : HALO + TY, S, warp, r0, n);
        const int gx = gx0 + lo2;
        const bool store_x = (lo2 >= HALO) && (lo2 < HALO + TXO) && gx < nx;
        const size_t g_off = (size_t)(gy0 + r0) * pitch + (gx < 0 ? 0 : gx);
        stage<G::L2, PX, PLANE, PHI_MODE, MOB, 1>(k, U + lo2, U + lo2, nullptr, r0, n, phi1, c1, rho1, g_off, pitch,
                                                  store_x, gx + 1 < nx);
        return;
    }
    tile_stage1<TY, S, PHI_MODE, MOB>(k, gx0, gy0, U, B);
    tile_stage2<TY, S, PHI_MODE, MOB>(k, gx0, gy0, U, B, phi1, c1, rho1);
}

// Per-thread staging of the window with corner (gx0, gy0) of u^n into U: periodic wrap in x,
// reflected ghost rows of phi and c, the reservoir row of rho above the top, zero rows beyond.
// nx % 4 == 0: every aligned 16-byte group is one asynchronous copy (cp.async, not waited for
// here); other widths: plain loads and stores.
template <class G>
__device__ __forceinline__ void issue_plain_g(const StepConst& k, int gx0, int gy0, const float* __restrict__ phi0,
                                              const float* __restrict__ c0, const float* __restrict__ rho0,
                                              float* __restrict__ U)
{
    constexpr int PX = G::PX, PLANE = G::PLANE, LY = G::LY;
    const int tid = threadIdx.x;
    const int nx = k.nx, ny = k.ny, pitch = k.pitch;
    auto field = [&](int f) { return f == 0 ? phi0 : (f == 1 ? c0 : rho0); };
    auto wrap = [&](int gx) {  // periodic x; one correction suffices when nx >= LX
        if (nx >= LX) {
            gx = gx < 0 ? gx + nx : gx;
            return gx >= nx ? gx - nx : gx;
        }
        gx %= nx;
        return gx < 0 ? gx + nx : gx;
    };
    // source row of staged row ly for field fld; -1: zero, -2: reservoir value
    auto src_row = [&](int fld, int ly) { return staged_src_row(fld, gy0 + ly, ny); };
    if ((nx & 3) == 0) {
        // x0 and nx are multiples of 4: each aligned group of 4 staged columns is
        // wholly inside [0, nx) or wholly wrapped
        constexpr int Q = LX / 4;
        for (int idx = tid; idx < 3 * LY * Q; idx += G::THREADS) {
            const int fld = idx / (LY * Q);
            const int rem = idx - fld * (LY * Q);
            const int ly = rem / Q, q = rem - ly * Q;
            float* dst = U + fld * PLANE + ly * PX + 4 * q;
            const int sr = src_row(fld, ly);
            if (sr < 0) {
                const float v = (sr == -2) ? k.rho_top : 0.f;
                *reinterpret_cast<float4*>(dst) = make_float4(v, v, v, v);
            } else {
                const float* src = field(fld) + (size_t)sr * pitch + wrap(gx0 + 4 * q);
                const unsigned sdst = (unsigned)__cvta_generic_to_shared(dst);
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sdst), "l"(src) : "memory");
            }
        }
    } else {
        for (int idx = tid; idx < 3 * LY * LX; idx += G::THREADS) {
            const int fld = idx / (LY * LX);
            const int rem = idx - fld * (LY * LX);
            const int ly = rem / LX, lx = rem - ly * LX;
            const int sr = src_row(fld, ly);
            float v = (sr == -2) ? k.rho_top : 0.f;
            if (sr >= 0) v = __ldg(field(fld) + (size_t)sr * pitch + wrap(gx0 + lx));
            U[fld * PLANE + ly * PX + lx] = v;
        }
    }
}

template <int TY, int S>
__device__ __forceinline__ void issue_plain(const StepConst& k, int gx0, int gy0, const float* __restrict__ phi0,
                                            const float* __restrict__ c0, const float* __restrict__ rho0,
                                            float* __restrict__ U)
{
    issue_plain_g<Geo<TY, S>>(k, gx0, gy0, phi0, c0, rho0, U);
}

// Thread 0 only: three TMA box copies (64 x LY per field) of the window with corner (gx0, gy0)
// into U, completing on the mbarrier at shared address mb (armed here for their bytes).
template <class G>
__device__ __forceinline__ void issue_tma_g(const StepMaps* maps, int gx0, int gy0, float* U, unsigned mb)
{
    constexpr int PLANE = G::PLANE;
    constexpr unsigned bytes = 3u * PLANE * sizeof(float);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(bytes) : "memory");
    const CUtensorMap* tm[3] = {&maps->phi, &maps->c, &maps->rho};
#pragma unroll
    for (int f = 0; f < 3; ++f) {
        const unsigned dst = (unsigned)__cvta_generic_to_shared(U + f * PLANE);
        asm volatile(
            "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
            " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
            "l"(reinterpret_cast<uint64_t>(tm[f])), "r"(gx0), "r"(gy0), "r"(mb)
            : "memory");
    }
}

template <int TY, int S>
__device__ __forceinline__ void issue_tma(const StepMaps* maps, int gx0, int gy0, float* U, unsigned mb)
{
    issue_tma_g<Geo<TY, S>>(maps, gx0, gy0, U, mb);
}

// Ghost rows of a TMA-staged window of u^n (corner row gy0).  The copy fills rows outside the domain
// with zeros; rows -2, -1, ny, ny+1 are then set as the per-thread staging sets them: mirrored from
// the domain rows inside the window, rho at row ny the reservoir value.  Rows farther out stay zero,
// as there.  Needs ny >= LY (the mirrored rows lie in the window); all threads, after the wait.
// Columns [xskip, xskip + 4) are left alone (a wrap fixup sets them in every row).
template <class G>
__device__ __forceinline__ void tma_ghost_rows(const StepConst& k, int gy0, float* __restrict__ U, int xskip)
{
    constexpr int PX = G::PX, PLANE = G::PLANE, LY = G::LY;
    const int ny = k.ny;
    for (int idx = threadIdx.x; idx < 3 * 4 * LX; idx += G::THREADS) {
        const int fld = idx / (4 * LX), rem = idx - fld * (4 * LX);
        const int g = rem / LX, x = rem - g * LX;
        const int gy = g < 2 ? -1 - g : ny + (g - 2);  // -1, -2, ny, ny + 1
        const int ly = gy - gy0;
        if (ly < 0 || ly >= LY || (x >= xskip && x < xskip + 4)) continue;
        float* Q = U + fld * PLANE + x;
        if (fld == 2 && gy == ny) {
            Q[ly * PX] = k.rho_top;
            continue;
        }
        const int sy = reflect(gy, ny) - gy0;
        if (sy >= 0 && sy < LY) Q[ly * PX] = Q[sy * PX];
    }
}

// The 4 staged columns that a TMA box reaching past an x edge fills with zeros: [0, 4) of a window
// from x = -4 (values of columns nx-4 .. nx-1), [60, 64) of a window ending at nx + 4 (columns 0 .. 3),
// every row by the staging rules.  Each thread loads its share into registers before the wait for
// the copy (the loads overlap it) and stores them after.
template <class G>
struct WrapCols {
    static constexpr int N = 3 * G::LY * 4;
    static constexpr int PER = (N + G::THREADS - 1) / G::THREADS;
};

template <class G>
__device__ __forceinline__ void wrap_load(const StepConst& k, int gy0, bool left, const float* __restrict__ phi0,
                                          const float* __restrict__ c0, const float* __restrict__ rho0,
                                          float (&v)[WrapCols<G>::PER])
{
    constexpr int LY = G::LY;
    const int ny = k.ny, pitch = k.pitch, xs = left ? k.nx - 4 : 0;
#pragma unroll
    for (int i = 0; i < WrapCols<G>::PER; ++i) {
        const int idx = threadIdx.x + i * G::THREADS;
        float val = 0.f;
        if (idx < WrapCols<G>::N) {
            const int fld = idx / (LY * 4), rem = idx - fld * (LY * 4);
            const int ly = rem >> 2, cc = rem & 3;
            const int sr = staged_src_row(fld, gy0 + ly, ny);
            const float* F = fld == 0 ? phi0 : (fld == 1 ? c0 : rho0);
            if (sr >= 0) val = __ldg(F + (size_t)sr * pitch + xs + cc);
            else if (sr == -2) val = k.rho_top;
        }
        v[i] = val;
    }
}

template <class G>
__device__ __forceinline__ void wrap_store(bool left, const float (&v)[WrapCols<G>::PER], float* __restrict__ U)
{
    constexpr int LY = G::LY, PX = G::PX, PLANE = G::PLANE;
    const int xd = left ? 0 : LX - 4;
#pragma unroll
    for (int i = 0; i < WrapCols<G>::PER; ++i) {
        const int idx = threadIdx.x + i * G::THREADS;
        if (idx < WrapCols<G>::N) {
            const int fld = idx / (LY * 4), rem = idx - fld * (LY * 4);
            const int ly = rem >> 2, cc = rem & 3;
            U[fld * PLANE + ly * PX + xd + cc] = v[i];
        }
    }
}

// Bounded poll of mbarrier phase `parity` by the calling thread: 1 if it completed within cap polls.
__device__ __forceinline__ unsigned poll_phase(unsigned mb, unsigned parity, int cap)
{
    unsigned done = 0;
    for (int it = 0; it < cap && !done; ++it)
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
            : "=r"(done) : "r"(mb), "r"(parity) : "memory");
    return done;
}

// One step of the output tile with corner (x0, y0) of one run (the whole CTA).
// STAGES = 2: the explicit midpoint step; STAGES = 1: one forward-Euler update
// u + dt R(u) with the dt held in k (the adjoint uses it for u* with dt/2).
template <int TY, int S, int PHI_MODE, int MOB, int STAGES = 2, bool TMA = false, bool TMA_EDGES = true>
__device__ __forceinline__ void step_tile(const StepConst& k, int x0, int y0, const float* __restrict__ phi0,
                                          const float* __restrict__ c0, const float* __restrict__ rho0,
                                          float* __restrict__ phi1, float* __restrict__ c1, float* __restrict__ rho1,
                                          const StepMaps* maps = nullptr, int* err = nullptr)
{
    using G = Geo<TY, S>;
    constexpr int PLANE = G::PLANE, LY = G::LY;
    extern __shared__ __align__(128) float smraw[];
    // TMA destinations need a 128-byte aligned base; that launch reserves the extra bytes
    float* const sm = TMA ? reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(smraw) + 127) & ~uintptr_t(127))
                          : smraw;
    float* const U = sm;               // u^n: phi, c, rho
    float* const B = sm + 3 * PLANE;   // u*:  phi, c, rho (followed by the guard rows)

    const int tid = threadIdx.x;
    const int gx0 = x0 - HALO, gy0 = y0 - HALO;
    const int nx = k.nx, ny = k.ny;

    // Wait for the previous step's grid (programmatic dependent launch) before reading.
    asm volatile("griddepcontrol.wait;" ::: "memory");

    // ---- TMA staging: three box copies (64 x LY each) completing on one mbarrier, for windows inside
    // the grid in x and (widths a multiple of 4) windows reaching 4 columns past an x edge.  Cells
    // outside the grid arrive as zeros; the wrapped columns and the ghost rows are set after the wait.
    const bool xin = gx0 >= 0 && gx0 + LX <= nx;
    const bool wleft = gx0 == -HALO, wright = gx0 + LX == nx + HALO;
    const bool xwrap = (wleft || wright) && (nx & 3) == 0 && nx >= LX;
    const bool tma_ok = TMA_EDGES ? (xin || xwrap) : (xin && gy0 >= 0 && gy0 + LY <= ny);
    bool staged = false;
    if (TMA && ny >= LY && tma_ok) {
        __shared__ __align__(8) uint64_t mbar;
        const unsigned mb = (unsigned)__cvta_generic_to_shared(&mbar);
        if (tid == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncthreads();
        if (tid == 0) issue_tma<TY, S>(maps, gx0, gy0, U, mb);
        float wv[WrapCols<G>::PER];
        if (!xin) wrap_load<G>(k, gy0, wleft, phi0, c0, rho0, wv);
        // bounded wait on phase 0; every thread votes so the whole CTA leaves together on a timeout
        const unsigned done = poll_phase(mb, 0, k.wait_cap);
        if (__syncthreads_or(!done)) {
            if (tid == 0 && err) atomicOr(err, ERR_BIT_TIMEOUT);
            poll_phase(mb, 0, 1 << 22);  // let the copies in flight land before leaving
            return;
        }
        // disjoint cells: the wrapped columns in every row, the ghost rows in the other columns;
        // ordered before the stages by the barrier below
        if (!xin) wrap_store<G>(wleft, wv, U);
        if (gy0 < 0 || gy0 + LY > ny) tma_ghost_rows<G>(k, gy0, U, xin ? LX : (wleft ? 0 : LX - 4));
        staged = true;
    }
    // ---- other tiles: stage u^n with its ghost rows
    if (!staged) {
        issue_plain<TY, S>(k, gx0, gy0, phi0, c0, rho0, U);
        asm volatile("cp.async.wait_all;" ::: "memory");
    }
    // Let the next step's grid begin launching; it waits for this grid to finish.
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    __syncthreads();

    compute_tile<TY, S, PHI_MODE, MOB, STAGES>(k, gx0, gy0, U, B, phi1, c1, rho1);
}

// One step of one run: a 2D grid of 56 x TY tiles.
template <int TY, int S, int PHI_MODE, int MOB>
__global__ void __launch_bounds__(Geo<TY, S>::THREADS, Geo<TY, S>::MINB)
step_kernel(const StepConst k, const float* __restrict__ phi0, const float* __restrict__ c0,
            const float* __restrict__ rho0, float* __restrict__ phi1, float* __restrict__ c1,
            float* __restrict__ rho1)
{
    step_tile<TY, S, PHI_MODE, MOB>(k, tile_x0(blockIdx.x, k.nx), blockIdx.y * TY, phi0, c0, rho0, phi1, c1, rho1);
}

// The same, with tiles staged by TMA through the tensor maps of the source state.
template <int TY, int S, int PHI_MODE, int MOB>
__global__ void __launch_bounds__(Geo<TY, S>::THREADS, Geo<TY, S>::MINB)
step_kernel_tma(const StepConst k, const float* __restrict__ phi0, const float* __restrict__ c0,
                const float* __restrict__ rho0, float* __restrict__ phi1, float* __restrict__ c1,
                float* __restrict__ rho1, const __grid_constant__ StepMaps maps, int* __restrict__ err)
{
    step_tile<TY, S, PHI_MODE, MOB, 2, true, PF_SINGLE_TMA_EDGES != 0>(k, tile_x0(blockIdx.x, k.nx), blockIdx.y * TY,
                                                                      phi0, c0, rho0, phi1, c1, rho1, &maps, err);
}

// One forward-Euler update of one run (dt taken from k).
template <int TY, int S, int PHI_MODE, int MOB>
__global__ void __launch_bounds__(Geo<TY, S>::THREADS, Geo<TY, S>::MINB)
euler_kernel(const StepConst k, const float* __restrict__ phi0, const float* __restrict__ c0,
             const float* __restrict__ rho0, float* __restrict__ phi1, float* __restrict__ c1,
             float* __restrict__ rho1)
{
    step_tile<TY, S, PHI_MODE, MOB, 1>(k, tile_x0(blockIdx.x, k.nx), blockIdx.y * TY, phi0, c0, rho0, phi1, c1,
                                       rho1);
}

// One step of every run of an ensemble: CTA b takes tile b of the table; runs
// step in lockstep, so one parity bit says which buffer of each run is current.
template <int TY, int S, int PHI_MODE, int MOB>
__global__ void __launch_bounds__(Geo<TY, S>::THREADS, Geo<TY, S>::MINB)
ens_step_kernel(const EnsTile* __restrict__ tiles, const EnsRun* __restrict__ runs, int parity)
{
    const EnsTile t = tiles[blockIdx.x];
    const EnsRun& r = runs[t.run];
    const int a = parity, b = 1 - parity;
    step_tile<TY, S, PHI_MODE, MOB>(r.k, t.x0, t.y0, r.f[a][0], r.f[a][1], r.f[a][2], r.f[b][0], r.f[b][1],
                                    r.f[b][2]);
}

// The same with TMA staging: every run's tensor maps of the current buffer travel with the launch as
// one kernel parameter (the form TMA reads without a tensor-map proxy fence).
template <int TY, int S, int PHI_MODE, int MOB>
__global__ void __launch_bounds__(Geo<TY, S>::THREADS, Geo<TY, S>::MINB)
ens_step_kernel_tma(const EnsTile* __restrict__ tiles, const EnsRun* __restrict__ runs, int parity,
                    const __grid_constant__ EnsMaps maps, int* __restrict__ err)
{
    const EnsTile t = tiles[blockIdx.x];
    const EnsRun& r = runs[t.run];
    const int a = parity, b = 1 - parity;
    step_tile<TY, S, PHI_MODE, MOB, 2, true>(r.k, t.x0, t.y0, r.f[a][0], r.f[a][1], r.f[a][2], r.f[b][0], r.f[b][1],
                                             r.f[b][2], &maps.run[t.run], err);
}

// ---- persistent tile loops for large grids and ensembles
//
// CTA b takes tiles b, b + G, b + 2G, ... of the row-major tile order (G = the grid: as many CTAs
// as are resident at once).  There is one staging buffer, as in the one-tile-per-CTA kernel, so
// 4 CTAs stay resident per SM: stage 1 reads the staged window; stage 2 reads u* and takes its base
// values u^n from global memory at the output cells (L2 holds them: the window was just staged),
// so as soon as stage 1 is done the buffer takes the next tile's staging -- TMA for interior tiles
// (thread 0, one mbarrier, after a fence.proxy.async ordering the buffer's generic reads before the
// asynchronous writes), per-thread cp.async otherwise -- which lands while stage 2 runs.  The
// per-cell arithmetic is that of the one-tile-per-CTA kernel, so the results are the same bit
// for bit.
template <int TY, int S>
struct RingGeo {
    static constexpr size_t BYTES = Geo<TY, S>::BYTES + 128;  // + slack to align the TMA destination
};

// Ring state of one CTA: the staging buffer, u*, the mbarrier, the phase it waits for next and
// whether the staged tile came by TMA.
struct Ring {
    float* U;
    float* B;
    unsigned mb;
    unsigned phase = 0u;
    bool tma = false;
};

template <int TY, int S>
__device__ __forceinline__ Ring ring_setup(uint64_t* mbar)
{
    extern __shared__ __align__(128) float smraw[];
    Ring r;
    r.U = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(smraw) + 127) & ~uintptr_t(127));
    r.B = r.U + 3 * Geo<TY, S>::PLANE;
    r.mb = (unsigned)__cvta_generic_to_shared(mbar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(r.mb) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    return r;
}

// Wait until the buffer holds its tile.  false: a TMA wait ran out (ERR_BIT_TIMEOUT set, the copies
// in flight drained with a bound): the whole CTA must leave.
__device__ __forceinline__ bool ring_wait(Ring& r, int cap, int* err)
{
    if (r.tma) {
        const unsigned done = poll_phase(r.mb, r.phase, cap);
        if (__syncthreads_or(!done)) {
            if (threadIdx.x == 0 && err) atomicOr(err, ERR_BIT_TIMEOUT);
            poll_phase(r.mb, r.phase, 1 << 22);
            asm volatile("cp.async.wait_all;" ::: "memory");
            return false;
        }
        r.phase ^= 1u;
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    return true;
}

// Stage the window with corner (gx0, gy0) into the buffer: TMA for interior windows when maps are
// given, else per-thread cp.async.  Every reader of the buffer passed a barrier before this.
template <int TY, int S>
__device__ __forceinline__ void ring_issue(Ring& r, const StepConst& k, int gx0, int gy0, const float* phi0,
                                           const float* c0, const float* rho0, const StepMaps* maps)
{
    constexpr int LY = Geo<TY, S>::LY;
    r.tma = maps && gx0 >= 0 && gx0 + LX <= k.nx && gy0 >= 0 && gy0 + LY <= k.ny;
    if (r.tma) {
        if (threadIdx.x == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue_tma<TY, S>(maps, gx0, gy0, r.U, r.mb);
        }
    } else {
        issue_plain<TY, S>(k, gx0, gy0, phi0, c0, rho0, r.U);
    }
}

// One step of one run over all its 56 x TY tiles (maps NULL: no TMA).
template <int TY, int S, int PHI_MODE, int MOB>
__global__ void __launch_bounds__(Geo<TY, S>::THREADS, Geo<TY, S>::MINB)
step_kernel_ring(const StepConst k, const float* __restrict__ phi0, const float* __restrict__ c0,
                 const float* __restrict__ rho0, float* __restrict__ phi1, float* __restrict__ c1,
                 float* __restrict__ rho1, const __grid_constant__ StepMaps maps, int use_maps, int* __restrict__ err)
{
    __shared__ __align__(8) uint64_t mbar;
    Ring r = ring_setup<TY, S>(&mbar);
    const int ntx = (k.nx + TXO - 1) / TXO, ntiles = ntx * ((k.ny + TY - 1) / TY);
    const StepMaps* mp = use_maps ? &maps : nullptr;
    asm volatile("griddepcontrol.wait;" ::: "memory");
    int t = blockIdx.x;
    if (t < ntiles) {
        const int ty = t / ntx;
        ring_issue<TY, S>(r, k, (t - ty * ntx) * TXO - HALO, ty * TY - HALO, phi0, c0, rho0, mp);
    }
#pragma unroll 1
    while (t < ntiles) {
        if (!ring_wait(r, k.wait_cap, err)) return;
        const int ty = t / ntx;
        const int gx0 = (t - ty * ntx) * TXO - HALO, gy0 = ty * TY - HALO;
        tile_stage1<TY, S, PHI_MODE, MOB>(k, gx0, gy0, r.U, r.B);
        const int tn = t + gridDim.x;
        if (tn < ntiles) {
            const int tyn = tn / ntx;
            ring_issue<TY, S>(r, k, (tn - tyn * ntx) * TXO - HALO, tyn * TY - HALO, phi0, c0, rho0, mp);
        } else {
            asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
        }
        tile_stage2<TY, S, PHI_MODE, MOB, 3>(k, gx0, gy0, r.U, r.B, phi1, c1, rho1, phi0, c0, rho0);
        __syncthreads();  // u* is rewritten by the next tile's stage 1
        t = tn;
    }
}

// One step of every run of an ensemble over its tile table (per-thread staging only).
template <int TY, int S, int PHI_MODE, int MOB>
__global__ void __launch_bounds__(Geo<TY, S>::THREADS, Geo<TY, S>::MINB)
ens_step_kernel_ring(const EnsTile* __restrict__ tiles, const EnsRun* __restrict__ runs, int ntiles, int parity)
{
    __shared__ __align__(8) uint64_t mbar;
    Ring r = ring_setup<TY, S>(&mbar);
    const int a = parity;
    asm volatile("griddepcontrol.wait;" ::: "memory");
    int t = blockIdx.x;
    if (t < ntiles) {
        const EnsTile e = tiles[t];
        const EnsRun& run = runs[e.run];
        ring_issue<TY, S>(r, run.k, e.x0 - HALO, e.y0 - HALO, run.f[a][0], run.f[a][1], run.f[a][2], nullptr);
    }
#pragma unroll 1
    while (t < ntiles) {
        ring_wait(r, 0, nullptr);  // per-thread copies only: no bounded TMA wait
        const EnsTile e = tiles[t];
        const EnsRun& run = runs[e.run];
        tile_stage1<TY, S, PHI_MODE, MOB>(run.k, e.x0 - HALO, e.y0 - HALO, r.U, r.B);
        const int tn = t + gridDim.x;
        if (tn < ntiles) {
            const EnsTile en = tiles[tn];
            const EnsRun& rn = runs[en.run];
            ring_issue<TY, S>(r, rn.k, en.x0 - HALO, en.y0 - HALO, rn.f[a][0], rn.f[a][1], rn.f[a][2], nullptr);
        } else {
            asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
        }
        tile_stage2<TY, S, PHI_MODE, MOB, 3>(run.k, e.x0 - HALO, e.y0 - HALO, r.U, r.B, run.f[1 - a][0],
                                             run.f[1 - a][1], run.f[1 - a][2], run.f[a][0], run.f[a][1], run.f[a][2]);
        __syncthreads();
        t = tn;
    }
}

// ---- the ensemble as one persistent launch over many steps
//
// One cooperative launch advances every run of an ensemble `nsteps` steps: as many CTAs as are
// resident walk the 56 x 24 tile table (largest runs first), step after step, with a grid-wide
// barrier between steps (a counter in global memory that every CTA increments once per step and
// polls, with a bounded number of polls; the host clears it before the launch).  Staging is per-
// thread cp.async.cg, which reads through L2, so a tile never sees a line cached in L1 from an
// earlier step (the ensemble's runs must have nx % 4 == 0 for that path).  A barrier wait that
// runs out sets ERR_BIT_TIMEOUT and the CTA leaves; the others then run out at their next barrier.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned target, int cap, int* err, int* abort_flag)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();  // this CTA's stores of the step, ordered before its arrival (after the bar.sync)
        atomicAdd(bar, 1u);
        unsigned v = 0;
        for (int it = 0;; ++it) {
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
            if (v >= target || it >= cap) break;
            __nanosleep(64);
        }
        *abort_flag = v < target;
        if (v < target && err) atomicOr(err, ERR_BIT_TIMEOUT);
        __threadfence();
    }
    __syncthreads();
    return !*abort_flag;
}

template <int TY, int S, int PHI_MODE, int MOB>
__global__ void __launch_bounds__(Geo<TY, S>::THREADS, Geo<TY, S>::MINB)
ens_persistent_kernel(const EnsTile* __restrict__ tiles, const EnsRun* __restrict__ runs, int ntiles, int parity,
                      int nsteps, unsigned* __restrict__ bar, int wait_cap, int* __restrict__ err)
{
    __shared__ int abort_flag;
    for (int s = 0; s < nsteps; ++s) {
        const int a = (parity + s) & 1;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
            const EnsTile e = tiles[t];
            const EnsRun& r = runs[e.run];
            step_tile<TY, S, PHI_MODE, MOB>(r.k, e.x0, e.y0, r.f[a][0], r.f[a][1], r.f[a][2], r.f[1 - a][0],
                                            r.f[1 - a][1], r.f[1 - a][2]);
            __syncthreads();  // the staging buffers are reused by the next tile
        }
        if (s + 1 < nsteps && !grid_barrier(bar, (unsigned)(s + 1) * gridDim.x, wait_cap, err, &abort_flag)) return;
    }
}

// ---- two explicit midpoint steps per launch (temporal blocking in shared memory)
//
// For grids that live in L2 the cost of a step is mostly its chain of launch, staging and store
// (a copy-only form of the one-step kernel takes 2.6 of its 4.95 us at 512^2).  This kernel pays
// that chain once for two steps: a CTA stages a 64 x (TY + 16) window of u^n (8-cell halo), then
// runs four stage passes, each consuming 2 cells of validity on every side:
//   A  u*      = u^n + dt/2 R(u^n)      rows [2, LY-2)   -> B
//   B  u^{n+1} = u^n + dt R(u*)         rows [4, LY-4)   -> U2 (shared memory)
//   C  u**     = u^{n+1} + dt/2 R(u^{n+1})  rows [6, LY-6) -> B
//   D  u^{n+2} = u^{n+1} + dt R(u**)    rows [8, 8+TY)   -> global memory, columns [8, 56): 48 per tile
// with the ghost rows of each shared-memory state filled where the tile touches the bottom or top.
// Every pass is stage(), the code of the one-step kernel, so two steps here equal two one-step
// launches bit for bit.
constexpr int HALO2 = 8;
constexpr int TXO2 = LX - 2 * HALO2;  // 48 output columns per tile

template <int TY, int S>
struct Geo2 {
    static constexpr int LY = TY + 2 * HALO2;  // staged rows
    static constexpr int PX = LX;
    static constexpr int PLANE = LY * PX;
    static constexpr int THREADS = 32 * S;
    static constexpr int cdiv(int a, int b) { return (a + b - 1) / b; }
    static constexpr int LA = cdiv(TY + 12, S), LB = cdiv(TY + 8, S), LC = cdiv(TY + 4, S), LD = cdiv(TY, S);
    static constexpr int GUARD = (LA + 4) * PX;  // rows read past the last plane by a segment's tail
    static constexpr size_t BYTES = (size_t(9) * PLANE + GUARD) * sizeof(float) + 128;  // u^n, u*, u^{n+1}
};

// Ghost rows of a staged state P (3 planes of LY rows, window rows from gy0) at the bottom and top
// of the domain, by the boundary rules of the staging: phi and c mirrored two rows deep, rho
// mirrored one row at the bottom and the reservoir value above the top.
template <class G>
__device__ __forceinline__ void ghost_rows(const StepConst& k, int gy0, float* __restrict__ P)
{
    constexpr int PX = G::PX, PLANE = G::PLANE, LY = G::LY;
    const int ny = k.ny;
    if (gy0 >= 0 && gy0 + LY <= ny) return;  // the window holds no row outside the domain
    for (int idx = threadIdx.x; idx < 3 * 2 * LX; idx += G::THREADS) {
        const int fld = idx / (2 * LX), rem = idx - fld * (2 * LX);
        const int d = rem / LX, x = rem - d * LX;  // ghost depth d + 1
        float* Q = P + fld * PLANE + x;
        const int gb = -1 - d, lb = gb - gy0, sb = reflect(gb, ny) - gy0;
        if (lb >= 0 && lb < LY && sb >= 0 && sb < LY && (fld < 2 || d == 0)) Q[lb * PX] = Q[sb * PX];
        const int gt = ny + d, lt = gt - gy0, st = reflect(gt, ny) - gy0;
        if (lt >= 0 && lt < LY) {
            if (fld == 2)
                Q[lt * PX] = (d == 0) ? k.rho_top : 0.f;
            else if (st >= 0 && st < LY)
                Q[lt * PX] = Q[st * PX];
        }
    }
}

template <int TY, int S, int PHI_MODE, int MOB, bool TMA>
__global__ void __launch_bounds__(Geo2<TY, S>::THREADS, 3)
step2_kernel(const StepConst k, const float* __restrict__ phi0, const float* __restrict__ c0,
             const float* __restrict__ rho0, float* __restrict__ phi1, float* __restrict__ c1,
             float* __restrict__ rho1, const __grid_constant__ StepMaps maps, int* __restrict__ err)
{
    using G = Geo2<TY, S>;
    constexpr int PX = G::PX, PLANE = G::PLANE, LY = G::LY;
    extern __shared__ __align__(128) float smraw[];
    float* const U = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(smraw) + 127) & ~uintptr_t(127));
    float* const B = U + 3 * PLANE;   // u* and u**
    float* const U2 = U + 6 * PLANE;  // u^{n+1} (followed by the guard rows)
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int gx0 = blockIdx.x * TXO2 - HALO2, gy0 = blockIdx.y * TY - HALO2;
    const int nx = k.nx, ny = k.ny, pitch = k.pitch;

    asm volatile("griddepcontrol.wait;" ::: "memory");
    bool staged = false;
    if (TMA && gx0 >= 0 && gx0 + LX <= nx && gy0 >= 0 && gy0 + LY <= ny) {
        __shared__ __align__(8) uint64_t mbar;
        const unsigned mb = (unsigned)__cvta_generic_to_shared(&mbar);
        if (tid == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncthreads();
        if (tid == 0) issue_tma_g<G>(&maps, gx0, gy0, U, mb);
        const unsigned done = poll_phase(mb, 0, k.wait_cap);
        if (__syncthreads_or(!done)) {
            if (tid == 0 && err) atomicOr(err, ERR_BIT_TIMEOUT);
            poll_phase(mb, 0, 1 << 22);  // let the copies in flight land before leaving
            return;
        }
        staged = true;
    }
    if (!staged) {
        issue_plain_g<G>(k, gx0, gy0, phi0, c0, rho0, U);
        asm volatile("cp.async.wait_all;" ::: "memory");
    }
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    __syncthreads();

    const int dlo = -gy0 > 0 ? -gy0 : 0;              // staged rows holding domain rows: [dlo, dhi)
    const int dhi = ny - gy0 < LY ? ny - gy0 : LY;
    const int lo2 = 2 * lane;
    auto lo = [&](int m) { return dlo > m ? dlo : m; };
    auto hi = [&](int m) { return dhi < LY - m ? dhi : LY - m; };
    int r0, n;
    // A: u* of step 1
    segment(lo(2), hi(2), S, warp, r0, n);
    stage<G::LA, PX, PLANE, PHI_MODE, MOB, 0>(k, U + lo2, nullptr, B + lo2, r0, n, nullptr, nullptr, nullptr, 0, 0,
                                              false, false);
    __syncthreads();
    ghost_rows<G>(k, gy0, B);
    __syncthreads();
    // B: u^{n+1} into shared memory
    segment(lo(4), hi(4), S, warp, r0, n);
    stage<G::LB, PX, PLANE, PHI_MODE, MOB, 2>(k, B + lo2, U + lo2, U2 + lo2, r0, n, nullptr, nullptr, nullptr, 0, 0,
                                              false, false);
    __syncthreads();
    ghost_rows<G>(k, gy0, U2);
    __syncthreads();
    // C: u* of step 2
    segment(lo(6), hi(6), S, warp, r0, n);
    stage<G::LC, PX, PLANE, PHI_MODE, MOB, 0>(k, U2 + lo2, nullptr, B + lo2, r0, n, nullptr, nullptr, nullptr, 0, 0,
                                              false, false);
    __syncthreads();
    ghost_rows<G>(k, gy0, B);
    __syncthreads();
    // D: u^{n+2} to global memory on the 48 x TY output cells
    segment(lo(HALO2), hi(HALO2), S, warp, r0, n);
    const int gx = gx0 + lo2;
    const bool store_x = (lo2 >= HALO2) && (lo2 < HALO2 + TXO2) && gx < nx;
    const size_t g_off = (size_t)(gy0 + r0) * pitch + (gx < 0 ? 0 : gx);
    stage<G::LD, PX, PLANE, PHI_MODE, MOB, 1>(k, B + lo2, U2 + lo2, nullptr, r0, n, phi1, c1, rho1, g_off, pitch,
                                              store_x, gx + 1 < nx);
}

// Opt the kernel into its dynamic shared-memory size (once per kernel function).
template <class Kern>
cudaError_t configure_smem(Kern kern, bool& configured, size_t smem)
{
    if (!configured) {  // the attribute is per function; setting it twice is harmless
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    return cudaSuccess;
}

// Launch configuration with programmatic dependent launch enabled.
cudaLaunchConfig_t pdl_config(dim3 grid, int threads, size_t smem, cudaStream_t s, cudaLaunchAttribute* attr)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

template <int TY, int S, int PHI_MODE, int MOB>
cudaError_t launch_t(const StepConst& k, const float* f0, const float* c0, const float* r0, float* f1,
                     float* c1, float* r1, cudaStream_t s, const StepMaps* maps, int* err)
{
    using G = Geo<TY, S>;
    const dim3 grid((k.nx + TXO - 1) / TXO, (k.ny + TY - 1) / TY);
    cudaLaunchAttribute attr[1];
    // TMA staging is built for the short and the large tile; the medium tile (ensembles only)
    // ignores the maps
    if constexpr ((TY == PF_LARGE_TY && S == PF_LARGE_S) || (TY == PF_SMALL_TY && S == PF_SMALL_S)) {
        if (maps) {
            auto kern = step_kernel_tma<TY, S, PHI_MODE, MOB>;
            static bool configured = false;
            cudaError_t e = configure_smem(kern, configured, G::TMA_BYTES);
            if (e != cudaSuccess) return e;
            cudaLaunchConfig_t cfg = pdl_config(grid, G::THREADS, G::TMA_BYTES, s, attr);
            return cudaLaunchKernelEx(&cfg, kern, k, f0, c0, r0, f1, c1, r1, *maps, err);
        }
    }
    auto kern = step_kernel<TY, S, PHI_MODE, MOB>;
    static bool configured = false;
    cudaError_t e = configure_smem(kern, configured, G::BYTES);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = pdl_config(grid, G::THREADS, G::BYTES, s, attr);
    return cudaLaunchKernelEx(&cfg, kern, k, f0, c0, r0, f1, c1, r1);
}

template <int TY, int S, int PHI_MODE, int MOB>
cudaError_t launch_euler_t(const StepConst& k, const float* f0, const float* c0, const float* r0, float* f1,
                           float* c1, float* r1, cudaStream_t s)
{
    using G = Geo<TY, S>;
    auto kern = euler_kernel<TY, S, PHI_MODE, MOB>;
    static bool configured = false;
    const dim3 grid((k.nx + TXO - 1) / TXO, (k.ny + TY - 1) / TY);
    cudaError_t e = configure_smem(kern, configured, G::BYTES);
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = pdl_config(grid, G::THREADS, G::BYTES, s, attr);
    return cudaLaunchKernelEx(&cfg, kern, k, f0, c0, r0, f1, c1, r1);
}

template <int TY, int S, int PHI_MODE, int MOB>
cudaError_t launch_ens_t(const EnsTile* tiles, const EnsRun* runs, int ntiles, int parity, cudaStream_t s,
                         const EnsMaps* maps, int* err)
{
    using G = Geo<TY, S>;
    const dim3 grid(ntiles);
    cudaLaunchAttribute attr[1];
    if constexpr ((TY == PF_LARGE_TY && S == PF_LARGE_S) || (TY == PF_SMALL_TY && S == PF_SMALL_S)) {
        if (maps) {
            auto kern = ens_step_kernel_tma<TY, S, PHI_MODE, MOB>;
            static bool configured = false;
            cudaError_t e = configure_smem(kern, configured, G::TMA_BYTES);
            if (e != cudaSuccess) return e;
            cudaLaunchConfig_t cfg = pdl_config(grid, G::THREADS, G::TMA_BYTES, s, attr);
            return cudaLaunchKernelEx(&cfg, kern, tiles, runs, parity, *maps, err);
        }
    }
    auto kern = ens_step_kernel<TY, S, PHI_MODE, MOB>;
    static bool configured = false;
    cudaError_t e = configure_smem(kern, configured, G::BYTES);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = pdl_config(grid, G::THREADS, G::BYTES, s, attr);
    return cudaLaunchKernelEx(&cfg, kern, tiles, runs, parity);
}

// Grid of a persistent kernel: as many CTAs as are resident at once (at most `ntiles`).
template <class Kern>
cudaError_t ring_grid(Kern kern, int threads, size_t smem, int ntiles, int& grid)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const long long g = (long long)sms * per_sm;
    grid = (int)(g < ntiles ? g : ntiles);
    return cudaSuccess;
}

template <class Kern>
cudaError_t configure_ring(Kern kern, bool& configured, size_t smem)
{
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        if (e != cudaSuccess) return e;
    }
    return configure_smem(kern, configured, smem);
}

template <int PHI_MODE, int MOB>
cudaError_t launch_ring_t(const StepConst& k, const float* f0, const float* c0, const float* r0, float* f1,
                          float* c1, float* r1, cudaStream_t s, const StepMaps* maps, int* err)
{
    constexpr int TY = PF_LARGE_TY, S = PF_LARGE_S;
    using G = Geo<TY, S>;
    auto kern = step_kernel_ring<TY, S, PHI_MODE, MOB>;
    static bool configured = false;
    static int grid_cache = 0;
    static int ntiles_cache = -1;
    const size_t smem = RingGeo<TY, S>::BYTES;
    cudaError_t e = configure_ring(kern, configured, smem);
    if (e != cudaSuccess) return e;
    const int ntiles = ((k.nx + TXO - 1) / TXO) * ((k.ny + TY - 1) / TY);
    if (ntiles != ntiles_cache) {
        e = ring_grid(kern, G::THREADS, smem, ntiles, grid_cache);
        if (e != cudaSuccess) return e;
        ntiles_cache = ntiles;
    }
    StepMaps none = {};
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = pdl_config(dim3(grid_cache), G::THREADS, smem, s, attr);
    return cudaLaunchKernelEx(&cfg, kern, k, f0, c0, r0, f1, c1, r1, maps ? *maps : none, maps ? 1 : 0, err);
}

template <int PHI_MODE, int MOB>
cudaError_t launch_ens_ring_t(const EnsTile* tiles, const EnsRun* runs, int ntiles, int parity, cudaStream_t s)
{
    constexpr int TY = PF_LARGE_TY, S = PF_LARGE_S;
    using G = Geo<TY, S>;
    auto kern = ens_step_kernel_ring<TY, S, PHI_MODE, MOB>;
    static bool configured = false;
    static int grid_cache = 0;
    static int ntiles_cache = -1;
    const size_t smem = RingGeo<TY, S>::BYTES;
    cudaError_t e = configure_ring(kern, configured, smem);
    if (e != cudaSuccess) return e;
    if (ntiles != ntiles_cache) {
        e = ring_grid(kern, G::THREADS, smem, ntiles, grid_cache);
        if (e != cudaSuccess) return e;
        ntiles_cache = ntiles;
    }
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = pdl_config(dim3(grid_cache), G::THREADS, smem, s, attr);
    return cudaLaunchKernelEx(&cfg, kern, tiles, runs, ntiles, parity);
}

#ifndef PF_STEP2_TY
#define PF_STEP2_TY 16
#endif

template <int PHI_MODE, int MOB>
cudaError_t launch_step2_t(const StepConst& k, const float* f0, const float* c0, const float* r0, float* f1,
                           float* c1, float* r1, cudaStream_t s, const StepMaps* maps, int* err)
{
    constexpr int TY = PF_STEP2_TY, S = 4;
    using G = Geo2<TY, S>;
    const dim3 grid((k.nx + TXO2 - 1) / TXO2, (k.ny + TY - 1) / TY);
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = pdl_config(grid, G::THREADS, G::BYTES, s, attr);
    StepMaps none = {};
    if (maps) {
        auto kern = step2_kernel<TY, S, PHI_MODE, MOB, true>;
        static bool configured = false;
        cudaError_t e = configure_smem(kern, configured, G::BYTES);
        if (e != cudaSuccess) return e;
        return cudaLaunchKernelEx(&cfg, kern, k, f0, c0, r0, f1, c1, r1, *maps, err);
    }
    auto kern = step2_kernel<TY, S, PHI_MODE, MOB, false>;
    static bool configured = false;
    cudaError_t e = configure_smem(kern, configured, G::BYTES);
    if (e != cudaSuccess) return e;
    return cudaLaunchKernelEx(&cfg, kern, k, f0, c0, r0, f1, c1, r1, none, err);
}

template <int PHI_MODE, int MOB>
cudaError_t launch_ens_persistent_t(const EnsTile* tiles, const EnsRun* runs, int ntiles, int parity, int nsteps,
                                    unsigned* bar, int wait_cap, int* err, cudaStream_t s)
{
    constexpr int TY = PF_LARGE_TY, S = PF_LARGE_S;
    using G = Geo<TY, S>;
    auto kern = ens_persistent_kernel<TY, S, PHI_MODE, MOB>;
    static bool configured = false;
    static int grid_cache = 0;
    static int ntiles_cache = -1;
    cudaError_t e = configure_smem(kern, configured, G::BYTES);
    if (e != cudaSuccess) return e;
    if (ntiles != ntiles_cache) {
        e = ring_grid(kern, G::THREADS, G::BYTES, ntiles, grid_cache);
        if (e != cudaSuccess) return e;
        ntiles_cache = ntiles;
    }
    e = cudaMemsetAsync(bar, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid_cache);
    cfg.blockDim = dim3(G::THREADS);
    cfg.dynamicSmemBytes = G::BYTES;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;  // all CTAs resident at once: the barrier relies on it
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, tiles, runs, ntiles, parity, nsteps, bar, wait_cap, err);
}

template <int TY, int S>
cudaError_t launch_tile(const StepConst& k, int phi_mode, int mob, const float* f0, const float* c0,
                        const float* r0, float* f1, float* c1, float* r1, cudaStream_t s, const StepMaps* maps,
                        int* err)
{
    if (phi_mode == 0) {
        if (mob == MOB_UNIFORM) return launch_t<TY, S, 0, MOB_UNIFORM>(k, f0, c0, r0, f1, c1, r1, s, maps, err);
        if (mob == MOB_BULK) return launch_t<TY, S, 0, MOB_BULK>(k, f0, c0, r0, f1, c1, r1, s, maps, err);
        return launch_t<TY, S, 0, MOB_SURF>(k, f0, c0, r0, f1, c1, r1, s, maps, err);
    }
    if (mob == MOB_UNIFORM) return launch_t<TY, S, 1, MOB_UNIFORM>(k, f0, c0, r0, f1, c1, r1, s, maps, err);
    if (mob == MOB_BULK) return launch_t<TY, S, 1, MOB_BULK>(k, f0, c0, r0, f1, c1, r1, s, maps, err);
    return launch_t<TY, S, 1, MOB_SURF>(k, f0, c0, r0, f1, c1, r1, s, maps, err);
}

template <int TY, int S>
cudaError_t launch_ens_tile(int phi_mode, int mob, const EnsTile* tiles, const EnsRun* runs, int ntiles,
                            int parity, cudaStream_t s, const EnsMaps* maps, int* err)
{
    if (phi_mode == 0) {
        if (mob == MOB_UNIFORM) return launch_ens_t<TY, S, 0, MOB_UNIFORM>(tiles, runs, ntiles, parity, s, maps, err);
        if (mob == MOB_BULK) return launch_ens_t<TY, S, 0, MOB_BULK>(tiles, runs, ntiles, parity, s, maps, err);
        return launch_ens_t<TY, S, 0, MOB_SURF>(tiles, runs, ntiles, parity, s, maps, err);
    }
    if (mob == MOB_UNIFORM) return launch_ens_t<TY, S, 1, MOB_UNIFORM>(tiles, runs, ntiles, parity, s, maps, err);
    if (mob == MOB_BULK) return launch_ens_t<TY, S, 1, MOB_BULK>(tiles, runs, ntiles, parity, s, maps, err);
    return launch_ens_t<TY, S, 1, MOB_SURF>(tiles, runs, ntiles, parity, s, maps, err);
}

}  // namespace

int choose_tile(int nx, int ny)
{
    // Grids up to ~1M cells need the short tile to give every SM several CTAs.
    return (long long)nx * ny <= (1LL << 20) ? TILE_SMALL : TILE_LARGE;
}

int tile_width() { return TXO; }

int tile_height(int tile)
{
    return tile == TILE_SMALL ? PF_SMALL_TY : (tile == TILE_MEDIUM ? PF_MEDIUM_TY : PF_LARGE_TY);
}

int tile_table(int tile) { return (tile == TILE_LARGE_RING || tile == TILE_LARGE_PERSIST) ? TILE_LARGE : tile; }

size_t step_smem_bytes(int tile)
{
    if (tile == TILE_SMALL) return Geo<PF_SMALL_TY, PF_SMALL_S>::BYTES;
    if (tile == TILE_MEDIUM) return Geo<PF_MEDIUM_TY, PF_MEDIUM_S>::BYTES;
    return Geo<PF_LARGE_TY, PF_LARGE_S>::BYTES;
}

cudaError_t launch_step(const StepConst& k, int tile, int phi_mode, int mob, const float* f0, const float* c0,
                        const float* r0, float* f1, float* c1, float* r1, cudaStream_t s, const StepMaps* maps,
                        int* err)
{
    if (tile == TILE_SMALL)
        return launch_tile<PF_SMALL_TY, PF_SMALL_S>(k, phi_mode, mob, f0, c0, r0, f1, c1, r1, s, maps, err);
    if (tile == TILE_MEDIUM)
        return launch_tile<PF_MEDIUM_TY, PF_MEDIUM_S>(k, phi_mode, mob, f0, c0, r0, f1, c1, r1, s, maps, err);
    return launch_tile<PF_LARGE_TY, PF_LARGE_S>(k, phi_mode, mob, f0, c0, r0, f1, c1, r1, s, maps, err);
}

cudaError_t launch_step_ring(const StepConst& k, int phi_mode, int mob, const float* f0, const float* c0,
                             const float* r0, float* f1, float* c1, float* r1, cudaStream_t s, const StepMaps* maps,
                             int* err)
{
    if (phi_mode == 0) {
        if (mob == MOB_UNIFORM) return launch_ring_t<0, MOB_UNIFORM>(k, f0, c0, r0, f1, c1, r1, s, maps, err);
        if (mob == MOB_BULK) return launch_ring_t<0, MOB_BULK>(k, f0, c0, r0, f1, c1, r1, s, maps, err);
        return launch_ring_t<0, MOB_SURF>(k, f0, c0, r0, f1, c1, r1, s, maps, err);
    }
    if (mob == MOB_UNIFORM) return launch_ring_t<1, MOB_UNIFORM>(k, f0, c0, r0, f1, c1, r1, s, maps, err);
    if (mob == MOB_BULK) return launch_ring_t<1, MOB_BULK>(k, f0, c0, r0, f1, c1, r1, s, maps, err);
    return launch_ring_t<1, MOB_SURF>(k, f0, c0, r0, f1, c1, r1, s, maps, err);
}

cudaError_t launch_step2(const StepConst& k, int phi_mode, int mob, const float* f0, const float* c0,
                         const float* r0, float* f1, float* c1, float* r1, cudaStream_t s, const StepMaps* maps,
                         int* err)
{
    if (phi_mode == 0) {
        if (mob == MOB_UNIFORM) return launch_step2_t<0, MOB_UNIFORM>(k, f0, c0, r0, f1, c1, r1, s, maps, err);
        if (mob == MOB_BULK) return launch_step2_t<0, MOB_BULK>(k, f0, c0, r0, f1, c1, r1, s, maps, err);
        return launch_step2_t<0, MOB_SURF>(k, f0, c0, r0, f1, c1, r1, s, maps, err);
    }
    if (mob == MOB_UNIFORM) return launch_step2_t<1, MOB_UNIFORM>(k, f0, c0, r0, f1, c1, r1, s, maps, err);
    if (mob == MOB_BULK) return launch_step2_t<1, MOB_BULK>(k, f0, c0, r0, f1, c1, r1, s, maps, err);
    return launch_step2_t<1, MOB_SURF>(k, f0, c0, r0, f1, c1, r1, s, maps, err);
}

cudaError_t launch_ens_persistent(int phi_mode, int mob, const EnsTile* tiles, const EnsRun* runs, int ntiles,
                                  int parity, int nsteps, unsigned* bar, int wait_cap, int* err, cudaStream_t s)
{
    if (ntiles <= 0 || nsteps <= 0) return cudaSuccess;
    if (phi_mode == 0) {
        if (mob == MOB_UNIFORM)
            return launch_ens_persistent_t<0, MOB_UNIFORM>(tiles, runs, ntiles, parity, nsteps, bar, wait_cap, err, s);
        if (mob == MOB_BULK)
            return launch_ens_persistent_t<0, MOB_BULK>(tiles, runs, ntiles, parity, nsteps, bar, wait_cap, err, s);
        return launch_ens_persistent_t<0, MOB_SURF>(tiles, runs, ntiles, parity, nsteps, bar, wait_cap, err, s);
    }
    if (mob == MOB_UNIFORM)
        return launch_ens_persistent_t<1, MOB_UNIFORM>(tiles, runs, ntiles, parity, nsteps, bar, wait_cap, err, s);
    if (mob == MOB_BULK)
        return launch_ens_persistent_t<1, MOB_BULK>(tiles, runs, ntiles, parity, nsteps, bar, wait_cap, err, s);
    return launch_ens_persistent_t<1, MOB_SURF>(tiles, runs, ntiles, parity, nsteps, bar, wait_cap, err, s);
}

int step2_box_rows() { return PF_STEP2_TY + 2 * HALO2; }
int step2_tile_width() { return TXO2; }
int step2_tile_height() { return PF_STEP2_TY; }

cudaError_t launch_euler(const StepConst& k, int phi_mode, int mob, const float* f0, const float* c0,
                         const float* r0, float* f1, float* c1, float* r1, cudaStream_t s)
{
    constexpr int TY = PF_SMALL_TY, S = PF_SMALL_S;
    if (phi_mode == 0) {
        if (mob == MOB_UNIFORM) return launch_euler_t<TY, S, 0, MOB_UNIFORM>(k, f0, c0, r0, f1, c1, r1, s);
        if (mob == MOB_BULK) return launch_euler_t<TY, S, 0, MOB_BULK>(k, f0, c0, r0, f1, c1, r1, s);
        return launch_euler_t<TY, S, 0, MOB_SURF>(k, f0, c0, r0, f1, c1, r1, s);
    }
    if (mob == MOB_UNIFORM) return launch_euler_t<TY, S, 1, MOB_UNIFORM>(k, f0, c0, r0, f1, c1, r1, s);
    if (mob == MOB_BULK) return launch_euler_t<TY, S, 1, MOB_BULK>(k, f0, c0, r0, f1, c1, r1, s);
    return launch_euler_t<TY, S, 1, MOB_SURF>(k, f0, c0, r0, f1, c1, r1, s);
}

cudaError_t launch_ens_step(int tile, int phi_mode, int mob, const EnsTile* tiles, const EnsRun* runs, int ntiles,
                            int parity, cudaStream_t s, const EnsMaps* maps, int* err)
{
    if (ntiles <= 0) return cudaSuccess;
    if (tile == TILE_LARGE_RING) {
        if (phi_mode == 0) {
            if (mob == MOB_UNIFORM) return launch_ens_ring_t<0, MOB_UNIFORM>(tiles, runs, ntiles, parity, s);
            if (mob == MOB_BULK) return launch_ens_ring_t<0, MOB_BULK>(tiles, runs, ntiles, parity, s);
            return launch_ens_ring_t<0, MOB_SURF>(tiles, runs, ntiles, parity, s);
        }
        if (mob == MOB_UNIFORM) return launch_ens_ring_t<1, MOB_UNIFORM>(tiles, runs, ntiles, parity, s);
        if (mob == MOB_BULK) return launch_ens_ring_t<1, MOB_BULK>(tiles, runs, ntiles, parity, s);
        return launch_ens_ring_t<1, MOB_SURF>(tiles, runs, ntiles, parity, s);
    }
    if (tile == TILE_SMALL)
        return launch_ens_tile<PF_SMALL_TY, PF_SMALL_S>(phi_mode, mob, tiles, runs, ntiles, parity, s, maps, err);
    if (tile == TILE_MEDIUM)  // no TMA form: per-thread staging
        return launch_ens_tile<PF_MEDIUM_TY, PF_MEDIUM_S>(phi_mode, mob, tiles, runs, ntiles, parity, s, nullptr,
                                                          nullptr);
    return launch_ens_tile<PF_LARGE_TY, PF_LARGE_S>(phi_mode, mob, tiles, runs, ntiles, parity, s, maps, err);
}

}  // namespace pf
