// Fused explicit-midpoint step of the phase-field PVD model (arXiv 2312.05410,
// Materials and Methods: composition Cahn-Hilliard equation with mobility
// M^Bulk + M^Surf, order-parameter equation with deposition source
// S = grad(phi).(rho v), vapor convection-diffusion; "Dataset": second-order
// central differences, explicit midpoint in time).
//
// One CTA owns a TX x TY block of output cells.  It stages (TX+8) x (TY+8)
// cells of phi, c, rho (4-cell halo, periodic wrap in x) in shared memory and
// runs four dependent levels there, each one ring narrower:
//   L1  mu_c, mu_phi, M_c        of u^n       (5-point Laplacians)
//   L2  u* = u^n + dt/2 R(u^n)               (flux divergences, source, vapor)
//   L3  mu_c, mu_phi, M_c        of u*
//   L4  u^{n+1} = u^n + dt R(u*) -> global memory
// so a step is one launch with 24 B of algorithmic HBM traffic per cell.
//
// Work layout: every thread owns four x-adjacent columns (a quad) and, in each
// level, streams down a segment of rows with a three-row register window, so a
// vertical neighbour is a register and each staged value is loaded from shared
// memory once per level as one 16-byte load (plus the two scalar west/east
// neighbours of the quad).  Quads are computed as two pairs with packed FP32x2
// arithmetic (fma/add/mul .f32x2).
//
// Boundary rules are applied once, where a level stores its results: the
// bottom and top domain rows are also written into the ghost row outside them
// (mirror), except that rho's ghost row above the top holds the reservoir
// value; the stencils themselves have no boundary branches.  Only domain rows
// are computed, so a ghost row has exactly one writer.
#include "pf_internal.h"

namespace pf {
namespace {

typedef float2 f2;
__device__ __forceinline__ f2 F2(float a) { return make_float2(a, a); }
__device__ __forceinline__ f2 add2(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 mul2(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }

// Four x-adjacent cells as two packed pairs: lo = (x, x+1), hi = (x+2, x+3).
struct q4 {
    f2 lo, hi;
};
__device__ __forceinline__ q4 Q(float a) { return {F2(a), F2(a)}; }
__device__ __forceinline__ q4 qadd(q4 a, q4 b) { return {add2(a.lo, b.lo), add2(a.hi, b.hi)}; }
__device__ __forceinline__ q4 qmul(q4 a, q4 b) { return {mul2(a.lo, b.lo), mul2(a.hi, b.hi)}; }
__device__ __forceinline__ q4 qfma(q4 a, q4 b, q4 c) { return {fma2(a.lo, b.lo, c.lo), fma2(a.hi, b.hi, c.hi)}; }
__device__ __forceinline__ q4 qsub(q4 a, q4 b) { return qfma(b, Q(-1.f), a); }
__device__ __forceinline__ q4 qneg(q4 a) { return {make_float2(-a.lo.x, -a.lo.y), make_float2(-a.hi.x, -a.hi.y)}; }
__device__ __forceinline__ q4 ld4(const float* p)
{
    const float4 v = *reinterpret_cast<const float4*>(p);
    return {make_float2(v.x, v.y), make_float2(v.z, v.w)};
}
__device__ __forceinline__ void st4(float* p, q4 v)
{
    *reinterpret_cast<float4*>(p) = make_float4(v.lo.x, v.lo.y, v.hi.x, v.hi.y);
}
// Horizontal neighbour sums u[x-1] + u[x+1] of the quad, given its west and east neighbours.
__device__ __forceinline__ q4 hsum(float W, q4 C, float E)
{
    return {make_float2(W + C.lo.y, C.lo.x + C.hi.x), make_float2(C.lo.y + C.hi.y, C.hi.x + E)};
}
// Central differences u[x+1] - u[x-1] of the quad.
__device__ __forceinline__ q4 hdiff(float W, q4 C, float E)
{
    return {make_float2(C.lo.y - W, C.hi.x - C.lo.x), make_float2(C.hi.y - C.lo.y, E - C.hi.x)};
}

constexpr int HALO = 4;
constexpr int PAD = 4;  // left padding of a staged row (keeps 16-B alignment)

template <int TX, int TY, int S>
struct Geo {
    static_assert(TX % 4 == 0, "tile width must be a multiple of 4");
    static constexpr int LX = TX + 2 * HALO;  // staged columns
    static constexpr int LY = TY + 2 * HALO;  // staged rows
    static constexpr int PX = LX + PAD;       // row pitch in floats; the east neighbour of the last
                                              // column reads the next row's padding (never used)
    static constexpr int PLANE = LY * PX;
    static constexpr int NQC = LX / 4;        // quad columns = threads per row segment
    static constexpr int THREADS = NQC * S;   // S row segments
    static constexpr size_t BYTES = (size_t(9) * PLANE + 8) * sizeof(float);  // + tail guard
    static constexpr int cdiv(int a, int b) { return (a + b - 1) / b; }
    static constexpr int L1 = cdiv(LY - 2, S);  // longest segment of each level
    static constexpr int L2 = cdiv(LY - 4, S);
    static constexpr int L3 = cdiv(LY - 6, S);
    static constexpr int L4 = cdiv(TY, S);
};

// p(phi) = 1/4 (2-phi)(1+phi)^2 = 1/2 + 3/4 phi - 1/4 phi^3
__device__ __forceinline__ q4 p_of(q4 f, q4 ff) { return qfma(qfma(Q(-0.25f), ff, Q(0.75f)), f, Q(0.5f)); }

// Rows [lo, hi) of a level split into S near-equal segments; segment s of them.
__device__ __forceinline__ void segment(int lo, int hi, int S, int s, int& r0, int& n)
{
    const int H = hi > lo ? hi - lo : 0;
    r0 = lo + (s * H) / S;
    n = lo + ((s + 1) * H) / S - r0;
}

// L1 / L3: mu_c, mu_phi and M_c of the staged (phi, c) over rows [r0, r0+n) of one
// quad column; o is the offset of (row 0, this quad) in a plane.
template <int L, int PX, int MOB>
__device__ __forceinline__ void level_mu(const StepConst& k, const float* __restrict__ P,
                                         const float* __restrict__ Cp, float* __restrict__ A0,
                                         float* __restrict__ A1, float* __restrict__ A2, int o, int r0, int n,
                                         int gy_r0, int ny)
{
    q4 fw[3], cw[3];
    const int b = o + r0 * PX;
    fw[0] = ld4(P + b - PX);
    fw[1] = ld4(P + b);
    cw[0] = ld4(Cp + b - PX);
    cw[1] = ld4(Cp + b);
#pragma unroll
    for (int i = 0; i < L; ++i) {
        if (i < n) {
            const int iS = i % 3, iC = (i + 1) % 3, iN = (i + 2) % 3;
            const int q = b + i * PX;
            fw[iN] = ld4(P + q + PX);
            cw[iN] = ld4(Cp + q + PX);
            const q4 f = fw[iC], c = cw[iC];
            const q4 sf = qadd(hsum(P[q - 1], f, P[q + 4]), qadd(fw[iN], fw[iS]));
            const q4 sc = qadd(hsum(Cp[q - 1], c, Cp[q + 4]), qadd(cw[iN], cw[iS]));
            const q4 ff = qmul(f, f);
            const q4 p = p_of(f, ff);
            const q4 qq = qfma(qneg(c), c, c);                                  // c (1 - c)
            const q4 g = qmul(qq, qq);                                          // g(c)
            const q4 Wdg = qmul(qq, qfma(Q(-4.f * k.Wc), c, Q(2.f * k.Wc)));  // W_c g'(c)
            // mu_c = p W_c g' - kappa_c L(c)
            q4 muc = qfma(Q(4.f * k.kc), c, qmul(p, Wdg));
            muc = qfma(Q(-k.kc), sc, muc);
            // mu_phi = -W_phi phi (1 - phi^2) + p'(phi) W_c g - kappa_phi L(phi),  p' = 3/4 (1 - phi^2)
            q4 muf = qmul(qfma(Q(k.Wf), ff, Q(-k.Wf)), f);
            muf = qfma(qfma(Q(-0.75f * k.Wc), ff, Q(0.75f * k.Wc)), g, muf);
            muf = qfma(Q(4.f * k.kf), f, muf);
            muf = qfma(Q(-k.kf), sf, muf);
            // M_c = p (MB + h dM) [+ exp(-(phi/sigma)^2)(MBs + h dMs)],  h = c^2 (3 - 2c)
            q4 M;
            if (MOB == MOB_UNIFORM) {
                M = qmul(p, Q(k.MBb));
            } else {
                const q4 h = qmul(qmul(c, c), qfma(Q(-2.f), c, Q(3.f)));
                M = qmul(p, qfma(h, Q(k.dMb), Q(k.MBb)));
                if (MOB == MOB_SURF) {
                    const q4 t = qmul(ff, Q(k.nisig2));
                    const q4 e = {make_float2(exp2f(t.lo.x), exp2f(t.lo.y)), make_float2(exp2f(t.hi.x), exp2f(t.hi.y))};
                    M = qfma(e, qfma(h, Q(k.dMs), Q(k.MBs)), M);
                }
            }
            st4(A0 + q, muc);
            st4(A1 + q, muf);
            st4(A2 + q, M);
        }
    }
    if (n > 0) {  // mirror ghosts outside the bottom / top domain rows (own writes: no barrier)
        if (gy_r0 == 0) {
            st4(A0 + b - PX, ld4(A0 + b));
            st4(A1 + b - PX, ld4(A1 + b));
            st4(A2 + b - PX, ld4(A2 + b));
        }
        const int t = b + (n - 1) * PX;
        if (gy_r0 + n - 1 == ny - 1) {
            st4(A0 + t + PX, ld4(A0 + t));
            st4(A1 + t + PX, ld4(A1 + t));
            st4(A2 + t + PX, ld4(A2 + t));
        }
    }
}

// L2 / L4: right-hand side of one quad column over rows [r0, r0+n).
// A0..A2: mu_c, mu_phi, M; P, R: the phi and rho the source and vapor terms use;
// Uc: the state the update starts from (phi, c, rho planes at Uc, Uc+PLANE, Uc+2 PLANE).
// FINAL = false: u* = u^n + dt/2 R into Bout (with ghost rows); true: u^{n+1} to global.
template <int L, int PX, int PLANE, int PHI_MODE, bool FINAL>
__device__ __forceinline__ void level_rhs(const StepConst& k, const float* __restrict__ A0,
                                          const float* __restrict__ A1, const float* __restrict__ A2,
                                          const float* __restrict__ P, const float* __restrict__ R,
                                          const float* __restrict__ Uc, float* __restrict__ Bout, int o, int r0,
                                          int n, int gy_r0, int ny, float* __restrict__ g_phi,
                                          float* __restrict__ g_c, float* __restrict__ g_rho, size_t g_off,
                                          int pitch, bool store_x, int valid_x)
{
    q4 mw[3], Mw[3], uw[3], fw[3], rw[3];
    const int b = o + r0 * PX;
    mw[0] = ld4(A0 + b - PX); mw[1] = ld4(A0 + b);
    Mw[0] = ld4(A2 + b - PX); Mw[1] = ld4(A2 + b);
    fw[0] = ld4(P + b - PX);  fw[1] = ld4(P + b);
    rw[0] = ld4(R + b - PX);  rw[1] = ld4(R + b);
    if (PHI_MODE == 0) { uw[0] = ld4(A1 + b - PX); uw[1] = ld4(A1 + b); }
    const q4 hdt = Q(FINAL ? k.dt : 0.5f * k.dt);
#pragma unroll
    for (int i = 0; i < L; ++i) {
        if (i < n) {
            const int iS = i % 3, iC = (i + 1) % 3, iN = (i + 2) % 3;
            const int q = b + i * PX;
            mw[iN] = ld4(A0 + q + PX);
            Mw[iN] = ld4(A2 + q + PX);
            fw[iN] = ld4(P + q + PX);
            rw[iN] = ld4(R + q + PX);
            if (PHI_MODE == 0) uw[iN] = ld4(A1 + q + PX);

            // conserved composition flux: sum_faces (M + M_nb)(mu_nb - mu) / (2 dx^2)
            const q4 m = mw[iC], M = Mw[iC];
            const float mW = A0[q - 1], mE = A0[q + 4], MW = A2[q - 1], ME = A2[q + 4];
            const float F0 = (MW + M.lo.x) * (m.lo.x - mW);       // face (x-1 | x)
            const float F1 = (M.lo.x + M.lo.y) * (m.lo.y - m.lo.x);  // face (x | x+1)
            const float F2_ = (M.lo.y + M.hi.x) * (m.hi.x - m.lo.y);
            const float F3 = (M.hi.x + M.hi.y) * (m.hi.y - m.hi.x);
            const float F4 = (M.hi.y + ME) * (mE - m.hi.y);         // face (x+3 | x+4)
            q4 rc = {make_float2(F1 - F0, F2_ - F1), make_float2(F3 - F2_, F4 - F3)};
            rc = qfma(qadd(M, Mw[iN]), qsub(mw[iN], m), rc);
            rc = qfma(qadd(M, Mw[iS]), qsub(mw[iS], m), rc);

            // deposition source S = grad(phi) . (rho v), central differences
            const q4 f = fw[iC], r = rw[iC];
            const float fW = P[q - 1], fE = P[q + 4], rW = R[q - 1], rE = R[q + 4];
            const q4 Src = qmul(r, qfma(Q(k.ax), hdiff(fW, f, fE), qmul(Q(k.ay), qsub(fw[iN], fw[iS]))));

            q4 Rf;
            if (PHI_MODE == 0) {
                const q4 u = uw[iC];
                const q4 su = qadd(hsum(A1[q - 1], u, A1[q + 4]), qadd(uw[iN], uw[iS]));
                Rf = qfma(Q(k.cF), qfma(Q(-4.f), u, su), Src);
            } else {
                Rf = qfma(Q(k.cF), ld4(A1 + q), Src);
            }
            // vapor: D L(rho) - div(rho v) - S (the ghost above the top row holds rho_top)
            const q4 lap = qfma(Q(-4.f), r, qadd(hsum(rW, r, rE), qadd(rw[iN], rw[iS])));
            const q4 adv = qfma(Q(k.ax), hdiff(rW, r, rE), qmul(Q(k.ay), qsub(rw[iN], rw[iS])));
            const q4 Rr = qsub(qfma(Q(k.cD), lap, qneg(adv)), Src);

            const q4 of = qfma(hdt, Rf, ld4(Uc + q));
            const q4 oc = qfma(hdt, qmul(rc, Q(k.cR)), ld4(Uc + PLANE + q));
            const q4 orr = qfma(hdt, Rr, ld4(Uc + 2 * PLANE + q));
            if (!FINAL) {
                st4(Bout + q, of);
                st4(Bout + PLANE + q, oc);
                st4(Bout + 2 * PLANE + q, orr);
            } else if (store_x) {
                const size_t g = g_off + size_t(i) * pitch;
                if (valid_x >= 4) {
                    st4(g_phi + g, of);
                    st4(g_c + g, oc);
                    st4(g_rho + g, orr);
                } else {
                    const float vf[4] = {of.lo.x, of.lo.y, of.hi.x, of.hi.y};
                    const float vc[4] = {oc.lo.x, oc.lo.y, oc.hi.x, oc.hi.y};
                    const float vr[4] = {orr.lo.x, orr.lo.y, orr.hi.x, orr.hi.y};
#pragma unroll
                    for (int e = 0; e < 3; ++e)
                        if (e < valid_x) {
                            g_phi[g + e] = vf[e];
                            g_c[g + e] = vc[e];
                            g_rho[g + e] = vr[e];
                        }
                }
            }
        }
    }
    if (!FINAL && n > 0) {  // ghosts: mirror below the bottom row; above the top, mirror and rho_top
        if (gy_r0 == 0) {
            st4(Bout + b - PX, ld4(Bout + b));
            st4(Bout + PLANE + b - PX, ld4(Bout + PLANE + b));
            st4(Bout + 2 * PLANE + b - PX, ld4(Bout + 2 * PLANE + b));
        }
        const int t = b + (n - 1) * PX;
        if (gy_r0 + n - 1 == ny - 1) {
            st4(Bout + t + PX, ld4(Bout + t));
            st4(Bout + PLANE + t + PX, ld4(Bout + PLANE + t));
            st4(Bout + 2 * PLANE + t + PX, Q(k.rho_top));
        }
    }
}

template <int TX, int TY, int S, int PHI_MODE, int MOB>
__global__ void __launch_bounds__(Geo<TX, TY, S>::THREADS)
step_kernel(const StepConst k, const float* __restrict__ phi0, const float* __restrict__ c0,
            const float* __restrict__ rho0, float* __restrict__ phi1, float* __restrict__ c1,
            float* __restrict__ rho1)
{
    using G = Geo<TX, TY, S>;
    constexpr int PX = G::PX, PLANE = G::PLANE;
    extern __shared__ __align__(16) float sm[];
    float* const U = sm;               // u^n: phi, c, rho
    float* const A = sm + 3 * PLANE;   // mu_c, mu_phi, M
    float* const B = sm + 6 * PLANE;   // u*: phi, c, rho

    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int gx0 = x0 - HALO, gy0 = y0 - HALO;
    const int nx = k.nx, ny = k.ny, pitch = k.pitch;

    // Wait for the previous step's grid (programmatic dependent launch) before reading.
    asm volatile("griddepcontrol.wait;" ::: "memory");

    // ---- stage u^n: domain rows, plus the ghost rows -1 and ny by the boundary rules
    // (mirror; rho above the top = rho_top); other out-of-domain rows are zero.
    // Every 16-byte group is an asynchronous global->shared copy, all in flight at once.
    {
        auto field = [&](int f) { return f == 0 ? phi0 : (f == 1 ? c0 : rho0); };
        auto wrap = [&](int gx) {  // periodic x; one correction suffices when nx >= LX
            if (nx >= G::LX) {
                gx = gx < 0 ? gx + nx : gx;
                return gx >= nx ? gx - nx : gx;
            }
            gx %= nx;
            return gx < 0 ? gx + nx : gx;
        };
        if ((nx & 3) == 0) {
            // x0 and nx are multiples of 4: each aligned group of 4 staged columns is
            // wholly inside [0, nx) or wholly wrapped
            constexpr int Q = G::LX / 4;
            for (int idx = tid; idx < 3 * G::LY * Q; idx += G::THREADS) {
                const int fld = idx / (G::LY * Q);
                const int rem = idx - fld * (G::LY * Q);
                const int ly = rem / Q, q = rem - ly * Q;
                int gy = gy0 + ly;
                float* dst = U + fld * PLANE + ly * PX + PAD + 4 * q;
                if ((fld == 2 && gy == ny) || gy < -1 || gy > ny) {
                    const float v = (gy == ny) ? k.rho_top : 0.f;
                    *reinterpret_cast<float4*>(dst) = make_float4(v, v, v, v);
                } else {
                    gy = gy < 0 ? 0 : (gy >= ny ? ny - 1 : gy);
                    const float* src = field(fld) + (size_t)gy * pitch + wrap(gx0 + 4 * q);
                    const unsigned sdst = (unsigned)__cvta_generic_to_shared(dst);
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sdst), "l"(src) : "memory");
                }
            }
            asm volatile("cp.async.wait_all;" ::: "memory");
        } else {
            for (int idx = tid; idx < 3 * G::LY * G::LX; idx += G::THREADS) {
                const int fld = idx / (G::LY * G::LX);
                const int rem = idx - fld * (G::LY * G::LX);
                const int ly = rem / G::LX, lx = rem - ly * G::LX;
                int gy = gy0 + ly;
                float v = 0.f;
                if (fld == 2 && gy == ny) {
                    v = k.rho_top;
                } else if (gy >= -1 && gy <= ny) {
                    gy = gy < 0 ? 0 : (gy >= ny ? ny - 1 : gy);
                    v = __ldg(field(fld) + (size_t)gy * pitch + wrap(gx0 + lx));
                }
                U[fld * PLANE + ly * PX + PAD + lx] = v;
            }
        }
    }
    // Let the next step's grid begin launching; it waits for this grid to finish.
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    __syncthreads();

    const int qc = tid % G::NQC, s = tid / G::NQC;
    const int o = PAD + 4 * qc;
    // staged rows holding domain rows: [dlo, dhi)
    const int dlo = -gy0 > 0 ? -gy0 : 0;
    const int dhi = ny - gy0 < G::LY ? ny - gy0 : G::LY;
    int r0, n;

    // ---- L1: mu, M of u^n on staged rows [1, LY-1)
    segment(dlo > 1 ? dlo : 1, dhi < G::LY - 1 ? dhi : G::LY - 1, S, s, r0, n);
    level_mu<G::L1, PX, MOB>(k, U, U + PLANE, A, A + PLANE, A + 2 * PLANE, o, r0, n, gy0 + r0, ny);
    __syncthreads();

    // ---- L2: u* on staged rows [2, LY-2)
    segment(dlo > 2 ? dlo : 2, dhi < G::LY - 2 ? dhi : G::LY - 2, S, s, r0, n);
    level_rhs<G::L2, PX, PLANE, PHI_MODE, false>(k, A, A + PLANE, A + 2 * PLANE, U, U + 2 * PLANE, U, B, o, r0, n,
                                                 gy0 + r0, ny, nullptr, nullptr, nullptr, 0, 0, false, false);
    __syncthreads();

    // ---- L3: mu, M of u* on staged rows [3, LY-3)
    segment(dlo > 3 ? dlo : 3, dhi < G::LY - 3 ? dhi : G::LY - 3, S, s, r0, n);
    level_mu<G::L3, PX, MOB>(k, B, B + PLANE, A, A + PLANE, A + 2 * PLANE, o, r0, n, gy0 + r0, ny);
    __syncthreads();

    // ---- L4: u^{n+1} on the output rows [4, 4+TY), stored for output columns in the domain
    segment(dlo > HALO ? dlo : HALO, dhi < HALO + TY ? dhi : HALO + TY, S, s, r0, n);
    const int gx = gx0 + 4 * qc;  // global column of the quad's first cell
    const bool store_x = (4 * qc >= HALO) && (4 * qc < HALO + TX) && gx < nx;
    const int valid_x = nx - gx;  // cells of the quad inside the domain (>= 4: all)
    const size_t g_off = (size_t)(gy0 + r0) * pitch + (gx < 0 ? 0 : gx);
    level_rhs<G::L4, PX, PLANE, PHI_MODE, true>(k, A, A + PLANE, A + 2 * PLANE, B, B + 2 * PLANE, U, nullptr, o, r0,
                                                n, gy0 + r0, ny, phi1, c1, rho1, g_off, pitch, store_x, valid_x);
}

template <int TX, int TY, int S, int PHI_MODE, int MOB>
cudaError_t launch_t(const StepConst& k, const float* f0, const float* c0, const float* r0, float* f1,
                     float* c1, float* r1, cudaStream_t s)
{
    using G = Geo<TX, TY, S>;
    auto kern = step_kernel<TX, TY, S, PHI_MODE, MOB>;
    static bool configured = false;  // the attribute is per function; setting it twice is harmless
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::BYTES);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((k.nx + TX - 1) / TX, (k.ny + TY - 1) / TY);
    cfg.blockDim = dim3(G::THREADS);
    cfg.dynamicSmemBytes = G::BYTES;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, k, f0, c0, r0, f1, c1, r1);
}

template <int TX, int TY, int S>
cudaError_t launch_tile(const StepConst& k, int phi_mode, int mob, const float* f0, const float* c0,
                        const float* r0, float* f1, float* c1, float* r1, cudaStream_t s)
{
    if (phi_mode == 0) {
        if (mob == MOB_UNIFORM) return launch_t<TX, TY, S, 0, MOB_UNIFORM>(k, f0, c0, r0, f1, c1, r1, s);
        if (mob == MOB_BULK) return launch_t<TX, TY, S, 0, MOB_BULK>(k, f0, c0, r0, f1, c1, r1, s);
        return launch_t<TX, TY, S, 0, MOB_SURF>(k, f0, c0, r0, f1, c1, r1, s);
    }
    if (mob == MOB_UNIFORM) return launch_t<TX, TY, S, 1, MOB_UNIFORM>(k, f0, c0, r0, f1, c1, r1, s);
    if (mob == MOB_BULK) return launch_t<TX, TY, S, 1, MOB_BULK>(k, f0, c0, r0, f1, c1, r1, s);
    return launch_t<TX, TY, S, 1, MOB_SURF>(k, f0, c0, r0, f1, c1, r1, s);
}

}  // namespace

int choose_tile(int nx, int ny)
{
    // Grids up to ~1M cells need the small tile to give every SM several CTAs.
    return (long long)nx * ny <= (1LL << 20) ? TILE_SMALL : TILE_LARGE;
}

#ifndef PF_SMALL_TX
#define PF_SMALL_TX 32
#define PF_SMALL_TY 16
#define PF_SMALL_S 16
#endif
#ifndef PF_LARGE_TX
#define PF_LARGE_TX 64
#define PF_LARGE_TY 32
#define PF_LARGE_S 16
#endif
#define PF_SMALL_TILE PF_SMALL_TX, PF_SMALL_TY, PF_SMALL_S
#define PF_LARGE_TILE PF_LARGE_TX, PF_LARGE_TY, PF_LARGE_S

size_t step_smem_bytes(int tile)
{
    return tile == TILE_SMALL ? Geo<PF_SMALL_TILE>::BYTES : Geo<PF_LARGE_TILE>::BYTES;
}

cudaError_t launch_step(const StepConst& k, int tile, int phi_mode, int mob, const float* f0, const float* c0,
                        const float* r0, float* f1, float* c1, float* r1, cudaStream_t s)
{
    if (tile == TILE_SMALL) return launch_tile<PF_SMALL_TILE>(k, phi_mode, mob, f0, c0, r0, f1, c1, r1, s);
    return launch_tile<PF_LARGE_TILE>(k, phi_mode, mob, f0, c0, r0, f1, c1, r1, s);
}

}  // namespace pf
