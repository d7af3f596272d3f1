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
// Threads work on x-adjacent cell pairs with packed FP32x2 arithmetic
// (fma/add/mul .f32x2).  Boundary rules live in the row-neighbour offsets:
// the bottom and top rows see themselves as their outer neighbour (mirror);
// rho's outer neighbour above the top row is the reservoir value.
#include "pf_internal.h"

namespace pf {
namespace {

typedef float2 f2;
__device__ __forceinline__ f2 F2(float a) { return make_float2(a, a); }
__device__ __forceinline__ f2 add2(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 mul2(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ f2 sub2(f2 a, f2 b) { return __ffma2_rn(b, F2(-1.f), a); }
__device__ __forceinline__ f2 neg2(f2 a) { return make_float2(-a.x, -a.y); }

constexpr int HALO = 4;
constexpr int PAD = 4;  // columns of padding on each side of a staged row (keeps 16-B alignment)

template <int TX, int TY>
struct Geo {
    static constexpr int LX = TX + 2 * HALO;  // staged columns
    static constexpr int LY = TY + 2 * HALO;  // staged rows
    static constexpr int PX = LX + 2 * PAD;   // row pitch in shared memory (floats)
    static constexpr int PLANE = LY * PX;
    static constexpr int NPLANES = 9;         // u^n (3), mu/M (3), u* (3)
    static constexpr size_t BYTES = size_t(NPLANES) * PLANE * sizeof(float);
};

// Pair of cells (x, x+1) of one staged plane, with its four neighbour pairs.
struct Nb {
    f2 C, N, S;
    float W, E;  // scalar west neighbour of x, east neighbour of x+1
};

__device__ __forceinline__ Nb load_nb(const float* p, int up, int dn)
{
    Nb r;
    r.C = *reinterpret_cast<const f2*>(p);
    r.N = *reinterpret_cast<const f2*>(p + up);
    r.S = *reinterpret_cast<const f2*>(p + dn);
    r.W = p[-1];
    r.E = p[2];
    return r;
}

// Sum of the four neighbours of each cell of the pair.
__device__ __forceinline__ f2 nb_sum(const Nb& a)
{
    f2 h = make_float2(a.W + a.C.y, a.C.x + a.E);
    return add2(h, add2(a.N, a.S));
}

// p(phi) = 1/4 (2-phi)(1+phi)^2 = 1/2 + 3/4 phi - 1/4 phi^3
__device__ __forceinline__ f2 p_of(f2 f, f2 f2sq)
{
    return fma2(fma2(F2(-0.25f), f2sq, F2(0.75f)), f, F2(0.5f));
}

// L1 / L3: chemical potentials and mobility of one pair from the staged (phi, c).
template <int MOB>
__device__ __forceinline__ void level_mu(const StepConst& k, const float* sphi, const float* sc,
                                         int up, int dn, float* o_muc, float* o_muf, float* o_M)
{
    const Nb F = load_nb(sphi, up, dn);
    const Nb Cc = load_nb(sc, up, dn);
    const f2 f = F.C, c = Cc.C;
    const f2 ff = mul2(f, f);
    const f2 p = p_of(f, ff);
    const f2 q = fma2(neg2(c), c, c);                               // c (1 - c)
    const f2 g = mul2(q, q);                                   // g(c) = c^2 (1-c)^2
    const f2 Wdg = mul2(q, fma2(F2(-4.f * k.Wc), c, F2(2.f * k.Wc)));  // W_c g'(c)
    // mu_c = p W_c g' - kappa_c L(c)
    f2 muc = fma2(F2(4.f * k.kc), c, mul2(p, Wdg));
    muc = fma2(F2(-k.kc), nb_sum(Cc), muc);
    // mu_phi = -W_phi phi (1 - phi^2) + p'(phi) W_c g - kappa_phi L(phi),  p' = 3/4 (1 - phi^2)
    f2 muf = mul2(fma2(F2(k.Wf), ff, F2(-k.Wf)), f);
    muf = fma2(fma2(F2(-0.75f * k.Wc), ff, F2(0.75f * k.Wc)), g, muf);
    muf = fma2(F2(4.f * k.kf), f, muf);
    muf = fma2(F2(-k.kf), nb_sum(F), muf);
    // M_c = p (MB + h dM) [+ exp(-(phi/sigma)^2)(MBs + h dMs)],  h = c^2 (3 - 2c)
    f2 M;
    if (MOB == MOB_UNIFORM) {
        M = mul2(p, F2(k.MBb));
    } else {
        const f2 h = mul2(mul2(c, c), fma2(F2(-2.f), c, F2(3.f)));
        M = mul2(p, fma2(h, F2(k.dMb), F2(k.MBb)));
        if (MOB == MOB_SURF) {
            const f2 t = mul2(ff, F2(k.nisig2));
            const f2 e = make_float2(exp2f(t.x), exp2f(t.y));
            M = fma2(e, fma2(h, F2(k.dMs), F2(k.MBs)), M);
        }
    }
    *reinterpret_cast<f2*>(o_muc) = muc;
    *reinterpret_cast<f2*>(o_muf) = muf;
    *reinterpret_cast<f2*>(o_M) = M;
}

// L2 / L4 right-hand side of one pair: R_phi, R_c, R_rho (not yet scaled by dt).
template <int PHI_MODE>
__device__ __forceinline__ void level_rhs(const StepConst& k, const float* smuc, const float* smuf,
                                          const float* sM, const float* sphi, const float* srho,
                                          int up, int dn, bool top, f2& Rf, f2& Rc, f2& Rr)
{
    // conserved composition flux: sum_faces (M + M_nb)(mu_nb - mu) / (2 dx^2)
    const Nb m = load_nb(smuc, up, dn);
    const Nb M = load_nb(sM, up, dn);
    const float Fa = (M.W + M.C.x) * (m.C.x - m.W);      // face (x-1 | x)
    const float Fb = (M.C.x + M.C.y) * (m.C.y - m.C.x);  // face (x | x+1)
    const float Fc = (M.C.y + M.E) * (m.E - m.C.y);      // face (x+1 | x+2)
    f2 rc = make_float2(Fb - Fa, Fc - Fb);
    rc = fma2(add2(M.C, M.N), sub2(m.N, m.C), rc);
    rc = fma2(add2(M.C, M.S), sub2(m.S, m.C), rc);
    Rc = mul2(rc, F2(k.cR));

    // deposition source S = grad(phi) . (rho v), central differences
    const Nb F = load_nb(sphi, up, dn);
    const Nb R = load_nb(srho, up, dn);
    const f2 gx = make_float2(F.C.y - F.W, F.E - F.C.x);
    const f2 gy = sub2(F.N, F.S);
    const f2 Src = mul2(R.C, fma2(F2(k.ax), gx, mul2(F2(k.ay), gy)));

    if (PHI_MODE == 0) {
        const Nb u = load_nb(smuf, up, dn);
        Rf = fma2(F2(k.cF), fma2(F2(-4.f), u.C, nb_sum(u)), Src);
    } else {
        const f2 u = *reinterpret_cast<const f2*>(smuf);
        Rf = fma2(F2(k.cF), u, Src);
    }

    // vapor: D L(rho) - div(rho v) - S, reservoir value above the top row
    const f2 rN = top ? F2(k.rho_top) : R.N;
    const f2 hs = make_float2(R.W + R.C.y, R.C.x + R.E);
    const f2 lap = fma2(F2(-4.f), R.C, add2(hs, add2(rN, R.S)));
    const f2 rx = make_float2(R.C.y - R.W, R.E - R.C.x);
    const f2 adv = fma2(F2(k.ax), rx, mul2(F2(k.ay), sub2(rN, R.S)));
    Rr = sub2(fma2(F2(k.cD), lap, neg2(adv)), Src);
}

template <int TX, int TY, int THREADS, int PHI_MODE, int MOB>
__global__ void __launch_bounds__(THREADS)
step_kernel(const StepConst k, const float* __restrict__ phi0, const float* __restrict__ c0,
            const float* __restrict__ rho0, float* __restrict__ phi1, float* __restrict__ c1,
            float* __restrict__ rho1)
{
    using G = Geo<TX, TY>;
    extern __shared__ __align__(16) float sm[];
    float* const U = sm;                  // u^n: phi, c, rho
    float* const A = sm + 3 * G::PLANE;   // mu_c, mu_phi, M
    float* const B = sm + 6 * G::PLANE;   // u*: phi, c, rho

    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int gx0 = x0 - HALO, gy0 = y0 - HALO;
    const int nx = k.nx, ny = k.ny, pitch = k.pitch;

    // ---- stage u^n (rows outside the domain are zero and never read by domain rows)
    // Wait for the previous step's grid (programmatic dependent launch) before reading.
    asm volatile("griddepcontrol.wait;" ::: "memory");
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
        // x0 and nx are multiples of 4, so every aligned group of 4 staged columns
        // is either wholly inside [0, nx) or wholly wrapped
        constexpr int Q = G::LX / 4;
        for (int idx = tid; idx < 3 * G::LY * Q; idx += THREADS) {
            const int fld = idx / (G::LY * Q);
            const int rem = idx - fld * (G::LY * Q);
            const int ly = rem / Q, q = rem - ly * Q;
            const int gy = gy0 + ly;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (gy >= 0 && gy < ny)
                v = __ldg(reinterpret_cast<const float4*>(field(fld) + (size_t)gy * pitch + wrap(gx0 + 4 * q)));
            *reinterpret_cast<float4*>(U + fld * G::PLANE + ly * G::PX + PAD + 4 * q) = v;
        }
    } else {
        for (int idx = tid; idx < 3 * G::LY * G::LX; idx += THREADS) {
            const int fld = idx / (G::LY * G::LX);
            const int rem = idx - fld * (G::LY * G::LX);
            const int ly = rem / G::LX, lx = rem - ly * G::LX;
            const int gy = gy0 + ly;
            float v = 0.f;
            if (gy >= 0 && gy < ny) v = __ldg(field(fld) + (size_t)gy * pitch + wrap(gx0 + lx));
            U[fld * G::PLANE + ly * G::PX + PAD + lx] = v;
        }
    }
    // Let the next step's grid begin launching; it waits for this grid to finish.
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    __syncthreads();

    // Row-neighbour offsets with the boundary rules folded in.
    auto offs = [&](int ly, int& up, int& dn, bool& top) {
        const int gy = gy0 + ly;
        top = (gy == ny - 1);
        up = (gy >= ny - 1) ? 0 : G::PX;
        dn = (gy <= 0) ? 0 : -G::PX;
    };

    // ---- L1: mu, M of u^n over rows [1, LY-1), all staged columns
    {
        constexpr int NP = G::LX / 2, NR = G::LY - 2;
        for (int idx = tid; idx < NP * NR; idx += THREADS) {
            const int r = idx / NP, pc = idx - r * NP;
            const int ly = 1 + r, o = ly * G::PX + PAD + 2 * pc;
            int up, dn; bool top;
            offs(ly, up, dn, top);
            level_mu<MOB>(k, U + o, U + G::PLANE + o, up, dn, A + o, A + G::PLANE + o, A + 2 * G::PLANE + o);
        }
    }
    __syncthreads();

    // ---- L2: u* over rows [2, LY-2), columns [2, LX-2)
    {
        constexpr int NP = (G::LX - 4) / 2, NR = G::LY - 4;
        const f2 hdt = F2(0.5f * k.dt);
        for (int idx = tid; idx < NP * NR; idx += THREADS) {
            const int r = idx / NP, pc = idx - r * NP;
            const int ly = 2 + r, o = ly * G::PX + PAD + 2 + 2 * pc;
            int up, dn; bool top;
            offs(ly, up, dn, top);
            f2 Rf, Rc, Rr;
            level_rhs<PHI_MODE>(k, A + o, A + G::PLANE + o, A + 2 * G::PLANE + o, U + o, U + 2 * G::PLANE + o,
                                up, dn, top, Rf, Rc, Rr);
            *reinterpret_cast<f2*>(B + o) = fma2(hdt, Rf, *reinterpret_cast<const f2*>(U + o));
            *reinterpret_cast<f2*>(B + G::PLANE + o) =
                fma2(hdt, Rc, *reinterpret_cast<const f2*>(U + G::PLANE + o));
            *reinterpret_cast<f2*>(B + 2 * G::PLANE + o) =
                fma2(hdt, Rr, *reinterpret_cast<const f2*>(U + 2 * G::PLANE + o));
        }
    }
    __syncthreads();

    // ---- L3: mu, M of u* over rows [3, LY-3), columns [2, LX-2)
    {
        constexpr int NP = (G::LX - 4) / 2, NR = G::LY - 6;
        for (int idx = tid; idx < NP * NR; idx += THREADS) {
            const int r = idx / NP, pc = idx - r * NP;
            const int ly = 3 + r, o = ly * G::PX + PAD + 2 + 2 * pc;
            int up, dn; bool top;
            offs(ly, up, dn, top);
            level_mu<MOB>(k, B + o, B + G::PLANE + o, up, dn, A + o, A + G::PLANE + o, A + 2 * G::PLANE + o);
        }
    }
    __syncthreads();

    // ---- L4: u^{n+1} over the TX x TY output block
    {
        constexpr int NP = TX / 2;
        const f2 dt = F2(k.dt);
        for (int idx = tid; idx < NP * TY; idx += THREADS) {
            const int r = idx / NP, pc = idx - r * NP;
            const int ly = HALO + r, o = ly * G::PX + PAD + HALO + 2 * pc;
            const int gy = y0 + r, gx = x0 + 2 * pc;
            if (gy >= ny || gx >= nx) continue;
            int up, dn; bool top;
            offs(ly, up, dn, top);
            f2 Rf, Rc, Rr;
            level_rhs<PHI_MODE>(k, A + o, A + G::PLANE + o, A + 2 * G::PLANE + o, B + o, B + 2 * G::PLANE + o,
                                up, dn, top, Rf, Rc, Rr);
            const f2 out[3] = {fma2(dt, Rf, *reinterpret_cast<const f2*>(U + o)),
                               fma2(dt, Rc, *reinterpret_cast<const f2*>(U + G::PLANE + o)),
                               fma2(dt, Rr, *reinterpret_cast<const f2*>(U + 2 * G::PLANE + o))};
            const size_t g = (size_t)gy * pitch + gx;
            if (gx + 1 < nx) {
                *reinterpret_cast<f2*>(phi1 + g) = out[0];
                *reinterpret_cast<f2*>(c1 + g) = out[1];
                *reinterpret_cast<f2*>(rho1 + g) = out[2];
            } else {
                phi1[g] = out[0].x;
                c1[g] = out[1].x;
                rho1[g] = out[2].x;
            }
        }
    }
}

template <int TX, int TY, int THREADS, int PHI_MODE, int MOB>
cudaError_t launch_t(const StepConst& k, const float* f0, const float* c0, const float* r0, float* f1,
                     float* c1, float* r1, cudaStream_t s)
{
    using G = Geo<TX, TY>;
    auto kern = step_kernel<TX, TY, THREADS, PHI_MODE, MOB>;
    static bool configured = false;  // the attribute is per function; setting it twice is harmless
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::BYTES);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((k.nx + TX - 1) / TX, (k.ny + TY - 1) / TY);
    cfg.blockDim = dim3(THREADS);
    cfg.dynamicSmemBytes = G::BYTES;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, k, f0, c0, r0, f1, c1, r1);
}

template <int TX, int TY, int THREADS>
cudaError_t launch_tile(const StepConst& k, int phi_mode, int mob, const float* f0, const float* c0,
                        const float* r0, float* f1, float* c1, float* r1, cudaStream_t s)
{
    if (phi_mode == 0) {
        if (mob == MOB_UNIFORM) return launch_t<TX, TY, THREADS, 0, MOB_UNIFORM>(k, f0, c0, r0, f1, c1, r1, s);
        if (mob == MOB_BULK) return launch_t<TX, TY, THREADS, 0, MOB_BULK>(k, f0, c0, r0, f1, c1, r1, s);
        return launch_t<TX, TY, THREADS, 0, MOB_SURF>(k, f0, c0, r0, f1, c1, r1, s);
    }
    if (mob == MOB_UNIFORM) return launch_t<TX, TY, THREADS, 1, MOB_UNIFORM>(k, f0, c0, r0, f1, c1, r1, s);
    if (mob == MOB_BULK) return launch_t<TX, TY, THREADS, 1, MOB_BULK>(k, f0, c0, r0, f1, c1, r1, s);
    return launch_t<TX, TY, THREADS, 1, MOB_SURF>(k, f0, c0, r0, f1, c1, r1, s);
}

}  // namespace

int choose_tile(int nx, int ny)
{
    // Grids up to ~1M cells need the small tile to give every SM several CTAs.
    return (long long)nx * ny <= (1LL << 20) ? TILE_SMALL : TILE_LARGE;
}

size_t step_smem_bytes(int tile)
{
    return tile == TILE_SMALL ? Geo<32, 16>::BYTES : Geo<64, 32>::BYTES;
}

cudaError_t launch_step(const StepConst& k, int tile, int phi_mode, int mob, const float* f0, const float* c0,
                        const float* r0, float* f1, float* c1, float* r1, cudaStream_t s)
{
    if (tile == TILE_SMALL) return launch_tile<32, 16, 256>(k, phi_mode, mob, f0, c0, r0, f1, c1, r1, s);
    return launch_tile<64, 32, 256>(k, phi_mode, mob, f0, c0, r0, f1, c1, r1, s);
}

}  // namespace pf
