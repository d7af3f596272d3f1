// Host-side folding of pf_params into the kernels' FP32 constants, shared by
// the single-run (pf_api.cu), ensemble (pf_ens.cu) and adjoint (pf_adjoint.cu) layers.
#include <cmath>

#include <cudaTypedefs.h>

#include "pf_internal.h"

namespace pf {

// v = v_mag (cos a, -sin a), a measured from the substrate; zero without deposition.
void velocity_of(const pf_params& p, double* vx, double* vy)
{
    if (!p.deposition) {
        *vx = *vy = 0.0;
        return;
    }
    const double a = p.v_angle_deg * (M_PI / 180.0);
    *vx = p.v_mag * std::cos(a);
    *vy = -p.v_mag * std::sin(a);
}

StepConst step_const_of(const pf_params& p, int nx, int ny, int pitch)
{
    StepConst k{};
    const double dx2 = p.dx * p.dx;
    double vx, vy;
    velocity_of(p, &vx, &vy);
    k.nx = nx;
    k.ny = ny;
    k.pitch = pitch;
    k.Wc = float(p.W_c);
    k.Wf = float(p.W_phi);
    k.kc = float(p.kappa_c / dx2);
    k.kf = float(p.kappa_phi / dx2);
    k.MBb = float(p.MB_bulk);
    k.dMb = float(p.MA_bulk - p.MB_bulk);
    k.MBs = float(p.MB_surf);
    k.dMs = float(p.MA_surf - p.MB_surf);
    k.nisig2 = (p.sigma_surf > 0.0) ? float(-1.0 / (M_LN2 * p.sigma_surf * p.sigma_surf)) : 0.f;
    k.cR = float(0.5 / dx2);
    k.cF = (p.phi_mode == 0) ? float(p.M_phi / dx2) : float(-p.L_phi);
    k.ax = float(vx / (2.0 * p.dx));
    k.ay = float(vy / (2.0 * p.dx));
    k.cD = float(p.D_rho / dx2);
    k.rho_top = float(p.rho_top);
    k.dt = float(p.dt);
    k.wait_cap = 1 << 22;  // a few milliseconds of polling; a TMA box lands in about a microsecond
    return k;
}

DiagConst diag_const_of(const pf_params& p, int nx, int ny, int pitch)
{
    DiagConst d{};
    d.nx = nx;
    d.ny = ny;
    d.pitch = pitch;
    d.Wc = float(p.W_c);
    d.Wf = float(p.W_phi);
    d.area = p.dx * p.dx;
    d.hkf = 0.5 * p.kappa_phi;
    d.hkc = 0.5 * p.kappa_c;
    return d;
}

int mob_kind_of(const pf_params& p)
{
    if (p.MA_surf != 0.0 || p.MB_surf != 0.0) return MOB_SURF;
    return (p.MA_bulk == p.MB_bulk) ? MOB_UNIFORM : MOB_BULK;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link to libcuda).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return (PFN_cuTensorMapEncodeTiled_v12000) nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    }();
    return fn;
}

// Tiled FP32 maps of the three planes of one state: dims (nx, ny), row stride pitch*4 bytes,
// box 64 x box_rows -- the staged window of one CTA.  An interior tile exists only if the tile at
// (interior_x, interior_y) keeps its whole staged window inside the grid; otherwise the TMA path
// would never be taken and no maps are made.
bool make_maps_box(const float* phi, const float* c, const float* rho, int nx, int ny, int pitch, int box_rows,
                   int interior_x, int interior_y, StepMaps* out)
{
    if (nx < interior_x + 64 || ny < interior_y + box_rows) return false;
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t dims[2] = {cuuint64_t(nx), cuuint64_t(ny)};
    const cuuint64_t strides[1] = {cuuint64_t(pitch) * sizeof(float)};
    const cuuint32_t box[2] = {64u, cuuint32_t(box_rows)};
    const cuuint32_t elem[2] = {1u, 1u};
    const float* f[3] = {phi, c, rho};
    CUtensorMap* m[3] = {&out->phi, &out->c, &out->rho};
    for (int q = 0; q < 3; ++q)
        if (enc(m[q], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(f[q]), dims, strides, box, elem,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
    return true;
}

// Maps of the one-step kernel's window (4-cell halo): the second tile column (x0 = 56) and row
// (y0 = TY) are the first whose windows may lie inside the grid.
bool make_step_maps(const float* phi, const float* c, const float* rho, int nx, int ny, int pitch, int tile,
                    StepMaps* out)
{
    const int TY = tile_height(tile), LY = TY + 8;
    return make_maps_box(phi, c, rho, nx, ny, pitch, LY, 56 - 4, TY - 4, out);
}

}  // namespace pf
