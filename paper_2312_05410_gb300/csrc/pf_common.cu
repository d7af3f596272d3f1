// Host-side folding of pf_params into the kernels' FP32 constants, shared by
// the single-run (pf_api.cu), ensemble (pf_ens.cu) and adjoint (pf_adjoint.cu) layers.
#include <cmath>

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

}  // namespace pf
