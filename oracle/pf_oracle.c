/*
 * FP64 CPU oracle of the explicit phase-field PVD time step (arXiv 2312.05410).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header or constant with the CUDA path.
 *
 * The checker is this file built without OpenMP (single thread).  Built with
 * -fopenmp (the CPU baseline over all host cores), the per-cell loops split their
 * rows over threads; every cell is computed by the same expressions either way,
 * so both builds give identical results.
 *
 * What it follows (all in "Materials and Methods", subsection "Phase-field
 * modeling of physical vapor deposition", and "Dataset"):
 *   [CH-c]   dc/dt   = div( M_c(phi,c) grad dF/dc )            composition
 *   [Mc]     M_c     = M^Bulk + M^Surf
 *   [MBulk]  M^Bulk  = 1/4 (2-phi)(1+phi)^2 ( h M_A^B + (1-h) M_B^B )
 *   [MSurf]  M^Surf  = exp(-(phi/sigma)^2) ( h M_A^S + (1-h) M_B^S )
 *   [CH-phi] dphi/dt = div( M_phi grad dF/dphi ) + S               order parameter
 *   [S]      S       = grad(phi) . (rho v)                       deposition source
 *   [rho]    drho/dt = div(D grad rho) - div(rho v) - grad(phi).(rho v)
 *   [disc]   second-order central differences for all spatial derivatives,
 *            explicit midpoint (two-stage Runge-Kutta) in time ("Dataset").
 *
 * Readings where the paper is silent or garbled (each is also listed in the
 * design notes of the repository):
 *   F (deferred to another paper): f = W_phi/4 (1-phi^2)^2 + p(phi) W_c g(c),
 *     g = c^2 (1-c)^2, p(phi) = 1/4 (2-phi)(1+phi)^2 (the same solid indicator
 *     the paper puts in M^Bulk); gradient energy kappa/2 |grad u|^2 for u = phi, c.
 *   h(c) (deferred): h = c^2 (3 - 2c), no clamping.
 *   M^Surf: the self-referencing "- M^Surf" inside the bracket is dropped.
 *   M(phi) in the phi equation: the constant M_phi.  phi_mode = 1 replaces the
 *     conserved form by Allen-Cahn relaxation -L_phi dF/dphi (same source S).
 *   v = V (cos theta, -sin theta), theta measured from the substrate; v = 0 when
 *     deposition is off.
 *   Boundaries: x periodic; bottom mirror (no flux) for every field; top mirror
 *     for phi, c and both chemical potentials, ghost value rho_top for rho.
 *     Chemical-potential ghosts are filled from the computed interior values.
 *   Face mobility: arithmetic mean of the two cells.
 *
 * Parity unpinned: the deposition-on dynamics have no closed form; they are
 * covered only through the pinned pieces (source direction and magnitude
 * against a continuum derivative, conservation of sum(c)).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    double dx, dt;
    double W_c, W_phi, kappa_c, kappa_phi;
    double MA_bulk, MB_bulk, MA_surf, MB_surf, sigma_surf;
    double M_phi, L_phi, D_rho, v_mag, v_angle_deg, rho_top;
    int phi_mode, deposition, diag_every;
} orc_params;

/* ---- pointwise functions of the free energy and mobility -------------- */

/* solid indicator p(phi) = 1/4 (2-phi)(1+phi)^2, [MBulk] */
double orc_p(double phi) { return 0.25 * (2.0 - phi) * (1.0 + phi) * (1.0 + phi); }
/* dp/dphi = 3/4 (1 - phi^2) */
double orc_dp(double phi) { return 0.75 * (1.0 - phi * phi); }
/* switching function h(c) = c^2 (3 - 2c) (reading) */
double orc_h(double c) { return c * c * (3.0 - 2.0 * c); }
/* chemical well g(c) = c^2 (1-c)^2 and its derivative (reading of F) */
double orc_g(double c) { return c * c * (1.0 - c) * (1.0 - c); }
double orc_dg(double c) { return 2.0 * c * (1.0 - c) * (1.0 - 2.0 * c); }

/* bulk free-energy density f(phi, c) (reading of F) */
double orc_f(const orc_params* P, double phi, double c)
{
    double w = 1.0 - phi * phi;
    return 0.25 * P->W_phi * w * w + orc_p(phi) * P->W_c * orc_g(c);
}

/* composition mobility M_c(phi, c) = M^Bulk + M^Surf, [Mc], [MBulk], [MSurf] */
double orc_mobility(const orc_params* P, double phi, double c)
{
    double h = orc_h(c);
    double bulk = orc_p(phi) * (h * P->MA_bulk + (1.0 - h) * P->MB_bulk);
    double s = phi / P->sigma_surf;
    double surf = exp(-s * s) * (h * P->MA_surf + (1.0 - h) * P->MB_surf);
    return bulk + surf;
}

/* ---- ghost cells ------------------------------------------------------- */

#define IDX(j, i) ((size_t)(j) * (size_t)nx + (size_t)(i))
#define PIDX(j, i) ((size_t)(j) * (size_t)(nx + 2) + (size_t)(i))

/* Copy u (ny x nx) into a padded (ny+2) x (nx+2) array with one ghost ring:
 * periodic in x, mirror at the bottom, mirror at the top unless top_value is
 * given (use_top_value != 0), in which case the top ghost row holds it. */
static void pad_field(int nx, int ny, const double* u, double* up, int use_top_value, double top_value)
{
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) up[PIDX(j + 1, i + 1)] = u[IDX(j, i)];
        up[PIDX(j + 1, 0)] = u[IDX(j, nx - 1)];
        up[PIDX(j + 1, nx + 1)] = u[IDX(j, 0)];
    }
    for (int i = 0; i < nx + 2; ++i) {
        up[PIDX(0, i)] = up[PIDX(1, i)];
        up[PIDX(ny + 1, i)] = use_top_value ? top_value : up[PIDX(ny, i)];
    }
}

/* 5-point sum of the four neighbours of padded cell (j+1, i+1) minus 4x centre. */
static double lap5(int nx, const double* up, int j, int i)
{
    const double uc = up[PIDX(j + 1, i + 1)];
    return up[PIDX(j + 1, i + 2)] + up[PIDX(j + 1, i)] + up[PIDX(j + 2, i + 1)] + up[PIDX(j, i + 1)] - 4.0 * uc;
}

/* ---- chemical potentials, [CH-c] and [CH-phi] with the reading of F ---- */

/* mu_c = dF/dc = p W_c g'(c) - kappa_c L(c);
 * mu_phi = dF/dphi = -W_phi phi (1-phi^2) + p'(phi) W_c g(c) - kappa_phi L(phi). */
int orc_chem_pot(const orc_params* P, int nx, int ny, const double* phi, const double* c,
                 double* mu_c, double* mu_phi)
{
    if (nx < 1 || ny < 1) return -1;
    const double idx2 = 1.0 / (P->dx * P->dx);
    double* pp = malloc(sizeof(double) * (size_t)(nx + 2) * (ny + 2));
    double* cp = malloc(sizeof(double) * (size_t)(nx + 2) * (ny + 2));
    if (!pp || !cp) { free(pp); free(cp); return -2; }
    pad_field(nx, ny, phi, pp, 0, 0.0);
    pad_field(nx, ny, c, cp, 0, 0.0);
#pragma omp parallel for
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            double f = phi[IDX(j, i)], cc = c[IDX(j, i)];
            double Lc = lap5(nx, cp, j, i) * idx2;
            double Lf = lap5(nx, pp, j, i) * idx2;
            mu_c[IDX(j, i)] = orc_p(f) * P->W_c * orc_dg(cc) - P->kappa_c * Lc;
            mu_phi[IDX(j, i)] = -P->W_phi * f * (1.0 - f * f) + orc_dp(f) * P->W_c * orc_g(cc) - P->kappa_phi * Lf;
        }
    free(pp); free(cp);
    return 0;
}

/* ---- right-hand side of the three equations ---------------------------- */

static void velocity(const orc_params* P, double* vx, double* vy)
{
    const double pi = 3.14159265358979323846;
    if (!P->deposition) { *vx = 0.0; *vy = 0.0; return; }
    double th = P->v_angle_deg * pi / 180.0;
    *vx = P->v_mag * cos(th);
    *vy = -P->v_mag * sin(th);
}

/* R = d(phi, c, rho)/dt at the given state, [CH-c], [CH-phi], [S], [rho]. */
int orc_rhs(const orc_params* P, int nx, int ny, const double* phi, const double* c, const double* rho,
            double* R_phi, double* R_c, double* R_rho)
{
    if (nx < 1 || ny < 1) return -1;
    const size_t n = (size_t)nx * ny, np = (size_t)(nx + 2) * (ny + 2);
    const double dx = P->dx, idx2 = 1.0 / (dx * dx);
    double vx, vy;
    velocity(P, &vx, &vy);

    double* mu_c = malloc(sizeof(double) * n);
    double* mu_f = malloc(sizeof(double) * n);
    double* Mc = malloc(sizeof(double) * n);
    double* pp = malloc(sizeof(double) * np);
    double* rp = malloc(sizeof(double) * np);
    double* mcp = malloc(sizeof(double) * np);
    double* mfp = malloc(sizeof(double) * np);
    double* Mp = malloc(sizeof(double) * np);
    if (!mu_c || !mu_f || !Mc || !pp || !rp || !mcp || !mfp || !Mp) {
        free(mu_c); free(mu_f); free(Mc); free(pp); free(rp); free(mcp); free(mfp); free(Mp);
        return -2;
    }
    orc_chem_pot(P, nx, ny, phi, c, mu_c, mu_f);
#pragma omp parallel for
    for (size_t k = 0; k < n; ++k) Mc[k] = orc_mobility(P, phi[k], c[k]);

    /* ghosts of the computed chemical potentials and mobility (mirror in y) */
    pad_field(nx, ny, mu_c, mcp, 0, 0.0);
    pad_field(nx, ny, mu_f, mfp, 0, 0.0);
    pad_field(nx, ny, Mc, Mp, 0, 0.0);
    pad_field(nx, ny, phi, pp, 0, 0.0);
    pad_field(nx, ny, rho, rp, 1, P->rho_top);

#pragma omp parallel for
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            const size_t k = IDX(j, i);
            /* conserved flux divergence of c: sum over faces of M_face (mu_nb - mu) / dx^2 */
            const double m0 = Mp[PIDX(j + 1, i + 1)], u0 = mcp[PIDX(j + 1, i + 1)];
            const int nbj[4] = {j + 1, j + 1, j + 2, j};
            const int nbi[4] = {i + 2, i, i + 1, i + 1};
            double rc = 0.0;
            for (int q = 0; q < 4; ++q) {
                double mface = 0.5 * (m0 + Mp[PIDX(nbj[q], nbi[q])]);
                rc += mface * (mcp[PIDX(nbj[q], nbi[q])] - u0);
            }
            R_c[k] = rc * idx2;

            /* deposition source S = grad(phi) . (rho v), central differences */
            const double dphix = (pp[PIDX(j + 1, i + 2)] - pp[PIDX(j + 1, i)]) / (2.0 * dx);
            const double dphiy = (pp[PIDX(j + 2, i + 1)] - pp[PIDX(j, i + 1)]) / (2.0 * dx);
            const double S = rho[k] * (vx * dphix + vy * dphiy);

            if (P->phi_mode == 0)
                R_phi[k] = P->M_phi * lap5(nx, mfp, j, i) * idx2 + S;
            else
                R_phi[k] = -P->L_phi * mu_f[k] + S;

            /* vapor: diffusion - advection - deposition sink */
            const double drx = (rp[PIDX(j + 1, i + 2)] - rp[PIDX(j + 1, i)]) / (2.0 * dx);
            const double dry = (rp[PIDX(j + 2, i + 1)] - rp[PIDX(j, i + 1)]) / (2.0 * dx);
            R_rho[k] = P->D_rho * lap5(nx, rp, j, i) * idx2 - (vx * drx + vy * dry) - S;
        }
    free(mu_c); free(mu_f); free(Mc); free(pp); free(rp); free(mcp); free(mfp); free(Mp);
    return 0;
}

/* ---- explicit midpoint time step, [disc] ------------------------------- */

/* u* = u^n + dt/2 R(u^n);  u^{n+1} = u^n + dt R(u*).  In place, nsteps times. */
int orc_step(const orc_params* P, int nx, int ny, double* phi, double* c, double* rho, long nsteps)
{
    if (nx < 1 || ny < 1 || nsteps < 0) return -1;
    const size_t n = (size_t)nx * ny;
    double* buf = malloc(sizeof(double) * n * 9);
    if (!buf) return -2;
    double *Rf = buf, *Rc = buf + n, *Rr = buf + 2 * n;
    double *fs = buf + 3 * n, *cs = buf + 4 * n, *rs = buf + 5 * n;
    double *Rf2 = buf + 6 * n, *Rc2 = buf + 7 * n, *Rr2 = buf + 8 * n;
    const double dt = P->dt;
    for (long s = 0; s < nsteps; ++s) {
        orc_rhs(P, nx, ny, phi, c, rho, Rf, Rc, Rr);
#pragma omp parallel for
        for (size_t k = 0; k < n; ++k) {
            fs[k] = phi[k] + 0.5 * dt * Rf[k];
            cs[k] = c[k] + 0.5 * dt * Rc[k];
            rs[k] = rho[k] + 0.5 * dt * Rr[k];
        }
        orc_rhs(P, nx, ny, fs, cs, rs, Rf2, Rc2, Rr2);
#pragma omp parallel for
        for (size_t k = 0; k < n; ++k) {
            phi[k] += dt * Rf2[k];
            c[k] += dt * Rc2[k];
            rho[k] += dt * Rr2[k];
        }
    }
    free(buf);
    return 0;
}

/* ---- diagnostics -------------------------------------------------------- */

/* Discrete free energy F_h = dx^2 sum f + kappa_phi/2 sum_faces (dphi)^2 + kappa_c/2 sum_faces (dc)^2.
 * Faces: every x face (periodic) and every interior y face; the mirror boundary faces add 0. */
double orc_free_energy(const orc_params* P, int nx, int ny, const double* phi, const double* c)
{
    double bulk = 0.0, gphi = 0.0, gc = 0.0;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            const size_t k = IDX(j, i), ke = IDX(j, (i + 1) % nx);
            bulk += orc_f(P, phi[k], c[k]);
            gphi += (phi[ke] - phi[k]) * (phi[ke] - phi[k]);
            gc += (c[ke] - c[k]) * (c[ke] - c[k]);
            if (j + 1 < ny) {
                const size_t kn = IDX(j + 1, i);
                gphi += (phi[kn] - phi[k]) * (phi[kn] - phi[k]);
                gc += (c[kn] - c[k]) * (c[kn] - c[k]);
            }
        }
    return P->dx * P->dx * bulk + 0.5 * P->kappa_phi * gphi + 0.5 * P->kappa_c * gc;
}

/* out = { dx^2 sum c, dx^2 sum phi, dx^2 sum rho, F_h } */
void orc_diag(const orc_params* P, int nx, int ny, const double* phi, const double* c, const double* rho,
              double* out)
{
    double sc = 0.0, sf = 0.0, sr = 0.0;
    for (size_t k = 0; k < (size_t)nx * ny; ++k) { sc += c[k]; sf += phi[k]; sr += rho[k]; }
    const double a = P->dx * P->dx;
    out[0] = a * sc;
    out[1] = a * sf;
    out[2] = a * sr;
    out[3] = orc_free_energy(P, nx, ny, phi, c);
}

/* ---- explicit stability limit ------------------------------------------ */

/* Stability function of the explicit midpoint method, |1 + z + z^2/2|. */
static double rk2_gain(double zr, double zi)
{
    double re = 1.0 + zr + 0.5 * (zr * zr - zi * zi);
    double im = zi + zr * zi;
    return sqrt(re * re + im * im);
}

/* Largest dt with |1 + z + z^2/2| <= 1 for every vapor mode on a fixed lattice
 * of wave numbers (theta_x in [-pi, pi], theta_y in [0, pi], 257 points per pi):
 * z = dt ( -D lam(theta) - i (vx sin theta_x + vy sin theta_y) / dx ). */
static int rho_stable(const orc_params* P, double dt)
{
    const double pi = 3.14159265358979323846;
    double vx, vy;
    velocity(P, &vx, &vy);
    const double dx = P->dx;
    for (int a = -256; a <= 256; ++a) {
        const double tx = pi * a / 256.0;
        for (int b = 0; b <= 256; ++b) {
            const double ty = pi * b / 256.0;
            const double sx = sin(0.5 * tx), sy = sin(0.5 * ty);
            const double lam = 4.0 / (dx * dx) * (sx * sx + sy * sy);
            const double zr = -dt * P->D_rho * lam;
            const double zi = -dt * (vx * sin(tx) + vy * sin(ty)) / dx;
            if (rk2_gain(zr, zi) > 1.0 + 1e-13) return 0;
        }
    }
    return 1;
}

/* out = { dt_lim, dt_c, dt_phi, dt_rho }.
 * lam_max = 8/dx^2 bounds the eigenvalues of -L; the real stability interval of the
 * midpoint method is [-2, 0].  Composition: |f_cc| <= 2 W_c (g'' in [-1, 2] on [0,1]),
 * mobility bounded by max bulk + max surface coefficient.  Order parameter: f_phiphi
 * <= 2 W_phi + 3/32 W_c (p'' = -3/2 phi, g <= 1/16). */
int orc_dt_limit(const orc_params* P, double* out)
{
    const double dx = P->dx, lam = 8.0 / (dx * dx);
    const double Mmax = fmax(P->MA_bulk, P->MB_bulk) + fmax(P->MA_surf, P->MB_surf);
    double dt_c = (Mmax > 0.0) ? 2.0 / (Mmax * (P->kappa_c * lam * lam + 2.0 * P->W_c * lam)) : INFINITY;
    const double fpp = 2.0 * P->W_phi + 3.0 / 32.0 * P->W_c;
    double dt_f;
    if (P->phi_mode == 0)
        dt_f = (P->M_phi > 0.0) ? 2.0 / (P->M_phi * (P->kappa_phi * lam * lam + fpp * lam)) : INFINITY;
    else
        dt_f = (P->L_phi > 0.0) ? 2.0 / (P->L_phi * (P->kappa_phi * lam + fpp)) : INFINITY;

    /* bisection for the vapor equation between 0 and the pure-diffusion bound */
    double hi = (P->D_rho > 0.0) ? 2.0 / (P->D_rho * lam) : 1.0;
    orc_params Q = *P;
    double lo = 0.0;
    if (rho_stable(&Q, hi)) {
        lo = hi;
    } else {
        for (int it = 0; it < 80; ++it) {
            double mid = 0.5 * (lo + hi);
            if (rho_stable(&Q, mid)) lo = mid; else hi = mid;
        }
    }
    double dt_r = lo;
    out[0] = fmin(dt_c, fmin(dt_f, dt_r));
    out[1] = dt_c;
    out[2] = dt_f;
    out[3] = dt_r;
    return 0;
}
