// The hybrid DNS / U-Net solver (declarations in include/pf.h).
//
// The paper's hybrid solver ("Hybrid" in Results; "U-Net with temporal
// conditioning", Methods) alternates stretches of direct numerical simulation
// with leaps of the neural operator over the time the DNS would have taken.
// Here a batch of equal-size runs advances in lockstep: `dns_lead` DNS steps
// first (the paper runs its solver alone for the first steps), then cycles of
//   1. DNS stretch: `dns_stretch` explicit steps of every run (one fused ensemble
//      launch per step, graph replays), with the state pushed as a look-back
//      frame of the surrogate `2 frame_every` and `frame_every` steps before its end;
//   2. backup of every run's state, then one U-Net jump of `jump_steps` steps
//      (tau = jump_steps / dt_ref_steps) on the tensor cores;
//   3. plausibility gate: if any run's prediction is non-finite or leaves the
//      given ranges, every run is restored from the backup and the jumped
//      stretch is run by DNS instead (the fallback);
// until fewer than one whole cycle of steps is left, which the DNS finishes.
#include <cstdarg>
#include <cstdio>
#include <string>
#include <vector>

#include "pf.h"
#include "pf_internal.h"

namespace {

thread_local std::string g_hybrid_error;

int hfail(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_hybrid_error = buf;
    return code;
}

struct Batch {
    int n = 0, nx = 0, ny = 0, pitch = 0;
    std::vector<float*> phi, c, rho;
};

// The runs of the ensemble, which must all have the U-Net's grid and one row pitch.
int batch_of(const pf_ens* e, const pf_unet* u, Batch& b)
{
    int un, ux, uy;
    pf::unet_shape(u, &un, &ux, &uy);
    b.n = pf::ens_runs(e);
    if (b.n != un) return hfail(PF_ERR_ARG, "ensemble of %d runs, U-Net batch of %d", b.n, un);
    b.phi.resize(b.n);
    b.c.resize(b.n);
    b.rho.resize(b.n);
    for (int r = 0; r < b.n; ++r) {
        int nx, ny, pitch;
        pf::ens_run_fields(e, r, &b.phi[r], &b.c[r], &b.rho[r], &nx, &ny, &pitch);
        if (nx != ux || ny != uy) return hfail(PF_ERR_ARG, "run %d is %d x %d, the U-Net's grid %d x %d", r, nx, ny, ux, uy);
        if (r == 0) b.pitch = pitch;
        if (pitch != b.pitch) return hfail(PF_ERR_LAYOUT, "runs with different row pitches");
    }
    b.nx = ux;
    b.ny = uy;
    return PF_OK;
}

int ens_steps(pf_ens* e, long n)
{
    const int rc = pf_ens_step(e, n);
    if (rc) return hfail(rc, "DNS stretch: %s", pf_ens_last_error());
    return PF_OK;
}

// Copy every run's state to (dir = 0) or from (dir = 1) the backup.
int copy_state(const Batch& b, float* backup, int dir, cudaStream_t s)
{
    const size_t rowb = size_t(b.pitch) * sizeof(float), plane = size_t(b.ny) * b.pitch;
    for (int r = 0; r < b.n; ++r) {
        float* f[3] = {b.phi[r], b.c[r], b.rho[r]};
        for (int q = 0; q < 3; ++q) {
            float* bk = backup + (size_t(r) * 3 + q) * plane;
            cudaError_t e = dir == 0 ? cudaMemcpy2DAsync(bk, rowb, f[q], rowb, size_t(b.nx) * sizeof(float), b.ny,
                                                         cudaMemcpyDeviceToDevice, s)
                                     : cudaMemcpy2DAsync(f[q], rowb, bk, rowb, size_t(b.nx) * sizeof(float), b.ny,
                                                         cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) return hfail(PF_ERR_CUDA, "state backup: %s", cudaGetErrorString(e));
        }
    }
    return PF_OK;
}

}  // namespace

extern "C" {

size_t pf_hybrid_workspace_size(const pf_ens* e)
{
    if (!e) return 0;
    size_t total = 0;
    for (int r = 0; r < pf::ens_runs(e); ++r) {
        float *a, *b, *c;
        int nx, ny, pitch;
        pf::ens_run_fields(e, r, &a, &b, &c, &nx, &ny, &pitch);
        total += 3 * size_t(ny) * pitch * sizeof(float);
    }
    return total;
}

int pf_hybrid_run(pf_ens* e, pf_unet* u, const pf_hybrid_params* hp, long total_steps, void* work, size_t work_bytes,
                  pf_hybrid_stats* stats)
{
    pf::TraceRange trace("pf_hybrid_run");
    if (!e || !u || !hp || !stats) return hfail(PF_ERR_ARG, "null pointer");
    if (total_steps < 0) return hfail(PF_ERR_ARG, "negative step count");
    if (hp->dns_stretch < 1 || hp->jump_steps < 1 || hp->frame_every < 1 || !(hp->dt_ref_steps > 0.0))
        return hfail(PF_ERR_ARG, "stretch, jump, frame spacing and dt_ref must be positive");
    if (hp->dns_lead < 0) return hfail(PF_ERR_ARG, "negative DNS lead-in");
    if (hp->dns_stretch < 2 * hp->frame_every)
        return hfail(PF_ERR_ARG, "the stretch (%ld) must hold the two look-back frames %ld steps apart", hp->dns_stretch,
                     hp->frame_every);
    if (pf::ens_stream(e) != pf::unet_stream(u)) return hfail(PF_ERR_ARG, "the ensemble and the U-Net must share a stream");
    Batch b;
    int rc = batch_of(e, u, b);
    if (rc) return rc;
    if (!work || reinterpret_cast<uintptr_t>(work) % 256) return hfail(PF_ERR_LAYOUT, "workspace must be 256-byte aligned");
    if (work_bytes < pf_hybrid_workspace_size(e))
        return hfail(PF_ERR_LAYOUT, "workspace of %zu bytes, %zu needed", work_bytes, pf_hybrid_workspace_size(e));
    cudaStream_t s = pf::ens_stream(e);
    float* backup = static_cast<float*>(work);
    const double tau = double(hp->jump_steps) / hp->dt_ref_steps;
    std::vector<int> ok(b.n);

    stats->jumps = 0;
    stats->fallbacks = 0;
    stats->dns_steps = 0;
    pf_unet_reset_frames(u);
    long t = hp->dns_lead < total_steps ? hp->dns_lead : total_steps;
    if (t > 0) {
        if ((rc = ens_steps(e, t))) return rc;
        stats->dns_steps += t;
    }
    const long cycle = hp->dns_stretch + hp->jump_steps;
    while (t + cycle <= total_steps) {
        // 1. the DNS stretch, with the two look-back frames pushed on the way
        const long lead = hp->dns_stretch - 2 * hp->frame_every;
        if ((rc = ens_steps(e, lead))) return rc;
        for (int f = 0; f < 2; ++f) {
            rc = pf_unet_frame(u, b.n, b.phi.data(), b.c.data(), b.rho.data(), b.pitch);
            if (rc) return hfail(rc, "look-back frame: %s", pf_unet_last_error());
            if ((rc = ens_steps(e, hp->frame_every))) return rc;
        }
        stats->dns_steps += hp->dns_stretch;
        // 2. backup and jump
        if ((rc = copy_state(b, backup, 0, s))) return rc;
        rc = pf_unet_jump(u, b.n, b.phi.data(), b.c.data(), b.rho.data(), b.pitch, tau);
        if (rc) return hfail(rc, "jump: %s", pf_unet_last_error());
        // 3. plausibility gate (synchronises), DNS fallback
        rc = pf_unet_check(u, hp->phi_lo, hp->phi_hi, hp->c_lo, hp->c_hi, hp->rho_lo, hp->rho_hi, ok.data());
        if (rc) return hfail(rc, "plausibility check: %s", pf_unet_last_error());
        bool all = true;
        for (int r = 0; r < b.n; ++r) all &= ok[r] != 0;
        if (all) {
            ++stats->jumps;
        } else {
            if ((rc = copy_state(b, backup, 1, s))) return rc;
            if ((rc = ens_steps(e, hp->jump_steps))) return rc;
            stats->dns_steps += hp->jump_steps;
            ++stats->fallbacks;
        }
        t += cycle;
    }
    if (t < total_steps) {
        if ((rc = ens_steps(e, total_steps - t))) return rc;
        stats->dns_steps += total_steps - t;
    }
    rc = pf_unet_sync(u);  // reports a tensor-core pipeline wait that ran out
    if (rc) return hfail(rc, "U-Net: %s", pf_unet_last_error());
    return PF_OK;
}

const char* pf_hybrid_last_error(void) { return g_hybrid_error.c_str(); }

}  // extern "C"
