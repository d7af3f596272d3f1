// C-ABI layer of the GB300 phase-field PVD step (declarations and contracts in
// include/pf.h).  Host code only: parameter validation, the explicit stability
// limit, workspace layout, the step loop with CUDA-graph replay, diagnostics.
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>

#include "pf.h"
#include "pf_internal.h"

namespace pf {

namespace {
thread_local std::string g_last_error;
}

int fail(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char* what)
{
    return fail(PF_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

constexpr int MAX_SIDE = 1 << 20;

int check_sizes(int nx, int ny, int pitch)
{
    if (nx < 1 || ny < 1) return fail(PF_ERR_ARG, "empty grid (nx=%d, ny=%d)", nx, ny);
    if (nx > MAX_SIDE || ny > MAX_SIDE)
        return fail(PF_ERR_ARG, "grid side above %d (nx=%d, ny=%d)", MAX_SIDE, nx, ny);
    if (pitch < nx || pitch % 4 != 0)
        return fail(PF_ERR_LAYOUT, "pitch %d must be >= nx=%d and a multiple of 4", pitch, nx);
    return PF_OK;
}

const char* last_error_text() { return g_last_error.c_str(); }

}  // namespace pf

namespace {

using pf::check_sizes;
using pf::cuda_fail;
using pf::fail;

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// Workspace layout (all offsets 256-byte aligned).
struct Layout {
    size_t state;     // 3 planes of ny x pitch floats (ping-pong partner of the caller's fields)
    size_t partials;  // 4 x diag_blocks doubles
    size_t out;       // 4 doubles
    size_t hist;      // 3 long long + capacity x 5 doubles
    size_t err;       // int
    size_t total;
};

Layout layout(int nx, int ny, int pitch, int history_rows)
{
    Layout L{};
    size_t off = 0;
    L.state = off;
    off = align256(off + 3 * size_t(ny) * size_t(pitch) * sizeof(float));
    L.partials = off;
    off = align256(off + 4 * size_t(pf::diag_blocks(nx, ny)) * sizeof(double));
    L.out = off;
    off = align256(off + 4 * sizeof(double));
    L.hist = off;
    off = align256(off + 3 * sizeof(long long) + 5 * size_t(history_rows) * sizeof(double));
    L.err = off;
    off = align256(off + sizeof(int));
    L.total = off;
    return L;
}

int check_params(const pf_params* p)
{
    if (!p) return fail(PF_ERR_ARG, "null params");
    if (!(p->dx > 0.0) || !std::isfinite(p->dx)) return fail(PF_ERR_ARG, "dx must be positive");
    if (!(p->dt > 0.0) || !std::isfinite(p->dt)) return fail(PF_ERR_ARG, "dt must be positive");
    if (p->phi_mode != 0 && p->phi_mode != 1) return fail(PF_ERR_ARG, "phi_mode must be 0 or 1");
    if (p->diag_every < 0) return fail(PF_ERR_ARG, "diag_every must be >= 0");
    if ((p->MA_surf != 0.0 || p->MB_surf != 0.0) && !(p->sigma_surf > 0.0))
        return fail(PF_ERR_ARG, "sigma_surf must be positive when a surface mobility is set");
    const double v[] = {p->W_c, p->W_phi, p->kappa_c, p->kappa_phi, p->MA_bulk, p->MB_bulk, p->MA_surf,
                        p->MB_surf, p->M_phi, p->L_phi, p->D_rho, p->v_mag, p->v_angle_deg, p->rho_top};
    for (double x : v)
        if (!std::isfinite(x)) return fail(PF_ERR_ARG, "non-finite parameter");
    return PF_OK;
}

void velocity(const pf_params* p, double* vx, double* vy) { pf::velocity_of(*p, vx, vy); }

// |R(z)| of the explicit midpoint method, R(z) = 1 + z + z^2/2.
double midpoint_gain(std::complex<double> z) { return std::abs(1.0 + z + 0.5 * z * z); }

bool vapor_stable(const pf_params* p, double dt)
{
    double vx, vy;
    velocity(p, &vx, &vy);
    const double dx = p->dx;
    for (int a = -256; a <= 256; ++a) {
        const double tx = M_PI * a / 256.0;
        for (int b = 0; b <= 256; ++b) {
            const double ty = M_PI * b / 256.0;
            const double lam = 4.0 / (dx * dx) * (std::pow(std::sin(0.5 * tx), 2) + std::pow(std::sin(0.5 * ty), 2));
            const std::complex<double> z(-dt * p->D_rho * lam, -dt * (vx * std::sin(tx) + vy * std::sin(ty)) / dx);
            if (midpoint_gain(z) > 1.0 + 1e-13) return false;
        }
    }
    return true;
}

}  // namespace

struct pf_handle {
    pf_params p;
    int nx, ny, pitch;
    float* u[2][3];  // [0]: caller's fields, [1]: workspace partner
    int cur;         // which of u[] holds the current state
    long step;
    cudaStream_t stream;
    double* partials;
    double* out;
    long long* hist;
    int hist_cap;
    int* err;
    pf::StepConst k;
    pf::DiagConst d;
    int mob;
    int tile;
    bool ring;              // large grids: the persistent tile loop (TILE_LARGE tiles, next tile staged ahead)
    bool tma;               // tiles staged by TMA through maps[buffer] (all but the wraps of widths not a multiple of 4)
    pf::StepMaps maps[2];   // tensor maps of u[0] and u[1]
    int spl;                // steps per launch: 1, or 2 (two steps per launch where the diagnostics allow)
    bool tma2;              // the two-step kernel's interior tiles staged by TMA through maps2[buffer]
    pf::StepMaps maps2[2];  // tensor maps of u[0] and u[1] with the two-step kernel's taller box
    cudaGraphExec_t gexec;
    long gsteps;  // steps per graph replay (0: no graph yet)
};

namespace {

int do_step(pf_handle* h)
{
    const int a = h->cur, b = 1 - h->cur;
    const pf::StepMaps* maps = h->tma ? &h->maps[a] : nullptr;
    cudaError_t e = h->ring ? pf::launch_step_ring(h->k, h->p.phi_mode, h->mob, h->u[a][0], h->u[a][1], h->u[a][2],
                                                   h->u[b][0], h->u[b][1], h->u[b][2], h->stream, maps, h->err)
                            : pf::launch_step(h->k, h->tile, h->p.phi_mode, h->mob, h->u[a][0], h->u[a][1], h->u[a][2],
                                              h->u[b][0], h->u[b][1], h->u[b][2], h->stream, maps, h->err);
    if (e != cudaSuccess) return cuda_fail(e, "step launch");
    h->cur = b;
    return PF_OK;
}

int do_step2(pf_handle* h)
{
    const int a = h->cur, b = 1 - h->cur;
    cudaError_t e = pf::launch_step2(h->k, h->p.phi_mode, h->mob, h->u[a][0], h->u[a][1], h->u[a][2], h->u[b][0],
                                     h->u[b][1], h->u[b][2], h->stream, h->tma2 ? &h->maps2[a] : nullptr, h->err);
    if (e != cudaSuccess) return cuda_fail(e, "two-step launch");
    h->cur = b;
    return PF_OK;
}

// Two steps in one launch from the current step: on when selected, at least two steps are left,
// and no diagnostic record falls between the two (an even period from an even step).
bool two_steps_now(const pf_handle* h, long left)
{
    if (h->spl != 2 || left < 2) return false;
    return h->p.diag_every <= 0 || (h->p.diag_every % 2 == 0 && h->step % 2 == 0);
}

int do_record(pf_handle* h)
{
    cudaError_t e = pf::launch_diag(h->d, h->u[h->cur][0], h->u[h->cur][1], h->u[h->cur][2], h->partials, h->err,
                                    h->out, h->hist, h->p.diag_every, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "diagnostic launch");
    return PF_OK;
}

// Enqueue steps [h->step, h->step + n) one launch at a time (no graph).
int run_plain(pf_handle* h, long n)
{
    for (long s = 0; s < n;) {
        if (h->p.diag_every > 0 && h->step % h->p.diag_every == 0) {
            int rc = do_record(h);
            if (rc) return rc;
        }
        if (two_steps_now(h, n - s)) {
            int rc = do_step2(h);
            if (rc) return rc;
            h->step += 2;
            s += 2;
        } else {
            int rc = do_step(h);
            if (rc) return rc;
            ++h->step;
            ++s;
        }
    }
    return PF_OK;
}

// Capture a graph of gsteps steps starting from buffer 0 at a step index aligned
// to the diagnostic period (gsteps is even, and a multiple of 4 with two steps per
// launch, so the graph has an even number of launches and ends in buffer 0).
int build_graph(pf_handle* h, long gsteps)
{
    cudaStream_t cap;
    cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "capture stream");
    pf_handle tmp = *h;
    tmp.stream = cap;
    tmp.cur = 0;
    tmp.step = 0;
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaStreamDestroy(cap);
        return cuda_fail(e, "begin capture");
    }
    int rc = run_plain(&tmp, gsteps);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(cap, &g);
    cudaStreamDestroy(cap);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "end capture");
    e = cudaGraphInstantiate(&h->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        h->gexec = nullptr;
        return cuda_fail(e, "graph instantiate");
    }
    h->gsteps = gsteps;
    return PF_OK;
}

// Copy the state between caller host arrays (row pitch host_pitch floats) and the handle's fields.
int host_copy(pf_handle* h, float* const* host, int host_pitch, bool to_device)
{
    if (!h || !host || !host[0] || !host[1] || !host[2]) return fail(PF_ERR_ARG, "null pointer");
    if (host_pitch < h->nx) return fail(PF_ERR_LAYOUT, "host pitch %d < nx %d", host_pitch, h->nx);
    const size_t rowd = size_t(h->pitch) * sizeof(float), rowh = size_t(host_pitch) * sizeof(float);
    const size_t width = size_t(h->nx) * sizeof(float);
    for (int q = 0; q < 3; ++q) {
        float* dev = h->u[h->cur][q];
        cudaError_t e = to_device ? cudaMemcpy2DAsync(dev, rowd, host[q], rowh, width, h->ny, cudaMemcpyHostToDevice,
                                                      h->stream)
                                  : cudaMemcpy2DAsync(host[q], rowh, dev, rowd, width, h->ny, cudaMemcpyDeviceToHost,
                                                      h->stream);
        if (e != cudaSuccess) return cuda_fail(e, to_device ? "host-to-device copy" : "device-to-host copy");
    }
    return PF_OK;
}

long graph_block(const pf_handle* h)
{
    const pf_params* p = &h->p;
    if (p->diag_every <= 0) return 256;
    long g = p->diag_every;
    while (g < 64) g *= 2;  // small periods: several records per replay
    if (g % 2) g *= 2;
    if (h->spl == 2 && g % 4) g *= 2;  // an even number of two-step launches
    return g;
}

}  // namespace

extern "C" {

const char* pf_strerror(int code)
{
    switch (code) {
    case PF_OK: return "ok";
    case PF_ERR_ARG: return "invalid argument";
    case PF_ERR_LAYOUT: return "invalid memory layout";
    case PF_ERR_UNSTABLE: return "time step above the explicit stability limit";
    case PF_ERR_NONFINITE: return "non-finite value in a field";
    case PF_ERR_TIMEOUT: return "bounded device wait ran out";
    case PF_ERR_CUDA: return "CUDA runtime error";
    default: return "unknown error";
    }
}

const char* pf_last_error(void) { return pf::last_error_text(); }

int pf_dt_limit(const pf_params* p, double out[4])
{
    if (!p || !out) return fail(PF_ERR_ARG, "null pointer");
    if (!(p->dx > 0.0)) return fail(PF_ERR_ARG, "dx must be positive");
    const double lam = 8.0 / (p->dx * p->dx);
    const double mmax = std::fmax(p->MA_bulk, p->MB_bulk) + std::fmax(p->MA_surf, p->MB_surf);
    const double dt_c = mmax > 0.0 ? 2.0 / (mmax * lam * (p->kappa_c * lam + 2.0 * p->W_c)) : INFINITY;
    const double fpp = 2.0 * p->W_phi + (3.0 / 32.0) * p->W_c;
    double dt_f;
    if (p->phi_mode == 0)
        dt_f = p->M_phi > 0.0 ? 2.0 / (p->M_phi * lam * (p->kappa_phi * lam + fpp)) : INFINITY;
    else
        dt_f = p->L_phi > 0.0 ? 2.0 / (p->L_phi * (p->kappa_phi * lam + fpp)) : INFINITY;
    double hi = p->D_rho > 0.0 ? 2.0 / (p->D_rho * lam) : 1.0, lo = 0.0;
    if (vapor_stable(p, hi)) {
        lo = hi;
    } else {
        for (int it = 0; it < 80; ++it) {
            const double mid = 0.5 * (lo + hi);
            (vapor_stable(p, mid) ? lo : hi) = mid;
        }
    }
    out[1] = dt_c;
    out[2] = dt_f;
    out[3] = lo;
    out[0] = std::fmin(dt_c, std::fmin(dt_f, lo));
    return PF_OK;
}

size_t pf_workspace_size(int nx, int ny, int pitch, int history_rows)
{
    if (nx < 1 || ny < 1 || pitch < nx || history_rows < 0) return 0;
    return layout(nx, ny, pitch, history_rows < 1 ? 1 : history_rows).total;
}

int pf_init(const pf_params* p, int nx, int ny, int pitch, float* phi, float* c, float* rho, void* work,
            size_t work_bytes, int history_rows, void* stream, pf_handle** out)
{
    if (!out) return fail(PF_ERR_ARG, "null output handle pointer");
    *out = nullptr;
    int rc = check_params(p);
    if (rc) return rc;
    rc = check_sizes(nx, ny, pitch);
    if (rc) return rc;
    if (!phi || !c || !rho || !work) return fail(PF_ERR_ARG, "null field or workspace pointer");
    if (!aligned(phi, 16) || !aligned(c, 16) || !aligned(rho, 16))
        return fail(PF_ERR_LAYOUT, "fields must be 16-byte aligned");
    if (!aligned(work, 256)) return fail(PF_ERR_LAYOUT, "workspace must be 256-byte aligned");
    if (history_rows < 0) return fail(PF_ERR_ARG, "history_rows must be >= 0");
    const int cap = history_rows < 1 ? 1 : history_rows;
    const Layout L = layout(nx, ny, pitch, cap);
    if (work_bytes < L.total)
        return fail(PF_ERR_LAYOUT, "workspace of %zu bytes, %zu needed", work_bytes, L.total);
    double lim[4];
    pf_dt_limit(p, lim);
    if (p->dt > lim[0] * (1.0 + 1e-12))
        return fail(PF_ERR_UNSTABLE, "dt=%.6g above the stability limit %.6g", p->dt, lim[0]);

    pf_handle* h = new (std::nothrow) pf_handle();
    if (!h) return fail(PF_ERR_ARG, "out of host memory");
    char* w = static_cast<char*>(work);
    const size_t plane = size_t(ny) * size_t(pitch);
    float* st = reinterpret_cast<float*>(w + L.state);
    h->p = *p;
    h->nx = nx;
    h->ny = ny;
    h->pitch = pitch;
    h->u[0][0] = phi;
    h->u[0][1] = c;
    h->u[0][2] = rho;
    h->u[1][0] = st;
    h->u[1][1] = st + plane;
    h->u[1][2] = st + 2 * plane;
    h->cur = 0;
    h->step = 0;
    h->stream = static_cast<cudaStream_t>(stream);
    h->partials = reinterpret_cast<double*>(w + L.partials);
    h->out = reinterpret_cast<double*>(w + L.out);
    h->hist = reinterpret_cast<long long*>(w + L.hist);
    h->hist_cap = cap;
    h->err = reinterpret_cast<int*>(w + L.err);
    h->k = pf::step_const_of(*p, nx, ny, pitch);
    h->d = pf::diag_const_of(*p, nx, ny, pitch);
    h->mob = pf::mob_kind_of(*p);
    h->tile = pf::choose_tile(nx, ny);
    h->ring = false;  // the tile loop is opt-in: one CTA per tile measured faster on GB300
    // tiles are staged by TMA whenever the grid holds an interior tile's full staged window
    h->tma =
             pf::make_step_maps(h->u[0][0], h->u[0][1], h->u[0][2], nx, ny, pitch, h->tile, &h->maps[0]) &&
             pf::make_step_maps(h->u[1][0], h->u[1][1], h->u[1][2], nx, ny, pitch, h->tile, &h->maps[1]);
    // one step per launch: two per launch (opt-in) measured no faster at 512^2 and slower at 64^2
    h->spl = 1;
    const int TY2 = pf::step2_tile_height();
    h->tma2 = pf::make_maps_box(h->u[0][0], h->u[0][1], h->u[0][2], nx, ny, pitch, pf::step2_box_rows(),
                                pf::step2_tile_width() - 8, TY2 - 8, &h->maps2[0]) &&
              pf::make_maps_box(h->u[1][0], h->u[1][1], h->u[1][2], nx, ny, pitch, pf::step2_box_rows(),
                                pf::step2_tile_width() - 8, TY2 - 8, &h->maps2[1]);
    h->gexec = nullptr;
    h->gsteps = 0;
    cudaError_t e = pf::launch_reset(h->hist, cap, 0, h->err, h->stream);
    if (e != cudaSuccess) {
        delete h;
        return cuda_fail(e, "workspace reset");
    }
    *out = h;
    return PF_OK;
}

int pf_step(pf_handle* h, long n)
{
    pf::TraceRange trace("pf_step");
    if (!h) return fail(PF_ERR_ARG, "null handle");
    if (n < 0) return fail(PF_ERR_ARG, "negative step count");
    const long G = graph_block(h);
    long left = n;
    while (left > 0) {
        const bool replay_ok = left >= G && (h->gexec != nullptr || n >= 2 * G);
        const bool phase_ok = h->p.diag_every <= 0 || h->step % h->p.diag_every == 0;
        if (replay_ok && phase_ok && h->cur == 0) {
            // The graph holds G steps from buffer 0 at a diagnostic-aligned step
            // (G is even and a multiple of the period), records tagged on the device.
            if (!h->gexec) {
                int rc = build_graph(h, G);
                if (rc) return rc;
            }
            cudaError_t e = cudaGraphLaunch(h->gexec, h->stream);
            if (e != cudaSuccess) return cuda_fail(e, "graph launch");
            h->step += G;
            left -= G;
            continue;
        }
        // single steps until a replay can start, or the whole tail when none can
        const long m = replay_ok ? 1 : left;
        int rc = run_plain(h, m);
        if (rc) return rc;
        left -= m;
    }
    if (h->cur != 0) {
        // leave the state in the caller's buffers
        const size_t rowb = size_t(h->pitch) * sizeof(float);
        for (int q = 0; q < 3; ++q) {  // the nx model columns; the caller's padding is left alone
            cudaError_t e = cudaMemcpy2DAsync(h->u[0][q], rowb, h->u[1][q], rowb, size_t(h->nx) * sizeof(float),
                                              size_t(h->ny), cudaMemcpyDeviceToDevice, h->stream);
            if (e != cudaSuccess) return cuda_fail(e, "copy back");
        }
        h->cur = 0;
    }
    return PF_OK;
}

int pf_diag(pf_handle* h, double out[4])
{
    if (!h || !out) return fail(PF_ERR_ARG, "null pointer");
    cudaError_t e = pf::launch_diag(h->d, h->u[h->cur][0], h->u[h->cur][1], h->u[h->cur][2], h->partials, h->err,
                                    h->out, nullptr, 0, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "diagnostic launch");
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
    int err = 0;
    e = cudaMemcpy(out, h->out, 4 * sizeof(double), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&err, h->err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "diagnostic read-back");
    if (err & pf::ERR_BIT_TIMEOUT) return fail(PF_ERR_TIMEOUT, "a step kernel's bounded wait for its TMA copies ran out");
    if (err & 1) return fail(PF_ERR_NONFINITE, "a diagnostic pass saw a NaN or Inf");
    return PF_OK;
}

int pf_diag_history(pf_handle* h, double* out, int max_rows, int* rows)
{
    if (!h || !rows || (max_rows > 0 && !out)) return fail(PF_ERR_ARG, "null pointer");
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
    long long meta[3];
    e = cudaMemcpy(meta, h->hist, sizeof meta, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "history read-back");
    const long long cnt = meta[0], cap = meta[2];
    const long long have = cnt < cap ? cnt : cap;
    const long long first = cnt - have;  // oldest record still held
    long long m = have < max_rows ? have : max_rows;
    const double* recs = reinterpret_cast<const double*>(h->hist + 3);
    for (long long r = 0; r < m; ++r) {
        const long long slot = (first + r) % cap;
        e = cudaMemcpy(out + 5 * r, recs + 5 * slot, 5 * sizeof(double), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "history read-back");
    }
    *rows = int(m);
    return PF_OK;
}

long pf_get_step(const pf_handle* h) { return h ? h->step : -1; }

int pf_set_step(pf_handle* h, long step)
{
    if (!h) return fail(PF_ERR_ARG, "null handle");
    if (step < 0) return fail(PF_ERR_ARG, "negative step");
    h->step = step;
    long long next = 0;
    if (h->p.diag_every > 0) next = ((step + h->p.diag_every - 1) / h->p.diag_every) * h->p.diag_every;
    cudaError_t e = pf::launch_reset(h->hist, h->hist_cap, next, nullptr, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "history reset");
    return PF_OK;
}

int pf_set_wait_limit(pf_handle* h, int polls)
{
    if (!h) return fail(PF_ERR_ARG, "null handle");
    if (polls < 0) return fail(PF_ERR_ARG, "the wait limit must be >= 0");
    if (h->gexec) {  // the captured graph holds the old constants
        cudaGraphExecDestroy(h->gexec);
        h->gexec = nullptr;
    }
    h->k.wait_cap = polls;
    return PF_OK;
}

int pf_staging_mode(const pf_handle* h) { return h ? (h->tma ? 1 : 0) : -1; }

int pf_set_steps_per_launch(pf_handle* h, int steps)
{
    if (!h) return fail(PF_ERR_ARG, "null handle");
    if (steps != 1 && steps != 2) return fail(PF_ERR_ARG, "steps per launch must be 1 or 2 (got %d)", steps);
    const int prev = h->spl;
    if (steps != h->spl && h->gexec) {  // the captured graph holds the other schedule
        cudaGraphExecDestroy(h->gexec);
        h->gexec = nullptr;
    }
    h->spl = steps;
    return prev;
}

int pf_set_tile_loop(pf_handle* h, int on)
{
    if (!h) return fail(PF_ERR_ARG, "null handle");
    if (h->tile != pf::TILE_LARGE) return fail(PF_ERR_ARG, "the tile loop is built for grids above 2^20 cells");
    const int prev = h->ring ? 1 : 0;
    if ((on != 0) != h->ring && h->gexec) {  // the captured graph holds the other kernel
        cudaGraphExecDestroy(h->gexec);
        h->gexec = nullptr;
    }
    h->ring = on != 0;
    return prev;
}

int pf_load_host(pf_handle* h, const float* phi, const float* c, const float* rho, int host_pitch)
{
    float* host[3] = {const_cast<float*>(phi), const_cast<float*>(c), const_cast<float*>(rho)};
    return host_copy(h, host, host_pitch, true);
}

int pf_store_host(pf_handle* h, float* phi, float* c, float* rho, int host_pitch)
{
    float* host[3] = {phi, c, rho};
    return host_copy(h, host, host_pitch, false);
}

int pf_clear_error(pf_handle* h)
{
    if (!h) return fail(PF_ERR_ARG, "null handle");
    cudaError_t e = cudaMemsetAsync(h->err, 0, sizeof(int), h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "clear error word");
    return PF_OK;
}

int pf_destroy(pf_handle* h)
{
    if (!h) return PF_OK;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    delete h;
    if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
    return PF_OK;
}

size_t pf_diag_workspace_size(int nx, int ny)
{
    if (nx < 1 || ny < 1) return 0;
    return align256(4 * size_t(pf::diag_blocks(nx, ny)) * sizeof(double)) + 256;
}

size_t pf_diag_error_offset(int nx, int ny)
{
    return align256(4 * size_t(pf::diag_blocks(nx, ny)) * sizeof(double));
}

int pf_diagnostics(const pf_params* p, int nx, int ny, int pitch, const float* phi, const float* c,
                   const float* rho, void* work, size_t work_bytes, double* out_dev, void* stream)
{
    if (!p) return fail(PF_ERR_ARG, "null params");
    if (!(p->dx > 0.0)) return fail(PF_ERR_ARG, "dx must be positive");
    int rc = check_sizes(nx, ny, pitch);
    if (rc) return rc;
    if (!phi || !c || !rho || !work || !out_dev) return fail(PF_ERR_ARG, "null pointer");
    if (!aligned(work, 256) || !aligned(out_dev, 8)) return fail(PF_ERR_LAYOUT, "misaligned workspace or output");
    if (work_bytes < pf_diag_workspace_size(nx, ny))
        return fail(PF_ERR_LAYOUT, "workspace of %zu bytes, %zu needed", work_bytes, pf_diag_workspace_size(nx, ny));
    char* w = static_cast<char*>(work);
    cudaError_t e = pf::launch_diag(pf::diag_const_of(*p, nx, ny, pitch), phi, c, rho, reinterpret_cast<double*>(w),
                                    reinterpret_cast<int*>(w + pf_diag_error_offset(nx, ny)), out_dev, nullptr, 0,
                                    static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "diagnostic launch");
    return PF_OK;
}

}  // extern "C"
