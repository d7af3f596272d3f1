// C-ABI layer of the batched ensemble (declarations in include/pf.h): many
// independent deposition runs of uneven grid sizes and per-run parameters
// advanced in lockstep, every step of every run in ONE launch of the fused
// step kernel over a table of tiles, long runs as CUDA-graph replays, and a
// small autotuner that picks the tile shape by timing it.
//
// The paper's dataset is a sweep of independent runs over deposition rate,
// angle and mobilities ("Dataset"); the ensemble is that sweep on one GPU.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <new>
#include <string>
#include <vector>

#include "pf.h"
#include "pf_internal.h"

namespace {

thread_local std::string g_ens_error;

int efail(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_ens_error = buf;
    return code;
}

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

struct EnsLayout {
    std::vector<size_t> state;  // per-run offset of the partner buffer (3 planes)
    size_t runs;                // EnsRun[nruns]
    size_t tiles[pf::NUM_TILE_TABLES];
    int ntiles[pf::NUM_TILE_TABLES];
    size_t partials, out, err, bar, total;
};

bool ens_layout(int nruns, const int* nx, const int* ny, const int* pitch, EnsLayout& L)
{
    size_t off = 0;
    L.state.resize(nruns);
    for (int r = 0; r < nruns; ++r) {
        if (nx[r] < 1 || ny[r] < 1 || pitch[r] < nx[r]) return false;
        L.state[r] = off;
        off = al256(off + 3 * size_t(ny[r]) * size_t(pitch[r]) * sizeof(float));
    }
    L.runs = off;
    off = al256(off + size_t(nruns) * sizeof(pf::EnsRun));
    for (int t = 0; t < pf::NUM_TILE_TABLES; ++t) {
        long long n = 0;
        for (int r = 0; r < nruns; ++r)
            n += (long long)((nx[r] + pf::tile_width() - 1) / pf::tile_width()) *
                 ((ny[r] + pf::tile_height(t) - 1) / pf::tile_height(t));
        if (n > (1LL << 30)) return false;
        L.ntiles[t] = int(n);
        L.tiles[t] = off;
        off = al256(off + size_t(n) * sizeof(pf::EnsTile));
    }
    L.partials = off;
    off = al256(off + 4 * size_t(pf::diag_blocks(1 << 20, 1 << 20)) * sizeof(double));
    L.out = off;
    off = al256(off + 4 * sizeof(double));
    L.err = off;
    off = al256(off + sizeof(int));
    L.bar = off;  // grid-barrier counter of the persistent kind
    off = al256(off + sizeof(unsigned));
    L.total = off;
    return true;
}

// dt of one run inside (0, its stability limit].
bool dt_ok(const pf_params& p)
{
    double lim[4];
    if (pf_dt_limit(&p, lim) != PF_OK) return false;
    return p.dt > 0.0 && p.dt <= lim[0] * (1.0 + 1e-12);
}

}  // namespace

struct pf_ens {
    int nruns;
    std::vector<pf_params> p;
    std::vector<int> nx, ny, pitch;
    std::vector<pf::EnsRun> host_runs;  // [0] buffers = caller's fields
    pf::EnsRun* runs;                    // device copy
    pf::EnsTile* tiles[pf::NUM_TILE_TABLES];
    int ntiles[pf::NUM_TILE_TABLES];
    int tile;
    int phi_mode, mob;
    int parity;  // which buffer of every run is current (0: caller's)
    long step;
    double* partials;
    double* out;
    int* err;
    unsigned* bar;    // grid-barrier counter of the persistent kind
    int wait_cap;     // polls of a barrier wait before it reports a timeout
    bool persist_ok;  // every run has nx % 4 == 0: the persistent kind can run
    std::vector<pf::EnsMaps> maps;  // [2 kind + buffer], kinds 0 (short) and 1 (large tile): TMA staging
    bool tma_ok[2];                 // the kind's maps are encoded for every run it can stage by TMA
    bool use_tma;                   // pf_ens_set_tma
    cudaStream_t stream;
    cudaGraphExec_t gexec;
    int gtile;
    long gsteps;
};

namespace {

// n steps of every run from buffer `parity` on stream s: one persistent launch for the persistent
// kind, else n one-step launches.
bool ens_tma(const pf_ens* e)
{
    return e->use_tma && (e->tile == pf::TILE_SMALL || e->tile == pf::TILE_LARGE) && e->tma_ok[e->tile];
}

cudaError_t ens_enqueue(pf_ens* e, long n, int parity, cudaStream_t s)
{
    const int tab = pf::tile_table(e->tile);
    if (e->tile == pf::TILE_LARGE_PERSIST)
        return pf::launch_ens_persistent(e->phi_mode, e->mob, e->tiles[tab], e->runs, e->ntiles[tab], parity, int(n),
                                         e->bar, e->wait_cap, e->err, s);
    const bool tma = ens_tma(e);
    for (long k = 0; k < n; ++k) {
        const int b = int((parity + k) & 1);
        cudaError_t c = pf::launch_ens_step(e->tile, e->phi_mode, e->mob, e->tiles[tab], e->runs, e->ntiles[tab], b,
                                            s, tma ? &e->maps[2 * e->tile + b] : nullptr, e->err);
        if (c != cudaSuccess) return c;
    }
    return cudaSuccess;
}

// Tensor maps of both buffers of every run for the short and the large tile: a run gets maps when
// some tile of it can be TMA-staged (nx >= 64, ny >= the window height); a kind whose maps the
// driver refuses for any such run stages per thread.
void ens_encode_maps(pf_ens* e)
{
    e->maps.assign(4, pf::EnsMaps{});
    for (int kind = 0; kind < 2; ++kind) {
        const int LY = pf::tile_height(kind) + 8;
        bool ok = e->nruns <= pf::ENS_TMA_MAX_RUNS;
        for (int b = 0; b < 2 && ok; ++b)
            for (int r = 0; r < e->nruns && ok; ++r) {
                if (e->nx[r] < 64 || e->ny[r] < LY) continue;
                const pf::EnsRun& R = e->host_runs[r];
                ok = pf::make_maps_box(R.f[b][0], R.f[b][1], R.f[b][2], e->nx[r], e->ny[r], e->pitch[r], LY, 0, 0,
                                       &e->maps[2 * kind + b].run[r]);
            }
        e->tma_ok[kind] = ok;
    }
}

int ens_launch(pf_ens* e)
{
    cudaError_t c = ens_enqueue(e, 1, e->parity, e->stream);
    if (c != cudaSuccess) return efail(PF_ERR_CUDA, "ensemble step launch: %s", cudaGetErrorString(c));
    e->parity = 1 - e->parity;
    return PF_OK;
}

int ens_graph(pf_ens* e, long G)
{
    if (e->gexec) {
        cudaGraphExecDestroy(e->gexec);
        e->gexec = nullptr;
    }
    cudaStream_t cap;
    cudaError_t c = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (c != cudaSuccess) return efail(PF_ERR_CUDA, "capture stream: %s", cudaGetErrorString(c));
    c = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (c != cudaSuccess) {
        cudaStreamDestroy(cap);
        return efail(PF_ERR_CUDA, "begin capture: %s", cudaGetErrorString(c));
    }
    int rc = PF_OK;
    c = ens_enqueue(e, G, 0, cap);
    if (c != cudaSuccess) rc = efail(PF_ERR_CUDA, "ensemble capture: %s", cudaGetErrorString(c));
    cudaGraph_t g = nullptr;
    c = cudaStreamEndCapture(cap, &g);
    cudaStreamDestroy(cap);
    if (rc != PF_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (c != cudaSuccess) return efail(PF_ERR_CUDA, "end capture: %s", cudaGetErrorString(c));
    c = cudaGraphInstantiate(&e->gexec, g, 0);
    cudaGraphDestroy(g);
    if (c != cudaSuccess) {
        e->gexec = nullptr;
        return efail(PF_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(c));
    }
    e->gtile = e->tile;
    e->gsteps = G;
    return PF_OK;
}

constexpr long ENS_GRAPH_STEPS = 100;  // even: a replay starts and ends in the caller's buffers

}  // namespace

namespace pf {

int ens_runs(const pf_ens* e) { return e ? e->nruns : 0; }

void ens_run_fields(const pf_ens* e, int run, float** phi, float** c, float** rho, int* nx, int* ny, int* pitch)
{
    const EnsRun& r = e->host_runs[run];
    *phi = r.f[0][0];
    *c = r.f[0][1];
    *rho = r.f[0][2];
    *nx = e->nx[run];
    *ny = e->ny[run];
    *pitch = e->pitch[run];
}

cudaStream_t ens_stream(const pf_ens* e) { return e->stream; }

}  // namespace pf

extern "C" {

size_t pf_ens_workspace_size(int nruns, const int* nx, const int* ny, const int* pitch)
{
    if (nruns < 1 || !nx || !ny || !pitch) return 0;
    EnsLayout L;
    if (!ens_layout(nruns, nx, ny, pitch, L)) return 0;
    return L.total;
}

int pf_ens_init(int nruns, const pf_params* params, const int* nx, const int* ny, const int* pitch,
                float* const* phi, float* const* c, float* const* rho, void* work, size_t work_bytes, void* stream,
                pf_ens** out)
{
    if (!out) return efail(PF_ERR_ARG, "null output handle pointer");
    *out = nullptr;
    if (nruns < 1 || !params || !nx || !ny || !pitch || !phi || !c || !rho || !work)
        return efail(PF_ERR_ARG, "null pointer or no runs");
    if (reinterpret_cast<uintptr_t>(work) % 256) return efail(PF_ERR_LAYOUT, "workspace must be 256-byte aligned");
    EnsLayout L;
    for (int r = 0; r < nruns; ++r) {
        if (nx[r] < 1 || ny[r] < 1 || nx[r] > (1 << 20) || ny[r] > (1 << 20))
            return efail(PF_ERR_ARG, "run %d: grid %d x %d out of range", r, nx[r], ny[r]);
        if (pitch[r] < nx[r] || pitch[r] % 4) return efail(PF_ERR_LAYOUT, "run %d: bad pitch %d", r, pitch[r]);
        if (!phi[r] || !c[r] || !rho[r]) return efail(PF_ERR_ARG, "run %d: null field", r);
        if ((reinterpret_cast<uintptr_t>(phi[r]) | reinterpret_cast<uintptr_t>(c[r]) |
             reinterpret_cast<uintptr_t>(rho[r])) % 16)
            return efail(PF_ERR_LAYOUT, "run %d: fields must be 16-byte aligned", r);
        const pf_params& p = params[r];
        if (!(p.dx > 0.0) || (p.phi_mode != 0 && p.phi_mode != 1))
            return efail(PF_ERR_ARG, "run %d: bad dx or phi_mode", r);
        if ((p.MA_surf != 0.0 || p.MB_surf != 0.0) && !(p.sigma_surf > 0.0))
            return efail(PF_ERR_ARG, "run %d: sigma_surf must be positive", r);
        if (p.phi_mode != params[0].phi_mode || pf::mob_kind_of(p) != pf::mob_kind_of(params[0]))
            return efail(PF_ERR_ARG, "run %d: all runs must share phi_mode and the mobility form", r);
        if (!dt_ok(p)) return efail(PF_ERR_UNSTABLE, "run %d: dt=%.6g outside (0, stability limit]", r, p.dt);
    }
    if (!ens_layout(nruns, nx, ny, pitch, L)) return efail(PF_ERR_ARG, "ensemble too large");
    if (work_bytes < L.total) return efail(PF_ERR_LAYOUT, "workspace of %zu bytes, %zu needed", work_bytes, L.total);

    pf_ens* e = new (std::nothrow) pf_ens();
    if (!e) return efail(PF_ERR_ARG, "out of host memory");
    char* w = static_cast<char*>(work);
    e->nruns = nruns;
    e->p.assign(params, params + nruns);
    e->nx.assign(nx, nx + nruns);
    e->ny.assign(ny, ny + nruns);
    e->pitch.assign(pitch, pitch + nruns);
    e->host_runs.resize(nruns);
    for (int r = 0; r < nruns; ++r) {
        pf::EnsRun& R = e->host_runs[r];
        R.k = pf::step_const_of(params[r], nx[r], ny[r], pitch[r]);
        const size_t plane = size_t(ny[r]) * size_t(pitch[r]);
        float* st = reinterpret_cast<float*>(w + L.state[r]);
        R.f[0][0] = phi[r];
        R.f[0][1] = c[r];
        R.f[0][2] = rho[r];
        R.f[1][0] = st;
        R.f[1][1] = st + plane;
        R.f[1][2] = st + 2 * plane;
    }
    e->runs = reinterpret_cast<pf::EnsRun*>(w + L.runs);
    e->stream = static_cast<cudaStream_t>(stream);
    // tile tables: largest runs first, so the tail of a launch is short tiles of small runs.  In a run whose
    // width is a multiple of 4 the last tile column starts at nx - 56, overlapping its neighbour (which
    // computes the same values for the shared cells), so its window reaches only 4 columns past the edge
    // and can be staged by TMA (the kernels' tile_x0 does the same for single runs).
    std::vector<int> order(nruns);
    for (int r = 0; r < nruns; ++r) order[r] = r;
    for (int i = 1; i < nruns; ++i)
        for (int j = i; j > 0 && (long long)nx[order[j]] * ny[order[j]] > (long long)nx[order[j - 1]] * ny[order[j - 1]];
             --j)
            std::swap(order[j], order[j - 1]);
    cudaError_t ce = cudaMemcpyAsync(e->runs, e->host_runs.data(), sizeof(pf::EnsRun) * nruns,
                                     cudaMemcpyHostToDevice, e->stream);
    std::vector<std::vector<pf::EnsTile>> tabs(pf::NUM_TILE_TABLES);
    for (int t = 0; t < pf::NUM_TILE_TABLES && ce == cudaSuccess; ++t) {
        const int TW = pf::tile_width(), TH = pf::tile_height(t);
        for (int r : order)
            for (int y = 0; y < ny[r]; y += TH)
                for (int x = 0; x < nx[r]; x += TW) {
                    const bool shift = nx[r] % 4 == 0 && nx[r] >= TW && x + TW > nx[r];
                    tabs[t].push_back(pf::EnsTile{r, shift ? nx[r] - TW : x, y});
                }
        e->tiles[t] = reinterpret_cast<pf::EnsTile*>(w + L.tiles[t]);
        e->ntiles[t] = int(tabs[t].size());
        if (!tabs[t].empty())
            ce = cudaMemcpyAsync(e->tiles[t], tabs[t].data(), sizeof(pf::EnsTile) * tabs[t].size(),
                                 cudaMemcpyHostToDevice, e->stream);
    }
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(e->stream);  // host tables go out of scope
    if (ce != cudaSuccess) {
        delete e;
        return efail(PF_ERR_CUDA, "ensemble tables: %s", cudaGetErrorString(ce));
    }
    long long cells = 0;
    for (int r = 0; r < nruns; ++r) cells += (long long)nx[r] * ny[r];
    e->tile = cells / nruns <= (1LL << 20) ? pf::TILE_SMALL : pf::TILE_LARGE;
    e->phi_mode = params[0].phi_mode;
    e->mob = pf::mob_kind_of(params[0]);
    e->parity = 0;
    e->step = 0;
    e->partials = reinterpret_cast<double*>(w + L.partials);
    e->out = reinterpret_cast<double*>(w + L.out);
    e->err = reinterpret_cast<int*>(w + L.err);
    e->bar = reinterpret_cast<unsigned*>(w + L.bar);
    e->wait_cap = 1 << 22;
    e->persist_ok = true;
    for (int r = 0; r < nruns; ++r) e->persist_ok &= (nx[r] % 4) == 0;
    e->use_tma = true;
    ens_encode_maps(e);
    e->gexec = nullptr;
    e->gtile = -1;
    e->gsteps = 0;
    ce = pf::launch_reset(nullptr, 0, 0, e->err, e->stream);
    if (ce != cudaSuccess) {
        delete e;
        return efail(PF_ERR_CUDA, "workspace reset: %s", cudaGetErrorString(ce));
    }
    *out = e;
    return PF_OK;
}

int pf_ens_step(pf_ens* e, long n)
{
    pf::TraceRange trace("pf_ens_step");
    if (!e) return efail(PF_ERR_ARG, "null handle");
    if (n < 0) return efail(PF_ERR_ARG, "negative step count");
    const long G = ENS_GRAPH_STEPS;
    long left = n;
    while (left > 0) {
        if (e->parity == 0 && left >= G && (n >= 2 * G || (e->gexec && e->gtile == e->tile))) {
            if (!e->gexec || e->gtile != e->tile) {
                int rc = ens_graph(e, G);
                if (rc) return rc;
            }
            cudaError_t c = cudaGraphLaunch(e->gexec, e->stream);
            if (c != cudaSuccess) return efail(PF_ERR_CUDA, "graph launch: %s", cudaGetErrorString(c));
            e->step += G;
            left -= G;
            continue;
        }
        if (e->tile == pf::TILE_LARGE_PERSIST) {  // the rest (or up to one graph block) as one launch
            const long m = left < G ? left : G;
            cudaError_t c = ens_enqueue(e, m, e->parity, e->stream);
            if (c != cudaSuccess) return efail(PF_ERR_CUDA, "persistent ensemble launch: %s", cudaGetErrorString(c));
            e->parity ^= int(m & 1);
            e->step += m;
            left -= m;
            continue;
        }
        int rc = ens_launch(e);
        if (rc) return rc;
        ++e->step;
        --left;
    }
    if (e->parity != 0) {  // leave every run's state in the caller's buffers
        for (int r = 0; r < e->nruns; ++r) {
            const size_t rowb = size_t(e->pitch[r]) * sizeof(float);
            for (int q = 0; q < 3; ++q) {  // the nx model columns; the caller's padding is left alone
                cudaError_t c = cudaMemcpy2DAsync(e->host_runs[r].f[0][q], rowb, e->host_runs[r].f[1][q], rowb,
                                                  size_t(e->nx[r]) * sizeof(float), size_t(e->ny[r]),
                                                  cudaMemcpyDeviceToDevice, e->stream);
                if (c != cudaSuccess) return efail(PF_ERR_CUDA, "copy back: %s", cudaGetErrorString(c));
            }
        }
        e->parity = 0;
    }
    return PF_OK;
}

int pf_ens_set_tile(pf_ens* e, int tile)
{
    if (!e) return efail(PF_ERR_ARG, "null handle");
    if (tile < 0 || tile >= pf::NUM_TILE_KINDS) return efail(PF_ERR_ARG, "tile kind %d out of range", tile);
    if (tile == pf::TILE_LARGE_PERSIST && !e->persist_ok)
        return efail(PF_ERR_ARG, "the persistent kind needs every run's nx to be a multiple of 4");
    e->tile = tile;
    return PF_OK;
}

int pf_ens_set_wait_limit(pf_ens* e, int polls)
{
    if (!e) return efail(PF_ERR_ARG, "null handle");
    if (polls < 0) return efail(PF_ERR_ARG, "the wait limit must be >= 0");
    if (e->gexec) {  // a captured graph holds the old limit
        cudaGraphExecDestroy(e->gexec);
        e->gexec = nullptr;
    }
    e->wait_cap = polls;
    // the TMA staging wait reads its limit from each run's constants (stream-ordered update)
    for (int r = 0; r < e->nruns; ++r) e->host_runs[r].k.wait_cap = polls;
    cudaError_t c = cudaMemcpyAsync(e->runs, e->host_runs.data(), sizeof(pf::EnsRun) * e->nruns,
                                    cudaMemcpyHostToDevice, e->stream);
    if (c == cudaSuccess) c = cudaStreamSynchronize(e->stream);  // the host table may change again
    if (c != cudaSuccess) return efail(PF_ERR_CUDA, "run table update: %s", cudaGetErrorString(c));
    return PF_OK;
}

int pf_ens_set_tma(pf_ens* e, int on)
{
    if (!e) return efail(PF_ERR_ARG, "null handle");
    if (e->gexec) {  // a captured graph holds the other kernel
        cudaGraphExecDestroy(e->gexec);
        e->gexec = nullptr;
    }
    e->use_tma = on != 0;
    return PF_OK;
}

int pf_ens_staging_mode(const pf_ens* e) { return e ? (ens_tma(e) ? 1 : 0) : -1; }

int pf_ens_get_tile(const pf_ens* e) { return e ? e->tile : -1; }

long pf_ens_get_step(const pf_ens* e) { return e ? e->step : -1; }

int pf_ens_autotune(pf_ens* e, int trial_steps, int* chosen, double* seconds_per_step)
{
    if (!e) return efail(PF_ERR_ARG, "null handle");
    if (trial_steps < 2 || trial_steps % 2) return efail(PF_ERR_ARG, "trial_steps must be even and >= 2");
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess)
        return efail(PF_ERR_CUDA, "event create");
    int best = e->tile;
    float best_ms = 0.f;
    int rc = PF_OK;
    for (int t = 0; t < pf::NUM_TILE_KINDS && rc == PF_OK; ++t) {
        if (t == pf::TILE_LARGE_PERSIST && !e->persist_ok) {
            if (seconds_per_step) seconds_per_step[t] = 0.0;  // not available for this ensemble
            continue;
        }
        e->tile = t;
        rc = ens_launch(e);  // warm the kernel (function attributes, caches)
        if (rc == PF_OK) rc = ens_launch(e);
        if (rc != PF_OK) break;
        e->step += 2;
        cudaEventRecord(a, e->stream);
        cudaError_t ce = ens_enqueue(e, trial_steps, e->parity, e->stream);  // trial_steps is even
        if (ce != cudaSuccess) rc = efail(PF_ERR_CUDA, "autotune launch: %s", cudaGetErrorString(ce));
        cudaEventRecord(b, e->stream);
        e->step += trial_steps;
        float ms = 0.f;
        if (rc == PF_OK && cudaEventSynchronize(b) == cudaSuccess && cudaEventElapsedTime(&ms, a, b) == cudaSuccess) {
            if (seconds_per_step) seconds_per_step[t] = ms * 1e-3 / trial_steps;
            if (t == 0 || ms < best_ms) {
                best = t;
                best_ms = ms;
            }
        } else if (rc == PF_OK) {
            rc = efail(PF_ERR_CUDA, "autotune timing");
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    e->tile = best;
    if (chosen) *chosen = best;
    return rc;
}

int pf_ens_diag(pf_ens* e, int run, double out[4])
{
    if (!e || !out) return efail(PF_ERR_ARG, "null pointer");
    if (run < 0 || run >= e->nruns) return efail(PF_ERR_ARG, "run %d out of range", run);
    const pf::DiagConst d = pf::diag_const_of(e->p[run], e->nx[run], e->ny[run], e->pitch[run]);
    const pf::EnsRun& R = e->host_runs[run];
    cudaError_t c = pf::launch_diag(d, R.f[e->parity][0], R.f[e->parity][1], R.f[e->parity][2], e->partials, e->err,
                                    e->out, nullptr, 0, e->stream);
    if (c == cudaSuccess) c = cudaStreamSynchronize(e->stream);
    int err = 0;
    if (c == cudaSuccess) c = cudaMemcpy(out, e->out, 4 * sizeof(double), cudaMemcpyDeviceToHost);
    if (c == cudaSuccess) c = cudaMemcpy(&err, e->err, sizeof(int), cudaMemcpyDeviceToHost);
    if (c != cudaSuccess) return efail(PF_ERR_CUDA, "ensemble diagnostics: %s", cudaGetErrorString(c));
    if (err & pf::ERR_BIT_TIMEOUT) return efail(PF_ERR_TIMEOUT, "a bounded grid-barrier wait ran out");
    if (err & 1) return efail(PF_ERR_NONFINITE, "a diagnostic pass saw a NaN or Inf");
    return PF_OK;
}

int pf_ens_destroy(pf_ens* e)
{
    if (!e) return PF_OK;
    cudaError_t c = cudaStreamSynchronize(e->stream);
    if (e->gexec) cudaGraphExecDestroy(e->gexec);
    delete e;
    if (c != cudaSuccess) return efail(PF_ERR_CUDA, "stream synchronize: %s", cudaGetErrorString(c));
    return PF_OK;
}

const char* pf_ens_last_error(void) { return g_ens_error.c_str(); }

}  // extern "C"
