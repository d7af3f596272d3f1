// Internal declarations shared by the kernels and the C-ABI layer (not installed).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "pf.h"

namespace pf {

// A named NVTX range over a C-ABI call (what the call enqueues, on the host timeline): profilers can
// select its kernels, e.g. ncu --nvtx --nvtx-include "pf_unet_jump/".  Without a tool attached the
// NVTX calls return at once.
struct TraceRange {
    explicit TraceRange(const char* name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};

// FP32 constants of one explicit midpoint step, folded from pf_params on the host.
struct StepConst {
    int nx, ny, pitch;
    float Wc;          // W_c
    float Wf;          // W_phi
    float kc;          // kappa_c / dx^2
    float kf;          // kappa_phi / dx^2
    float MBb, dMb;    // bulk mobility MB_bulk and MA_bulk - MB_bulk
    float MBs, dMs;    // surface mobility MB_surf and MA_surf - MB_surf
    float nisig2;      // -log2(e) / sigma_surf^2 (exp(-(phi/sigma)^2) = 2^(nisig2 phi^2))
    float cR;          // 1 / (2 dx^2): face mean 1/2 (M + M_nb) and the 1/dx^2 of the divergence
    float cF;          // phi_mode 0: M_phi / dx^2; phi_mode 1: -L_phi
    float ax, ay;      // v_x / (2 dx), v_y / (2 dx)
    float cD;          // D_rho / dx^2
    float rho_top;     // reservoir ghost value above the top row
    float dt;          // time step
    int wait_cap;      // polls of a bounded TMA wait before it reports a timeout
};

enum MobKind { MOB_UNIFORM = 0, MOB_BULK = 1, MOB_SURF = 2 };


// Output tile of the fused step kernel (4-cell halo staged around it): 56 columns
// by tile_height(kind) rows; TILE_SMALL gives small grids many CTAs.  TILE_LARGE_RING is the
// 56 x 24 tile walked by a persistent kernel that stages the next tile while computing one
// (it uses TILE_LARGE's tile table and tensor maps).
// TILE_LARGE_PERSIST (ensembles only) is one cooperative launch over many steps, with a bounded
// grid barrier between steps, on the same 56 x 24 tiles.
enum TileKind { TILE_SMALL = 0, TILE_LARGE = 1, TILE_MEDIUM = 2, TILE_LARGE_RING = 3, TILE_LARGE_PERSIST = 4 };
constexpr int NUM_TILE_KINDS = 5;
constexpr int NUM_TILE_TABLES = 3;  // tile tables: TILE_SMALL, TILE_LARGE, TILE_MEDIUM
int choose_tile(int nx, int ny);
int tile_width();
int tile_height(int tile);
int tile_table(int tile);  // the tile table (and tensor-map box) a tile kind uses

// Ensemble of independent runs stepped by one launch: per-run constants and the
// two buffers of its ping-pong pair; one table entry per output tile.
struct EnsRun {
    StepConst k;
    float* f[2][3];  // [buffer][phi, c, rho]
};
struct EnsTile {
    int run, x0, y0;
};
struct EnsMaps;
// One step of every run (tile kind `tile`).  maps (may be NULL): the current buffer's maps of every
// run, for TMA staging of the tiles inside their run's grid in x (short and large tiles); err: the
// word that records a TMA wait that ran out.
cudaError_t launch_ens_step(int tile, int phi_mode, int mob, const EnsTile* tiles, const EnsRun* runs, int ntiles,
                            int parity, cudaStream_t s, const EnsMaps* maps = nullptr, int* err = nullptr);
// nsteps steps of every run in one cooperative launch (TILE_LARGE tiles); clears *bar first.
cudaError_t launch_ens_persistent(int phi_mode, int mob, const EnsTile* tiles, const EnsRun* runs, int ntiles,
                                  int parity, int nsteps, unsigned* bar, int wait_cap, int* err, cudaStream_t s);

// TMA descriptors of the three fields of one state, box = 64 columns x (tile height + 8) rows.
struct StepMaps {
    CUtensorMap phi, c, rho;
};
// Tensor maps of one buffer of every run, passed by value with a launch (3 x 128 B per run): the
// most runs whose maps fit the 32,764-byte kernel-parameter space with room to spare.  Larger
// ensembles stage every tile per thread.
constexpr int ENS_TMA_MAX_RUNS = 80;
struct EnsMaps {
    StepMaps run[ENS_TMA_MAX_RUNS];
};
static_assert(sizeof(EnsMaps) + 64 <= 32764, "ensemble maps exceed the kernel-parameter space");
// Encode the maps for a state (false: the driver refused, use the cp.async staging).
bool make_step_maps(const float* phi, const float* c, const float* rho, int nx, int ny, int pitch, int tile,
                    StepMaps* out);
// The same with an explicit box height (rows) and the first interior tile's corner (x, y): false also
// when no tile of that geometry is interior (the maps would never be used).
bool make_maps_box(const float* phi, const float* c, const float* rho, int nx, int ny, int pitch, int box_rows,
                   int interior_x, int interior_y, StepMaps* out);

// Error-word bits set by kernels (bit 0: NaN/Inf seen by diagnostics).
constexpr int ERR_BIT_TIMEOUT = 2;  // a bounded wait for a TMA copy ran out

// Launch one fused step: (phi0, c0, rho0) -> (phi1, c1, rho1) with programmatic
// dependent launch enabled (the kernel waits for the previous grid before reading).
// maps (may be NULL) are the tensor maps of (phi0, c0, rho0): tiles are then
// staged by TMA; err receives ERR_BIT_TIMEOUT if a staging wait ran out.
cudaError_t launch_step(const StepConst& k, int tile, int phi_mode, int mob,
                        const float* phi0, const float* c0, const float* rho0,
                        float* phi1, float* c1, float* rho1, cudaStream_t s,
                        const StepMaps* maps = nullptr, int* err = nullptr);
size_t step_smem_bytes(int tile);
// Two explicit midpoint steps in one launch (48 x step2_tile_height() output tiles from a 64 x
// step2_box_rows() staged window; maps: box of step2_box_rows() rows, or NULL).
cudaError_t launch_step2(const StepConst& k, int phi_mode, int mob, const float* phi0, const float* c0,
                         const float* rho0, float* phi1, float* c1, float* rho1, cudaStream_t s,
                         const StepMaps* maps, int* err);
int step2_box_rows();
int step2_tile_width();
int step2_tile_height();
// One fused step by the persistent 56 x 24 tile loop (maps: those of TILE_LARGE, or NULL for
// per-thread staging only).
cudaError_t launch_step_ring(const StepConst& k, int phi_mode, int mob, const float* phi0, const float* c0,
                             const float* rho0, float* phi1, float* c1, float* rho1, cudaStream_t s,
                             const StepMaps* maps, int* err);
// One forward-Euler update u + k.dt R(u) (the adjoint's u* with k.dt = dt/2), small tile.
cudaError_t launch_euler(const StepConst& k, int phi_mode, int mob, const float* phi0, const float* c0,
                         const float* rho0, float* phi1, float* c1, float* rho1, cudaStream_t s);

// Diagnostics: per-block FP64 partials then a fixed-order final reduction over at
// most DIAG_MAX_BLOCKS blocks (8 per SM on 152 SMs).
constexpr int DIAG_MAX_BLOCKS = 1216;
struct DiagConst {
    int nx, ny, pitch;
    float Wc, Wf;
    double area;       // dx^2
    double hkf, hkc;   // kappa_phi / 2, kappa_c / 2
};
int diag_blocks(int nx, int ny);
// hist (may be NULL): {count, next record step, capacity} then capacity records of
// {step, sum c, sum phi, sum rho, F_h}; each call appends one record and advances
// the next-record step by step_stride.
cudaError_t launch_diag(const DiagConst& d, const float* phi, const float* c, const float* rho,
                        double* partials, int* err, double* out, long long* hist, long long step_stride,
                        cudaStream_t s);
// Reset the history bookkeeping and the error word of a workspace.
cudaError_t launch_reset(long long* hist, long long capacity, long long next_step, int* err, cudaStream_t s);

// Host-side folding of pf_params (shared by the single-run, ensemble and adjoint layers).
void velocity_of(const pf_params& p, double* vx, double* vy);
StepConst step_const_of(const pf_params& p, int nx, int ny, int pitch);
DiagConst diag_const_of(const pf_params& p, int nx, int ny, int pitch);
int mob_kind_of(const pf_params& p);

// Error reporting and size checks of the C-ABI layer (pf_api.cu): fail() records the
// thread-local text that pf_last_error() returns and passes the code through.
int fail(int code, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);
int check_sizes(int nx, int ny, int pitch);

// Accessors used by the hybrid driver (pf_hybrid.cu): the run fields of an ensemble
// (pf_ens.cu) and the shape and stream of a U-Net handle (pf_unet_api.cu).
int ens_runs(const pf_ens* e);
void ens_run_fields(const pf_ens* e, int run, float** phi, float** c, float** rho, int* nx, int* ny, int* pitch);
cudaStream_t ens_stream(const pf_ens* e);
void unet_shape(const pf_unet* u, int* batch, int* nx, int* ny);
cudaStream_t unet_stream(const pf_unet* u);

}  // namespace pf
