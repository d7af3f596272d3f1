/*
 * pf.h - C ABI of the GB300 (sm_103a) explicit phase-field PVD time step.
 *
 * The method (arXiv 2312.05410, Materials and Methods, "Phase-field modeling of
 * physical vapor deposition" and "Dataset"): three fields on a uniform 2D mesh,
 *   phi  order parameter, solid +1 / vapor -1,
 *   c    concentration of one species (conserved, Cahn-Hilliard),
 *   rho  vapor density (convection-diffusion with a deposition sink),
 * advanced by second-order central differences in space and the explicit
 * midpoint (two-stage Runge-Kutta) method in time.  Closures the paper defers to
 * another reference (free energy, switching function h, boundary conditions) are
 * fixed as documented on pf_params below.
 *
 * Memory: every field is a caller-owned FP32 device array of ny rows of nx
 * values, x fastest, with a row pitch of `pitch` floats (pitch >= nx, pitch a
 * multiple of 4, base address 16-byte aligned).  The library never allocates
 * device memory: scratch comes from a caller-owned workspace of
 * pf_workspace_size() bytes.  All launches go to the caller's CUDA stream; only
 * pf_diag() and pf_diag_history() synchronise it.
 *
 * Errors: every int-returning call returns PF_OK (0) or a negative PF_ERR_*
 * code; pf_last_error() gives a message for the calling thread.  No call
 * throws across the ABI.
 */
#ifndef PF_H
#define PF_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PF_OK             0
#define PF_ERR_ARG       -1  /* bad argument (null pointer, size, mode)            */
#define PF_ERR_LAYOUT    -2  /* pitch / alignment / workspace too small            */
#define PF_ERR_UNSTABLE  -3  /* dt above the explicit stability limit              */
#define PF_ERR_NONFINITE -4  /* NaN or Inf seen in a field by a diagnostic pass    */
#define PF_ERR_TIMEOUT   -5  /* a bounded device wait ran out                      */
#define PF_ERR_CUDA      -6  /* a CUDA runtime call failed                         */

/*
 * Model parameters (host, FP64; the device computes in FP32).
 *
 *  dx, dt            mesh spacing and time step; dt must not exceed pf_dt_limit().
 *  W_c, W_phi        well heights of the bulk free energy
 *                    f(phi,c) = W_phi/4 (1-phi^2)^2 + p(phi) W_c c^2 (1-c)^2,
 *                    p(phi) = 1/4 (2-phi)(1+phi)^2 (the paper's M^Bulk prefactor).
 *  kappa_c, kappa_phi  gradient-energy coefficients (kappa/2 |grad u|^2).
 *  MA_bulk, MB_bulk, MA_surf, MB_surf, sigma_surf
 *                    composition mobility M_c = p(phi)(h MA_b + (1-h) MB_b)
 *                      + exp(-(phi/sigma)^2)(h MA_s + (1-h) MB_s), h = c^2 (3-2c)
 *                    (the paper's M^Bulk and M^Surf; its self-referencing
 *                    "- M^Surf" term is dropped).
 *  M_phi             constant mobility of the conserved phi equation (phi_mode 0).
 *  L_phi             relaxation rate of the Allen-Cahn variant (phi_mode 1).
 *  D_rho             vapor diffusivity.
 *  v_mag, v_angle_deg  incident vapor velocity v = v_mag (cos a, -sin a), angle a
 *                    from the substrate (90 = normal incidence).
 *  rho_top           vapor reservoir value held in the ghost row above the top.
 *  phi_mode          0: dphi/dt = div(M_phi grad dF/dphi) + S (the paper's
 *                    Cahn-Hilliard form with source); 1: dphi/dt = -L_phi dF/dphi + S.
 *  deposition        0 switches the incident flux off (v = 0, S = 0).
 *  diag_every        0: no periodic diagnostics; k > 0: pf_step records
 *                    {sum c, sum phi, sum rho, F_h} of every state whose step
 *                    index is a multiple of k (step 0 included).
 * Boundaries: x periodic; bottom row mirror for all fields; top row mirror for
 * phi and c (and both chemical potentials), reservoir value rho_top for rho.
 */
typedef struct pf_params {
    double dx, dt;
    double W_c, W_phi, kappa_c, kappa_phi;
    double MA_bulk, MB_bulk, MA_surf, MB_surf, sigma_surf;
    double M_phi, L_phi, D_rho, v_mag, v_angle_deg, rho_top;
    int phi_mode, deposition, diag_every;
} pf_params;

typedef struct pf_handle pf_handle;

/*
 * Explicit stability limit of the midpoint method for these parameters
 * ("Dataset": explicit midpoint integration).  out[0] = min(out[1..3]);
 * out[1] composition, out[2] order parameter, out[3] vapor (largest dt with
 * |1 + z + z^2/2| <= 1 over a fixed 513 x 257 lattice of wave numbers).
 * Host only; returns PF_ERR_ARG on a null pointer or non-positive dx.
 */
int pf_dt_limit(const pf_params* p, double out[4]);

/* Bytes of caller-owned device workspace pf_init() needs for an nx x ny grid
 * with the given row pitch (ping-pong state, reduction partials, diagnostic
 * history of `history_rows` records, error word). 0 on bad sizes. */
size_t pf_workspace_size(int nx, int ny, int pitch, int history_rows);

/*
 * Bind a simulation to caller-owned device fields and workspace.
 *  phi, c, rho   device FP32 fields (state at step 0), ny rows, row pitch `pitch`.
 *  work          device workspace of at least pf_workspace_size(nx, ny, pitch,
 *                history_rows) bytes, 256-byte aligned; contents undefined on entry.
 *  stream        cudaStream_t (NULL = legacy default stream) for every launch.
 * Validates the parameters (PF_ERR_ARG), the layout (PF_ERR_LAYOUT) and
 * dt <= pf_dt_limit() (PF_ERR_UNSTABLE) before touching the device; then one
 * tiny kernel resets the workspace's history counter and error word.  The
 * fields are not read.  The caller keeps ownership of every buffer; the handle
 * holds pointers only.
 */
int pf_init(const pf_params* p, int nx, int ny, int pitch,
            float* phi, float* c, float* rho,
            void* work, size_t work_bytes, int history_rows,
            void* stream, pf_handle** out);

/*
 * Advance n >= 0 explicit midpoint steps (all rows of the method: Laplacians,
 * chemical potentials, mobility, conserved flux divergences, Allen-Cahn
 * variant, deposition source, vapor transport, two RK stages) with one fused
 * kernel launch per step.  Asynchronous on the bound stream; when the stream
 * reaches the end of the call, phi, c and rho hold the state at step
 * (step0 + n).  Long runs replay a captured CUDA graph of whole step blocks.
 */
int pf_step(pf_handle* h, long n);

/* Diagnostics of the current state: out = {dx^2 sum c, dx^2 sum phi,
 * dx^2 sum rho, F_h} with the discrete free energy F_h = dx^2 sum f +
 * kappa_phi/2 sum_faces (dphi)^2 + kappa_c/2 sum_faces (dc)^2.  Per-cell terms
 * in FP32, accumulation in FP64 in a fixed order (deterministic).  Synchronises
 * the stream.  Returns PF_ERR_NONFINITE if any diagnostic pass so far saw a
 * NaN or Inf (the error word is sticky until pf_clear_error). */
int pf_diag(pf_handle* h, double out[4]);

/* Copy up to max_rows recorded diagnostic records (step, sum c, sum phi,
 * sum rho, F_h as 5 doubles each, oldest first) to host memory `out`;
 * *rows receives the count.  Synchronises the stream. */
int pf_diag_history(pf_handle* h, double* out, int max_rows, int* rows);

/* Step counter of the bound state (starts at 0; pf_set_step is for resuming
 * from a checkpoint, so that periodic diagnostics keep their phase). */
long pf_get_step(const pf_handle* h);
int pf_set_step(pf_handle* h, long step);

/* Polls a step kernel spends waiting for its TMA copies before it gives up
 * (default 2^22, a few milliseconds; a copy lands in about a microsecond).  On a
 * timeout the kernel sets the error word, lets the copies in flight land, leaves
 * its tile unwritten and returns; pf_diag then reports PF_ERR_TIMEOUT.  A limit
 * of 0 makes every wait give up at once, to exercise that path. */
int pf_set_wait_limit(pf_handle* h, int polls);

/* 1 when tiles are staged by TMA (tensor maps encoded at pf_init; grids with at least
 * one interior tile: nx >= 116 and ny >= 20 up to 2^20 cells, ny >= 52 above): every
 * tile whose window lies inside the grid in x, the bottom and top tiles included (their
 * ghost rows are set in shared memory after the copy), and in grids whose width is a
 * multiple of 4 the tiles that wrap in x (the last tile column starts at nx - 56, and
 * the 4 wrapped columns are set after the copy); other wrapping tiles use per-thread
 * copies.  0 when every tile uses per-thread asynchronous copies (smaller
 * grids, or a driver without tensor-map support); -1 on NULL. */
int pf_staging_mode(const pf_handle* h);

/* Steps per kernel launch: 1 (the default), or 2: a CTA stages a 64 x (TY + 16) window
 * of the state once and runs both explicit midpoint steps on it in shared memory, writing
 * 48 x TY cells of u^{n+2}.  Two steps are taken in one launch only where no diagnostic
 * record falls between them (an even diag_every reached from an even step, or no
 * diagnostics).  Both settings give identical results; on GB300 two per launch measured
 * the same time per step at 512^2 and more at 64^2.  Returns the previous setting, or
 * PF_ERR_ARG. */
int pf_set_steps_per_launch(pf_handle* h, int steps);

/* Grids above 2^20 cells (56 x 24 tiles): on = 1 steps them with a persistent kernel
 * in which every resident CTA walks a share of the tiles and stages the next tile (TMA
 * for interior tiles) while it computes the current one's second stage; on = 0 (the
 * default) launches one CTA per tile, which measured faster on GB300.  Both give
 * identical results.  Returns the previous setting (0 or 1), or PF_ERR_ARG for a
 * smaller grid or a null handle. */
int pf_set_tile_loop(pf_handle* h, int on);

/*
 * Host-buffer state transfer (the end-to-end path of a caller whose fields live in
 * host memory): pf_load_host copies host arrays phi, c, rho (ny rows of nx floats,
 * row pitch host_pitch >= nx floats) into the handle's current state; pf_store_host
 * copies the current state out to such arrays.  Asynchronous on the handle's stream
 * (use page-locked host memory for a copy that overlaps; the host arrays must stay
 * valid until the stream reaches the copy).  Call them between pf_step calls.
 * Nothing is allocated.  PF_ERR_ARG on a null pointer, PF_ERR_LAYOUT on a pitch below nx.
 */
int pf_load_host(pf_handle* h, const float* phi, const float* c, const float* rho, int host_pitch);
int pf_store_host(pf_handle* h, float* phi, float* c, float* rho, int host_pitch);

/* Clear the sticky device error word (async). */
int pf_clear_error(pf_handle* h);

/* Release the handle (no device memory is freed: the caller owns it).
 * Synchronises the stream first. */
int pf_destroy(pf_handle* h);

/*
 * Diagnostics of arbitrary fields without a handle: writes the 4 doubles of
 * pf_diag() to the DEVICE pointer out_dev (8-byte aligned), asynchronously on
 * `stream`.  work: device scratch of pf_diag_workspace_size(nx, ny) bytes
 * (per-block FP64 partials and the error word), caller-owned.  A NaN or Inf in
 * any field sets bit 0 of the int at work + pf_diag_error_offset(nx, ny).
 */
size_t pf_diag_workspace_size(int nx, int ny);
size_t pf_diag_error_offset(int nx, int ny);
int pf_diagnostics(const pf_params* p, int nx, int ny, int pitch,
                   const float* phi, const float* c, const float* rho,
                   void* work, size_t work_bytes, double* out_dev, void* stream);

/*
 * pf_diagnostics without a workspace, for callers that must not allocate
 * device memory themselves (for example a plug-in inside an application that
 * owns all device memory through its own pool, or a latency-critical loop in
 * which cudaMalloc/cudaFree would synchronise the device).  The paper has no
 * counterpart: this is a packaging variant of the diagnostics above.
 *
 * Same inputs and the same 4 doubles written to out_dev (device, 8-byte
 * aligned) as pf_diagnostics.  If err_dev (device int) is not NULL it receives
 * 1 when a field holds a NaN or Inf, else 0.  The reduction scratch is one
 * static device array of 1216 x 4 doubles plus an error word (about 39 KB)
 * that every GPU loading the library keeps until the process exits; any grid
 * the library accepts (sides up to 2^20) fits in it, other sizes are rejected
 * with PF_ERR_ARG / PF_ERR_LAYOUT (pf_last_error() gives the reason).  The
 * array's device address is looked up on every call made outside a stream
 * capture and remembered per device and CUDA context; a call made while
 * `stream` is being captured reuses the remembered address, so make the first
 * call on each device, and the first after a cudaDeviceReset, before any
 * stream capture.  All calls share the array: calls that can overlap on the
 * GPU (unordered streams) race.  Nothing is allocated.
 * Returns PF_OK or a PF_ERR_* code; asynchronous on `stream`.
 */
int pf_diagnostics_static(const pf_params* p, int nx, int ny, int pitch,
                          const float* phi, const float* c, const float* rho,
                          double* out_dev, int* err_dev, void* stream);

/*
 * Ensemble: nruns independent runs (uneven grid sizes, per-run parameters; the
 * paper's dataset is such a sweep over deposition rate, angle and mobilities,
 * "Dataset") advanced in lockstep.  Every step of every run is ONE launch of
 * the fused step kernel over a table of tiles of all runs; long stretches are
 * replays of a captured CUDA graph.  All runs must share phi_mode and the
 * mobility form (uniform / bulk / bulk + surface); their coefficients, dt,
 * velocity, sizes and pitches may differ.  diag_every is ignored.
 *
 * pf_ens_workspace_size: bytes of caller-owned device workspace (ping-pong
 *   partner of every run, run and tile tables, reduction scratch); 0 on bad sizes.
 * pf_ens_init: phi[r], c[r], rho[r] are run r's caller-owned device fields
 *   (layout as for pf_init); work is 256-byte aligned.  Errors as pf_init.
 * pf_ens_step: advance every run n steps (async on the stream); the caller's
 *   fields hold the new states when the stream reaches the end of the call.
 * pf_ens_autotune: time trial_steps (even, >= 2) steps with each tile kind the
 *   ensemble can run and keep the fastest; these are real steps of the simulation
 *   (trial_steps + 2 per kind tried).  chosen (may be NULL) receives the tile kind,
 *   seconds_per_step (may be NULL, 5 doubles) the timings (0 for a kind not tried).
 *   Synchronises.
 * pf_ens_set_tile / pf_ens_get_tile: tile kind 0 (56x8), 1 (56x24), 2 (56x16),
 *   3: 56x24 tiles walked by a persistent kernel (one CTA per resident slot) that
 *   stages the next tile while it computes one, or 4: one cooperative launch that
 *   advances every run through up to 100 steps (a graph replay holds one such launch),
 *   its resident CTAs walking the 56x24 tiles of a step and meeting at a grid-wide
 *   barrier (a counter in the workspace, bounded polls) between steps; kind 4 needs
 *   every run's nx to be a multiple of 4 (PF_ERR_ARG otherwise).  All kinds give
 *   identical results.
 * pf_ens_set_wait_limit: polls of kind 4's barrier wait, and of the TMA staging wait
 *   of kinds 0 and 1, before it reports a timeout (default 2^22); a wait that runs out
 *   makes pf_ens_diag return PF_ERR_TIMEOUT.  Updates the device run table on the
 *   stream and synchronises; PF_ERR_ARG on NULL or polls < 0.
 * pf_ens_set_tma: 1 (the default) stages the tiles of kinds 0 and 1 by TMA: the tiles
 *   inside their run's grid in x, and in runs whose width is a multiple of 4 also the
 *   tiles that wrap in x (the last tile column starts at nx - 56); every run's tensor
 *   maps travel with the launch as a kernel parameter (ensembles of up to 80 runs; maps
 *   encoded at pf_ens_init).  0: per-thread copies for every tile.  Identical results.
 *   Returns PF_OK, or PF_ERR_ARG on NULL.
 * pf_ens_staging_mode: 1 if the current tile kind stages by TMA, 0 if not, -1 on NULL.
 * pf_ens_diag: pf_diag of run `run` (synchronises).
 */
typedef struct pf_ens pf_ens;
size_t pf_ens_workspace_size(int nruns, const int* nx, const int* ny, const int* pitch);
int pf_ens_init(int nruns, const pf_params* params, const int* nx, const int* ny, const int* pitch,
                float* const* phi, float* const* c, float* const* rho,
                void* work, size_t work_bytes, void* stream, pf_ens** out);
int pf_ens_step(pf_ens* e, long n);
int pf_ens_autotune(pf_ens* e, int trial_steps, int* chosen, double* seconds_per_step);
int pf_ens_set_tile(pf_ens* e, int tile);
int pf_ens_set_wait_limit(pf_ens* e, int polls);
int pf_ens_set_tma(pf_ens* e, int on);
int pf_ens_staging_mode(const pf_ens* e);
int pf_ens_get_tile(const pf_ens* e);
long pf_ens_get_step(const pf_ens* e);
int pf_ens_diag(pf_ens* e, int run, double out[4]);
int pf_ens_destroy(pf_ens* e);
const char* pf_ens_last_error(void);

/*
 * Discrete adjoint of the explicit midpoint step (the paper's inverse-design
 * motivation, Discussion: finding deposition parameters for a target
 * microstructure).  Runs nsteps forward steps from (phi0, c0, rho0), storing a
 * checkpoint every K steps, then the hand-written adjoint backwards through
 * them (each segment recomputed from its checkpoint).  It returns the exact
 * gradient of the linear functional L = sum(w_phi*phi_N + w_c*c_N + w_rho*rho_N)
 * of the final state (w = dLoss/du_N for any loss of u_N):
 *   g_phi0, g_c0, g_rho0  dL/d(initial fields), device, layout of the fields;
 *   g_params (host, 3)    {dL/dv_mag, dL/ds with M_c -> s M_c at s = 1, dL/dkappa_c};
 * dt is held fixed.  w_rho may be NULL (zero).  final_* (device, may all be
 * NULL) receive u_N.  work: pf_adjoint_workspace_size(nx, ny, pitch, nsteps, K)
 * bytes, 256-byte aligned (two work states, nsteps/K + 1 checkpoints, K segment
 * states, cotangents, scratch).  Synchronises the stream.  Per-cell terms are
 * FP32; the parameter sums are FP64 in a fixed order.
 */
size_t pf_adjoint_workspace_size(int nx, int ny, int pitch, long nsteps, int K);
int pf_adjoint(const pf_params* p, int nx, int ny, int pitch,
               const float* phi0, const float* c0, const float* rho0, long nsteps, int K,
               const float* w_phi, const float* w_c, const float* w_rho,
               float* g_phi0, float* g_c0, float* g_rho0, double* g_params,
               float* final_phi, float* final_c, float* final_rho,
               void* work, size_t work_bytes, void* stream);
const char* pf_adjoint_last_error(void);

/* Text for an error code, and the last error message of the calling thread. */
/*
 * Tensor-core convolution primitives of the U-Net surrogate ("U-Net with temporal
 * conditioning", Methods: the convolution of each conv_block and the transposed
 * convolution of the up-sampling path), as implicit GEMMs on tcgen05 with BF16
 * operands and FP32 accumulation in tensor memory.
 *
 * pf_conv3x3_bf16: out[n][y][x][out_coff + co] = BF16( sum_{ky,kx,ci} in[n][y+ky-1][x+kx-1][ci]
 *   * wgt[3 ky + kx][co][ci] ), zero outside the image (the paper's conv with 'same'
 *   zero padding, no bias).  in: device BF16 NHWC [n][h][w][cin]; wgt: device BF16
 *   [9][cout][cin]; out: device BF16 NHWC buffer of out_cstride channels per pixel,
 *   of which [out_coff, out_coff + cout) are written.  partials (device, may be NULL):
 *   the group-normalisation statistics of the FP32 results over `groups` equal
 *   channel groups, as FP32 [n][groups][h*w/128][4][2]: the sum and the sum of
 *   squares over each quarter (32 pixels) of each 128-pixel tile.
 * pf_tconv2x2_bf16: out[n][2y+dy][2x+dx][out_coff + co] = BF16( sum_ci in[n][y][x][ci]
 *   * wgt[(2 dy + dx) cout + co][ci] ) (stride-2 2x2 transposed convolution, no bias);
 *   out is n x 2h x 2w pixels.
 * Shapes: cin % 32 == 0 (<= 1024); conv: cout in {32, 64, 128, 256} with groups
 * = 8 (the U-Net's widths); transposed conv: cout in {16, 32, 64, 128}; h*w % 128
 * == 0 and w a multiple or a divisor of 128; n h w < 2^27 (2^20 tiles of 128 pixels); pointers
 * 16-byte aligned; out_coff and out_cstride multiples of 8.  err_dev: device int;
 * bit 1 is set if a bounded pipeline wait ran out (the kernel then stops early).
 * Asynchronous on `stream`; PF_ERR_ARG / PF_ERR_LAYOUT / PF_ERR_CUDA on errors, with
 * the text in pf_unet_last_error().  Nothing is allocated.
 */
int pf_conv3x3_bf16(const void* in, int n, int h, int w, int cin, const void* wgt, int cout, void* out,
                    int out_cstride, int out_coff, int groups, float* partials, int* err_dev, void* stream);
int pf_tconv2x2_bf16(const void* in, int n, int h, int w, int cin, const void* wgt, int cout, void* out,
                     int out_cstride, int out_coff, int* err_dev, void* stream);
/*
 * pf_conv_halo: selects how pf_conv3x3_bf16 (and the U-Net's convolutions) stage a tile
 * with cin == 64, cout <= 64 and w a multiple of 128.  on = 1 (the default): one copy of
 * the tile's three input rows of 130 pixels serves all nine taps, and the weights of
 * all taps stay in shared memory.  on = 0: one copy per tap, like every other shape.
 * Both give the same sums.  A process-wide setting (not thread-safe against
 * concurrent launches); returns the previous setting.
 */
int pf_conv_halo(int on);
/*
 * The time-conditioned U-Net surrogate and its jump ("U-Net with temporal
 * conditioning", Methods; the hybrid solver of Results alternates DNS stretches
 * with such jumps).  For each of `batch` runs it maps the state at time t, with
 * look-back frames before t, to a prediction at t + dt.  Structure:
 *   - input planes: lb = 3 frames of (phi, c, rho), oldest first (the paper's
 *     operator reads lb = 3 consecutive frames of its field), then tau = dt / dt_ref;
 *     the two older frames are the ones pushed with pf_unet_frame, the newest is
 *     the fields being advanced;
 *   - encoder z1 = block(x), zp = block(down(z_{p-1})), with block = GELU(GN(conv3x3));
 *   - conditioning zc_p = z_p * (W_p f(tau)), where f is the sin MLP;
 *   - decoder d3 = up(block(zc4)), d2 = up(block(zc3 ++ d3)), d1 = up(block(zc2 ++ d2));
 *   - output (phi, c, rho) += gamma * conv3x3(block(zc1 ++ d1)) + beta, a
 *     per-channel affine increment of the newest frame.  The paper predicts its one
 *     normalised composition field and applies a final group normalisation.  Here:
 *     - the state is the three coupled fields, whose per-sample mean and spread vary
 *       with film thickness and incident composition, so the increment form is used;
 *     - the vapor density is predicted as well, because resetting it after each jump
 *       instead costs 12.6% relative L2 in phi over 25 exact jumps.
 * Channels are 32-64-128-256, with 8 groups in the hidden normalisations.  Weights and activations are stored as BF16 and
 * accumulated in FP32; the 3x3 and transposed convolutions of levels 2-4, of
 * the decoder and of the output layer run on the tensor cores (the kernels of
 * pf_conv3x3_bf16 / pf_tconv2x2_bf16; the output layer as a 16-column tile whose
 * epilogue adds the affine increment to the fields); the first convolution, the
 * normalisations (GELU through the hardware tanh) and the MLP run on the CUDA cores.
 *
 * pf_unet_workspace_size: bytes of caller-owned device workspace (weights in
 *   device layouts, all activations, statistics, tables); 0 if the shape is
 *   unsupported.  Supported shapes: sides >= 128 and multiples of 8, nx/8 dividing
 *   or a multiple of 128, (nx/8)(ny/8) a multiple of 128 (e.g. 128^2, 256^2, 512^2),
 *   and batch nx ny < 2^27.
 * pf_unet_init: weights = 40 host FP32 arrays, in PyTorch layouts and this order:
 *   0-5   mlp_w0 [128][1], mlp_b0 [128], mlp_w1 [128][128], mlp_b1, mlp_w2 [128][128], mlp_b2
 *   6-9   proj1..proj4 [C_p][128] (C = 32, 64, 128, 256)
 *   10-13 enc1 [32][10][3][3], enc2 [64][32][3][3], enc3 [128][64][3][3], enc4 [256][128][3][3]
 *         (enc1's input planes: frames oldest first, (phi, c, rho) each, then tau)
 *   14-17 dec4 [256][256][3][3], dec3 [128][256][3][3], dec2 [64][128][3][3], dec1 [32][64][3][3]
 *   18-20 up4 [256][128][2][2], up3 [128][64][2][2], up2 [64][32][2][2]  ([Cin][Cout][dy][dx])
 *   21    out [3][32][3][3]
 *   22-39 (gamma, beta) of enc1..enc4, dec4..dec1 (group normalisation) and of out
 *   (the output affine).  Convolution weights are rounded to BF16; the MLP and
 *   projections are kept in FP64 and the affine parameters in FP32.  Everything is
 *   copied into the workspace (synchronises once).
 *   work: 256-byte aligned.
 * pf_unet_frame: push the current fields of every run (same arguments as the jump's)
 *   as the newest look-back frame, rounded to BF16 into the workspace; the handle keeps
 *   the two newest pushed frames.  One kernel launch, asynchronous.
 * pf_unet_reset_frames: forget the pushed frames (host only).  A jump made with fewer
 *   than two frames held takes the oldest frame held, or the current fields when none
 *   is, in place of the missing ones.
 * pf_unet_jump: advances (phi[i], c[i], rho[i]) of runs i < n (n == batch; device
 *   FP32 fields ny x nx with row pitch `pitch` floats) in place by the predicted
 *   increments for jump length tau, the pushed frames being its look-back.
 *   Asynchronous on the handle's stream, 28 kernel launches (29 when tau differs
 *   from the previous jump's: the MLP basis).  The pushed frames are kept.
 * pf_unet_sync: synchronise; PF_ERR_TIMEOUT if a tensor-core pipeline wait ran out.
 * pf_unet_check: plausibility of the last jump's prediction, the hybrid solver's
 *   gate for its plain-DNS fallback.  ok[i] (host, n ints) is 1 if every phi, c and
 *   rho of run i is finite and inside its range, else 0.  Synchronises.
 * pf_unet_buffer: device pointer and channel count of activation buffer `which`
 *   (0-14: pre1, cat1, p1, pre2, cat2, p2, pre3, cat3, p3, pre4, zc4, h4, h3, h2,
 *   h1; NHWC BF16 at level resolution), for inspection.
 */
typedef struct pf_unet pf_unet;
size_t pf_unet_workspace_size(int batch, int nx, int ny);
int pf_unet_init(const float* const* weights, int nweights, int batch, int nx, int ny, void* work, size_t work_bytes,
                 void* stream, pf_unet** out);
int pf_unet_frame(pf_unet* u, int n, const float* const* phi, const float* const* c, const float* const* rho,
                  int pitch);
int pf_unet_reset_frames(pf_unet* u);
int pf_unet_jump(pf_unet* u, int n, float* const* phi, float* const* c, float* const* rho, int pitch, double tau);
int pf_unet_sync(pf_unet* u);
int pf_unet_check(pf_unet* u, double phi_lo, double phi_hi, double c_lo, double c_hi, double rho_lo, double rho_hi,
                  int* ok);
int pf_unet_buffer(const pf_unet* u, int which, void** ptr, int* channels);
int pf_unet_destroy(pf_unet* u);
const char* pf_unet_last_error(void);

/*
 * The hybrid DNS / U-Net solver ("Hybrid" in Results: stretches of direct
 * simulation alternate with leaps of the neural operator over the time the DNS
 * would have taken).  Every run of ensemble `e` must have the U-Net's grid
 * (batch = number of runs, one row pitch for all), and both handles must use the
 * same stream.  pf_hybrid_run advances every run `total_steps` steps: first
 * `dns_lead` DNS steps (the paper starts its hybrid with the solver alone; the
 * deposited film's early growth amplifies a perturbation most), then cycles of
 *   1. `dns_stretch` DNS steps (pf_ens_step), pushing the state as a look-back frame
 *      (pf_unet_frame) 2 frame_every and frame_every steps before the stretch ends;
 *   2. a backup of every run's state, then one jump (pf_unet_jump) standing for
 *      `jump_steps` steps, with tau = jump_steps / dt_ref_steps;
 *   3. the plausibility gate (pf_unet_check with the given ranges; synchronises):
 *      if any run fails, every run is restored and the jumped steps are run by DNS.
 * The steps left after the last whole cycle are run by DNS.  stats receives the
 * jumps kept, the fallbacks and the DNS steps taken.  work: caller-owned device
 * scratch of pf_hybrid_workspace_size(e) bytes (the backup), 256-byte aligned.
 * Returns PF_OK or a PF_ERR_* code, with the text in pf_hybrid_last_error();
 * PF_ERR_TIMEOUT if a tensor-core pipeline wait of a jump ran out.
 */
typedef struct pf_hybrid_params {
    long dns_stretch;     /* DNS steps before each jump, >= 2 frame_every */
    long jump_steps;      /* steps one jump stands for */
    long frame_every;     /* steps between the look-back frames */
    double dt_ref_steps;  /* the network's time unit in steps */
    double phi_lo, phi_hi, c_lo, c_hi, rho_lo, rho_hi;  /* plausible ranges of a prediction */
    long dns_lead;        /* DNS steps before the first cycle, >= 0 (part of total_steps) */
} pf_hybrid_params;
typedef struct pf_hybrid_stats {
    long jumps, fallbacks, dns_steps;
} pf_hybrid_stats;
size_t pf_hybrid_workspace_size(const pf_ens* e);
int pf_hybrid_run(pf_ens* e, pf_unet* u, const pf_hybrid_params* hp, long total_steps, void* work, size_t work_bytes,
                  pf_hybrid_stats* stats);
const char* pf_hybrid_last_error(void);

/*
 * Two-point autocorrelation of the solid A phase ("Autocorrelations", Results; the
 * hybrid solver's error metric, "Error metrics", Methods): with I(x) = 1 where
 * phi > 0 and c > 0.5 (FP32 comparisons), counts[ry + R][rx + R] = sum_x I(x) I(x + r)
 * over periodic shifts r = (rx, ry), |rx|, |ry| <= R; S2(r) = counts / (nx ny).
 * phi, c: device FP32 fields with row pitch `pitch`; scratch: device, nx*ny bytes;
 * counts: device int64 [(2R+1)^2].  R <= 127 and 2R+1 <= min(nx, ny).  Integer
 * arithmetic (exact).  Asynchronous on `stream`; PF_ERR_ARG / PF_ERR_CUDA.
 */
int pf_s2_counts(const float* phi, const float* c, int nx, int ny, int pitch, int R, unsigned char* scratch,
                 long long* counts, void* stream);

const char* pf_strerror(int code);
const char* pf_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PF_H */
