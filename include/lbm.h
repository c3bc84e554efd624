/*
 * lbm.h -- C ABI of the B300 library for the fused lattice-Boltzmann LES step
 * with the Tau-orthogonal (TO) subgrid-scale forcing of "Reduced Subgrid-Scale
 * Terms for Turbulence Simulations with the Lattice Boltzmann Method".
 *
 * One time step (Sec. 3, Eqs. LES-1..3 with the predictor-corrector of Sec. 4):
 *   stream (pull, periodic x/z, halfway bounce-back walls in y)
 *   -> moments -> effective relaxation time (Smagorinsky or WALE, Sec. 5)
 *   -> BGK relaxation (Eq. LES-1) + body force (exact-difference method, Eq.
 *      collide-and-stream; or Guo's scheme) giving the predictor f^{p*}
 *   -> QoIs, sensitivities and Gram matrix on v^{p*} (Sec. 4.1-4.2, App. A)
 *   -> dQ from the coefficient source (Eq. LRS, Eq. dQ-from-ref, or random gamma)
 *   -> pattern solve and dv_SGS = sum gamma_i O_i (Eqs. TO-ansatz, O-from-V,
 *      tau-from-dQ) applied as an equilibrium difference (Eq. LES-2).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Every function returns an lbm_status; nothing aborts, prints or traps.
 *   After a non-OK status, lbm_last_error() gives a one-line reason.
 * - Memory ownership: the CALLER owns all device memory and streams.  The
 *   library asks for a byte count (lbm_required_bytes), the caller allocates
 *   one device buffer of at least that size (256-byte aligned) and passes it
 *   to lbm_create together with a CUDA stream; every device array lives in
 *   that buffer and the library never frees it.  lbm_destroy frees only the
 *   library's host-side state (and its CUDA graph / events).
 * - Host pointers passed in are read during the call only; the library keeps
 *   no caller pointer except the device buffer and the stream.
 * - Grid layout: node index n = (z*ny + y)*nx + x, x fastest.  2-D runs use
 *   nz = 1.  A velocity field is [3][nz][ny][nx] (component-major); the z
 *   component of 2-D runs is zero.  Populations are [Q][nz][ny][nx] with the
 *   population order below.
 * - With walls (wall flag 1) rows y = 0 and y = ny-1 are solid; the walls
 *   sit half a cell inside them.  Solid rows are never collided; their
 *   density reads back as 1 and their velocity as 0.
 *
 * Population order (Q = 9 in 2-D, Q = 19 in 3-D):
 *   D2Q9 : rest, +x, +y, -x, -y, (+x+y), (-x+y), (-x-y), (+x-y)
 *   D3Q19: rest, +x, -x, +y, -y, +z, -z, (+x+y), (-x-y), (+x-y), (-x+y),
 *          (+x+z), (-x-z), (+x-z), (-x+z), (+y+z), (-y-z), (+y-z), (-y+z)
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LBM_OK = 0,
    LBM_ERR_ARG = 1,            /* invalid argument or configuration            */
    LBM_ERR_BUDGET = 2,         /* buffer too small / batch memory budget full  */
    LBM_ERR_CUDA = 3,           /* a CUDA runtime call failed                   */
    LBM_ERR_UNSTABLE = 4,       /* non-finite state, rho <= 0 or |v| > c_s      */
    LBM_ERR_SINGULAR_GRAM = 5,  /* reported through QoI flags, not as a status  */
    LBM_ERR_TIMEOUT = 6,        /* a kernel's bounded wait on its bulk copies gave up */
    LBM_ERR_STATE = 7           /* call not valid in the current state          */
} lbm_status;

enum { LBM_FORCING_EDM = 0, LBM_FORCING_GUO = 1 };
enum { LBM_SUBSTRATE_NONE = 0, LBM_SUBSTRATE_SMAG = 1, LBM_SUBSTRATE_WALE = 2 };
/* Populations are always stored shifted, as g_i = f_i - w_i. */
enum { LBM_STORAGE_FP32 = 0, LBM_STORAGE_FP16 = 1, LBM_STORAGE_BF16 = 2 };
enum { LBM_QOI_ENERGY = 0, LBM_QOI_ENSTROPHY = 1 };
enum { LBM_FILTER_GAUSS = 0, LBM_FILTER_LAPLACE = 1, LBM_FILTER_BINOMIAL = 2,
       LBM_FILTER_FOURIER = 3 /* sharp band l - 1/2 <= |k| < m + 1/2; periodic 2-D, nx = ny */ };
enum {
    LBM_TO_OFF = 0,      /* substrate-only LES, no QoIs                              */
    LBM_TO_OBSERVE = 1,  /* QoIs and Gram on the predictor, no forcing (dQ = 0)      */
    LBM_TO_GAMMA = 2,    /* gamma_i = gamma_std * z_i, z Philox normals per step     */
    LBM_TO_LRS = 3,      /* online TO-LRS: dQ = LRS(q_h) - q^{n*} (Eq. LRS)         */
    LBM_TO_TRACK = 4,    /* dQ = Q_ref(t^n) - q^{n*} (Eq. dQ-from-ref)              */
    LBM_TO_FIXED_GAMMA = 5  /* gamma_i given by the caller (lbm_set_to_coeffs), held
                               for every step; dQ_i = gamma_i sum V_i . O_i          */
};

#define LBM_MAX_QOI 16   /* scale-aware QoIs + mean-profile bands */

/* QoI flags in the per-step QoI block */
#define LBM_FLAG_SINGULAR 1u  /* Gram pivot <= 1e-14 max diag: SGS skipped */
#define LBM_FLAG_UNSTABLE 2u  /* instability seen during this step        */

typedef struct {
    int32_t kind;    /* LBM_QOI_ENERGY or LBM_QOI_ENSTROPHY                      */
    int32_t filter;  /* LBM_FILTER_*                                               */
    int32_t scale;   /* s of G_s / L_s (odd, >= 1); ignored for binomial;
                        lower wavenumber bin l of a Fourier band                  */
    int32_t band_hi; /* upper wavenumber bin m of a Fourier band (else unused)    */
} lbm_qoi_spec;

typedef struct {
    int32_t dim;        /* 2 (D2Q9) or 3 (D3Q19)                                  */
    int32_t nx, ny, nz; /* lattice size; nz = 1 in 2-D                             */
    int32_t walls;      /* 1: halfway bounce-back walls in y, 0: periodic in y     */
    int32_t forcing;    /* LBM_FORCING_*                                           */
    int32_t substrate;  /* LBM_SUBSTRATE_*                                         */
    int32_t storage;    /* LBM_STORAGE_*                                           */
    double tau;         /* molecular relaxation time (nu = (tau - 1/2)/3)          */
    double body_force[3];  /* constant force density                           */
    double kolmo_amp;   /* force density kolmo_amp*sin(2 pi kolmo_k y/ny) along x  */
    double kolmo_drag;  /* linear drag: force density -kolmo_drag * rho u          */
    int32_t kolmo_k;
    int32_t to_mode;    /* LBM_TO_*                                                */
    double c_smag;      /* Smagorinsky constant                                    */
    double c_wale;      /* WALE constant                                           */
    int32_t n_qoi;      /* number of scale-aware QoIs in qoi[]                     */
    int32_t n_mp;       /* number of mean-profile bands (walls only)               */
    lbm_qoi_spec qoi[LBM_MAX_QOI];
    int32_t h;          /* LRS history length (LBM_TO_LRS)                         */
    int32_t qoi_ring;   /* device QoI ring capacity in rows (0: 4096)              */
    double gamma_std;   /* LBM_TO_GAMMA: std of the per-step gamma                 */
    uint64_t seed;      /* Philox key word 0                                       */
    uint64_t member;    /* Philox key word 1 (ensemble member id)                  */
    int64_t track_len;  /* LBM_TO_TRACK, or LBM_TO_LRS with spinup: reference rows held */
    int64_t spinup;     /* LBM_TO_LRS: the first spinup steps are nudged to the
                           reference series (dQ = Q_ref - q*, the reference enters
                           the histories), as online runs start after a tracked
                           spin-up; needs track_len >= 1 and sigma_ref > 0 */
} lbm_config;

typedef struct lbm_ctx lbm_ctx;

/* Length of one QoI block row: [step, q*[N], dQ[N], gamma[N], flags], N =
 * n_qoi + n_mp.  Values are doubles. */
int lbm_qoi_row_len(const lbm_config* cfg, int64_t* len);

/* Bytes of device memory lbm_create needs for this configuration.
 * ERR_ARG if the configuration is invalid (the text says why), including
 * grids with 6 nx ny nz >= 2^31 (node and field-component offsets are
 * 32-bit; population offsets are 64-bit, so a 171 M-node D3Q19 grid is
 * accepted). */
int lbm_required_bytes(const lbm_config* cfg, size_t* bytes);

/* Build a simulation inside the caller's device buffer.
 *   dev_buf      device pointer, 256-byte aligned, at least lbm_required_bytes
 *   bytes        its size (ERR_BUDGET if too small)
 *   cuda_stream  cudaStream_t on which all work is queued (NULL = legacy default)
 *   out          receives the handle
 * The state starts at rest (f = w); call lbm_init_macros or
 * lbm_set_populations next.  Device errors: ERR_CUDA. */
int lbm_create(const lbm_config* cfg, void* dev_buf, size_t bytes, void* cuda_stream, lbm_ctx** out);

/* Free host-side state.  Does not touch dev_buf.  Waits for queued work. */
int lbm_destroy(lbm_ctx* ctx);

/* Text of the last error on this context (NUL-terminated, truncated to len). */
int lbm_last_error(const lbm_ctx* ctx, char* buf, size_t len);

/* Set the state to f = f^eq(rho, u) from host FP64 arrays rho[nz][ny][nx]
 * (NULL: rho = 1) and u[3][nz][ny][nx].  Resets the step counter, the QoI
 * ring, the mean profile and the LRS histories.  Synchronous. */
int lbm_init_macros(lbm_ctx* ctx, const double* rho, const double* u);

/* Coefficient source of the TO forcing (Sec. 4.3-4.4).  Host FP64 inputs:
 *   C          [(2h+1)*N + 1][N] row-major LRS matrix; rows ordered as the
 *              input vector [q^{n-1..n-h}, q^{n*}, q^{n-1*..n-h*}, 1] (Eq. LRS)
 *   mu, Sigma  residual mean [N] and covariance [N][N] (scaled units);
 *              Sigma must be symmetric positive definite (ERR_ARG otherwise)
 *   sigma_ref  [N] per-QoI reference scales (> 0)
 *   q_hist, qs_hist  optional [h][N] initial histories, row k = q^{n-1-k}
 *              (NULL: zeros)
 * Only valid for LBM_TO_LRS.  Synchronous. */
int lbm_set_lrs(lbm_ctx* ctx, const double* C, const double* mu, const double* Sigma,
                const double* sigma_ref, const double* q_hist, const double* qs_hist);

/* Coefficient source of the TO forcing in one call (Sec. 4.3-4.4: the
 * coefficients gamma_i of Eq. TO-ansatz, from Eq. tau-from-dQ).
 *   mode        must equal cfg.to_mode of the context (ERR_STATE otherwise):
 *               the device arrays of each source are placed at lbm_create
 *   h           LRS history length; must equal cfg.h for LBM_TO_LRS, else ignored
 *   C, mu, Sigma, sigma_ref   LBM_TO_LRS only, as in lbm_set_lrs (zero initial
 *               histories); NULL for the other modes
 *   gamma_fixed [N] host FP64, N = n_qoi + n_mp: LBM_TO_FIXED_GAMMA only
 *               (required there, finite); every step then applies
 *               dv_SGS = sum_i gamma_i O_i and reports dQ_i = gamma_i sum V_i . O_i
 * LBM_TO_OFF, LBM_TO_OBSERVE, LBM_TO_GAMMA (gamma_std * Philox normals) and
 * LBM_TO_TRACK (lbm_set_track_reference) take no coefficients here: the call
 * only checks the mode.  Synchronous.  A context in LBM_TO_LRS or
 * LBM_TO_FIXED_GAMMA refuses lbm_step (ERR_STATE) until its coefficients are set.
 * Errors: ERR_ARG (NULL or invalid array, h mismatch, Sigma not SPD),
 * ERR_STATE (mode mismatch), ERR_CUDA. */
int lbm_set_to_coeffs(lbm_ctx* ctx, int mode, int32_t h, const double* C, const double* mu, const double* Sigma,
                      const double* sigma_ref, const double* gamma_fixed);

/* Reference QoI series for LBM_TO_TRACK (or the spin-up of LBM_TO_LRS):
 * qref[len][N], row n used at step n (len <= cfg.track_len; steps past the
 * end reuse the last row). */
int lbm_set_track_reference(lbm_ctx* ctx, const double* qref, int64_t len);

/* Queue nsteps time steps on the stream (asynchronous).  Returns the status
 * of previously completed work only; instabilities surface at lbm_sync. */
int lbm_step(lbm_ctx* ctx, int64_t nsteps);

/* Wait for queued work; ERR_UNSTABLE if any step saw an unstable state,
 * ERR_TIMEOUT if a kernel's bounded wait for its asynchronous bulk copies gave
 * up (the step's results are then not valid). */
int lbm_sync(lbm_ctx* ctx);

/* Drain QoI block rows written since the last drain into out[capacity][row_len]
 * (host).  Synchronises the stream.  If more rows were produced than the ring
 * holds, the oldest are lost and *n_lost says how many. */
int lbm_qoi(lbm_ctx* ctx, double* out, int64_t capacity, int64_t* n_written, int64_t* n_lost);

/* Density rho[nz][ny][nx] and velocity u[3][nz][ny][nx] = sum c f / rho of
 * the current post-collision state, as host FP64.  Synchronous. */
int lbm_get_macros(lbm_ctx* ctx, double* rho, double* u);

/* Full populations f (not shifted) as host FP64 [Q][nz][ny][nx]. */
int lbm_get_populations(lbm_ctx* ctx, double* f);
int lbm_set_populations(lbm_ctx* ctx, const double* f);

/* Running sum over steps of the plane-mean streamwise velocity of the
 * corrected post-collision state, prof[ny], and the number of steps summed
 * (accumulated only while the TO phase runs). */
int lbm_get_profile(lbm_ctx* ctx, double* prof, int64_t* nsteps);

/* Steps completed (device counter; synchronises). */
int lbm_get_step(lbm_ctx* ctx, int64_t* step);

/* Checkpoint: the whole device state (populations, counters, LRS model and
 * histories, tracking reference, QoI ring, profile) as an opaque host blob of
 * lbm_state_bytes bytes.  lbm_load requires a context created with the same
 * configuration and needs no other set-up call before stepping. */
int lbm_state_bytes(lbm_ctx* ctx, size_t* bytes);
int lbm_save(lbm_ctx* ctx, void* host_buf, size_t bytes);
int lbm_load(lbm_ctx* ctx, const void* host_buf, size_t bytes);

/* Execution controls.
 *   lbm_set_graphs(ctx, 1): lbm_step replays a captured CUDA graph of two
 *     steps (default on); 0 launches every kernel eagerly.
 *   lbm_profile(ctx, 1): eager launches bracketed by CUDA events on the
 *     context's stream, accumulated per kernel class; lbm_profile_read
 *     returns the totals.  Class ids are the LBM_K_* values. */
enum {
    LBM_K_MOMENTS = 0,  /* predictor pass: v^{p*} (TO modes), post-stream u (WALE) */
    LBM_K_COLLIDE = 1,  /* stream-collide, with the step's SGS corrector in TO modes */
    LBM_K_CURL = 2, LBM_K_FILTER = 3, LBM_K_SENS = 4,
    LBM_K_REDUCE = 5, LBM_K_LRS = 6, LBM_K_SOLVE = 7,
    LBM_K_APPLY = 8,    /* reserved: the corrector runs inside the collide */
    LBM_K_GAUSS_X = 9,   /* R R of a 3-D Gaussian / binomial filter: x pass     */
    LBM_K_LAP1 = 10,     /* 3-D L_1 cross (or a one-pass Laplacian kernel)      */
    LBM_K_FFT = 11,      /* cuFFT transforms of the Fourier-band filters        */
    LBM_K_WALE = 12,     /* reserved: WALE runs inside the collide              */
    LBM_K_GAUSS_Z = 13,  /* R R of a 3-D Gaussian / binomial filter: z pass     */
    LBM_K_GAUSS_Y = 14,  /* R R of a 3-D Gaussian / binomial filter: y pass     */
    LBM_K_LAP3 = 15,     /* 3-D L_3 (nx % 4 == 0): box and stride-3 cross fused */
    LBM_K_RESERVED16 = 16, /* unused                                            */
    LBM_K_TOTALS = 17,   /* cross-block sums of the reduction partials          */
    LBM_K_COUNT = 18
};
int lbm_set_graphs(lbm_ctx* ctx, int enable);

/* Step branching (default on): the LRS history product (Eq. LRS, the terms
 * known before the current QoIs) and the step's normals need only the previous
 * step, so lbm_step runs them on a second stream of the context beside the
 * field kernels and joins before the solve.  0 runs them in line on the
 * context's stream (members of an lbm_batch do: they already overlap one
 * another).  Results are identical either way.  Must precede the first
 * lbm_step (LBM_ERR_STATE after it). */
int lbm_set_branching(lbm_ctx* ctx, int enable);

/* ------------------------------------------------------------------------
 * Projection phi_m and QoIs of a given field (Sec. 3, coarse graining;
 * the HF reference trajectories used for tracking, Sec. 4.4, and for
 * training, Sec. 4.5).
 *
 * phi_m maps the state of a high-fidelity (HF) context onto an m-times
 * coarser lattice (velocities unchanged: the coarse time step is m times
 * longer).
 *   2-D, doubly periodic: bicubic interpolation (Keys cubic convolution,
 *     a = -1/2) at the LF block centres (m i + (m-1)/2, m j + (m-1)/2);
 *     LF grid nx/m x ny/m.
 *   3-D channel: wall-anchored stride-m subsampling, odd m: LF fluid row j
 *     on HF row m j - (m-1)/2 so that the walls coincide, solid rows on solid
 *     rows, x and z on the block centres; LF grid nx/m x ((ny-2)/m + 2) x nz/m
 *     (1475x237x490 with m = 5 gives 295x49x98, Sec. 7.1).
 * Other geometries, even m in 3-D and sizes that do not divide return
 * LBM_ERR_ARG.
 *
 * lbm_project_shape: the LF grid {nx, ny, nz} of phi_m for a configuration.
 * lbm_project: enqueues, on the HF context's stream, phi_m of its current
 *   state into caller-owned DEVICE buffers drho[N_LF] (density - 1) and
 *   u[3][N_LF] (u_z = 0 in 2-D; solid LF rows 0).  Reads only the HF
 *   populations at the sampled nodes.
 * lbm_eval_qoi: enqueues, on the context's stream, the context's QoIs
 *   (its scale-aware QoIs and mean-profile bands, to_mode != LBM_TO_OFF)
 *   evaluated on a caller-supplied DEVICE velocity u[3][N] of its grid,
 *   written to the DEVICE array q[N_Q].  Uses the context's TO scratch: do
 *   not overlap it with lbm_step of the same context on another stream.
 * ------------------------------------------------------------------------ */
int lbm_project_shape(const lbm_config* cfg, int m, int32_t* lf_dims);
int lbm_project(lbm_ctx* hf, int m, float* drho_lf, float* u_lf);
int lbm_eval_qoi(lbm_ctx* ctx, const float* u, double* q);

/* Autotuner (default on): before the first lbm_step the library times the
 * candidate launch shapes of its kernels on this context's buffers (node-pair
 * vs single-node collide and predictor pass, the z-segment count of the fused 3-D filters, the
 * line segments of 2-D filter passes) and keeps the fastest, cached per grid
 * shape for the process.  Per node, every candidate evaluates the same
 * arithmetic.  lbm_set_autotune must precede the first lbm_step; 0 keeps the
 * built-in shapes.  lbm_get_tuning returns [tuned, collide_pair,
 * corrector_in_collide (1 when the step's SGS corrector runs inside the
 * collide: every TO mode but OFF and OBSERVE), march_threads, blocks_per_sm
 * of filter slot 0..7 (0 = default), throughput goal, predict_pair] (up to
 * count values). */
int lbm_set_autotune(lbm_ctx* ctx, int enable);
int lbm_get_tuning(lbm_ctx* ctx, int32_t* values, int count);

/* Launch goal (default LBM_GOAL_LATENCY): launch shapes that make this
 * context's step fastest when it has the GPU to itself; for small grids the
 * fused 3-D filters then split z into many short segments, re-reading 2R halo
 * planes each.  LBM_GOAL_THROUGHPUT: one z segment per block column, the
 * least total work, for a context that shares the GPU with many others
 * (members of an lbm_batch use it).  Results are identical either way.  Must
 * precede the first lbm_step (LBM_ERR_STATE after it); lbm_get_tuning
 * reports it as value 12 (1: throughput). */
enum { LBM_GOAL_LATENCY = 0, LBM_GOAL_THROUGHPUT = 1 };
int lbm_set_launch_goal(lbm_ctx* ctx, int goal);
int lbm_profile(lbm_ctx* ctx, int enable);
int lbm_profile_read(lbm_ctx* ctx, double* ms, int64_t* launches, int count);

/* Kernel launches one lbm_step(ctx, 1) queues (for launch accounting). */
int lbm_launches_per_step(lbm_ctx* ctx, int64_t* launches);

/* Algorithmic floating-point operations of one step's filter applications,
 * per kernel class (LBM_K_GAUSS3, LBM_K_LAP3, LBM_K_FILTER): 2 x taps x
 * components x nodes, with G_s and B3 counted as d separable factors and
 * L_s as the box B_s (d factors of s taps) times the (4d + 1)-point cross
 * of l at stride s (Sec. 4.1: L_s is L_1 dilated by the s^d block of ones);
 * halo recomputation excluded. */
int lbm_filter_flops_per_step(lbm_ctx* ctx, double* flops, int count);

/* ------------------------------------------------------------------------
 * Ensembles: many independent members (different grids, seeds, horizons)
 * advancing together on one GPU.  The paper runs ensembles of five replicas
 * per configuration (Sec. 6.4, Sec. 7.4); the batch API runs any number of
 * members concurrently so that small grids fill the device.
 *
 * The caller owns one device pool; the batch carves each admitted member out
 * of it (first fit, 256-byte aligned) and returns LBM_ERR_BUDGET when a member
 * does not fit or no slot is free, so admission is by HBM budget.  Every
 * member has its own stream; lbm_batch_run queues the steps of all active
 * members without waiting, either as persistent batched kernels over all
 * members (default, lbm_batch_set_persistent) or as per-member graphs that
 * the device overlaps.  A member's results are bit-identical whether it runs
 * alone or in a mix (its kernels read only its own memory, on the block
 * indices of its own launch).
 * ------------------------------------------------------------------------ */
typedef struct lbm_batch lbm_batch;

typedef struct {
    int32_t slot;        /* member slot                                        */
    int32_t status;      /* LBM_OK or LBM_ERR_UNSTABLE                         */
    int64_t steps;       /* steps completed (= horizon)                        */
    uint64_t tag;        /* caller's tag from lbm_batch_admit                  */
    double t_done_ms;    /* device time of completion, ms since lbm_batch_create */
} lbm_completion;

/* n_slots members at most, carved from dev_pool (device, 256-byte aligned). */
int lbm_batch_create(int32_t n_slots, void* dev_pool, size_t pool_bytes, lbm_batch** out);
int lbm_batch_destroy(lbm_batch* b);

/* Admit a member: allocate from the pool, create it, set f = f^eq(1, u0)
 * (u0 host FP64 [3][nz][ny][nx]).  horizon = steps to run.  For LBM_TO_LRS
 * call lbm_set_lrs on lbm_batch_member(slot) before the next lbm_batch_run.
 * LBM_ERR_BUDGET: no free slot or not enough contiguous pool memory. */
int lbm_batch_admit(lbm_batch* b, const lbm_config* cfg, const double* u0, int64_t horizon, uint64_t tag,
                    int32_t* slot);

/* The member's context (for lbm_set_lrs, lbm_qoi, lbm_get_macros, ...). */
int lbm_batch_member(lbm_batch* b, int32_t slot, lbm_ctx** ctx);

/* Queue up to `steps` more steps of every active member (stopping at each
 * member's horizon).  Asynchronous.  A member's first call records its step
 * (and runs lbm_step's checks and tuning). */
int lbm_batch_run(lbm_batch* b, int64_t steps);

/* How members advance.  A member of at most max_nodes nodes (default 16384)
 * with lanes > 0 (default 1) runs persistent: members whose steps run the
 * same kernels form a class, split over `lanes` lanes (each with its own
 * stream); every launch of a lane's step runs as one persistent kernel over
 * all its active members (blocks draw (member, block) work items from a
 * global queue over a member table in device memory), and a call's steps of
 * a lane are one CUDA graph.  Other members, and those whose step makes a
 * library call (Fourier-band filters: cuFFT), replay their own two-step graph
 * on their own stream (lanes = 0: every member).  Small members gain from the
 * persistent kernels (one launch per step kernel for the whole class); larger
 * ones run faster as hardware-scheduled graphs overlapping on their streams.
 * Results are bit-identical either way.  lanes 0..64, max_nodes >= 0; set
 * before the members' first lbm_batch_run (LBM_ERR_STATE otherwise). */
int lbm_batch_set_persistent(lbm_batch* b, int lanes, int64_t max_nodes);

/* Flow control for a scheduler: block until at most `rounds` (0..3) of the
 * most recent lbm_batch_run calls are still executing on any member.
 * rounds = 1 keeps one call queued behind the running one, so the device is
 * never drained between calls while the host admits and releases members
 * (members that were not active in a call do not wait for it). */
int lbm_batch_wait(lbm_batch* b, int32_t rounds);

/* Members whose horizon has been reached on the device (non-blocking):
 * up to cap completions into out, count in *n.  Each is reported once. */
int lbm_batch_poll(lbm_batch* b, lbm_completion* out, int32_t cap, int32_t* n);

/* Free a member's slot and pool memory (after its results were read). */
int lbm_batch_release(lbm_batch* b, int32_t slot);

/* Pool bytes free in total and in the largest contiguous block; active members. */
int lbm_batch_stats(lbm_batch* b, size_t* free_bytes, size_t* largest, int32_t* active);

/* QoIs of a velocity field, for callers that cannot allocate device memory.
 *
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot call cudaMalloc or hand the library a buffer: code that runs
 * while a CUDA graph is being captured, code embedded in a host framework
 * that owns every device allocation through its own arena, and real-time
 * loops that cannot afford the implicit device synchronisation of an
 * allocation.  It computes the same scale-aware QoIs as the TO phase of
 * lbm_step (the Tau-orthogonal SGS forcing step) reports for each
 * cfg->qoi[i], for a field the caller supplies, using only a scratch array
 * compiled into the library.
 *
 *   cfg     grid (dim, nx, ny, nz, walls) and the scale-aware QoIs:
 *           n_qoi in 1..8, Gaussian, Laplacian or binomial filters
 *           (LBM_FILTER_FOURIER is refused); mean-profile bands are not
 *           supported (n_mp must be 0); to_mode and the LBM fields are ignored
 *   u       device pointer, FP32 velocity [3][nz][ny][nx] (z component
 *           ignored in 2-D); values on solid rows are treated as zero
 *   q       device pointer, receives n_qoi doubles
 *   stream  cudaStream_t the work is queued on (asynchronous)
 *
 * Scratch: one file-scope device array of LBM_STATIC_SCRATCH_BYTES that every
 * GPU loading the library holds until the process exits.  The grid and QoI
 * set must fit in it (about 200 bytes per node for six 3-D QoIs over three
 * filters); larger requests return LBM_ERR_BUDGET and say how many bytes they
 * would need.  Nothing is allocated: no cudaMalloc, no cudaFree, no
 * allocating library call.  The first call in each CUDA context (each
 * device's primary context, a context recreated after cudaDeviceReset, or a
 * context of the caller's own) looks up the array's device address
 * (cudaGetSymbolAddress with that context current) and caches it under the
 * context's unique id; make that first call before any stream capture
 * begins.  Every call shares the one array and it keeps the previous call's
 * contents, so calls whose work overlaps on the GPU (other streams, other
 * host threads) race with each other; serialise them.
 * Errors: LBM_ERR_ARG (invalid grid or QoI set), LBM_ERR_BUDGET (too large
 * for the scratch), LBM_ERR_CUDA; the text is lbm_last_error(NULL, ...). */
#define LBM_STATIC_SCRATCH_BYTES (64u << 20)
int lbm_qoi_eval_static(const lbm_config* cfg, const float* u, double* q, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
