// Internal declarations shared by the library's CUDA sources.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lbm.h"

namespace lbm {

constexpr int kMaxQoi = LBM_MAX_QOI;
constexpr int kLrsRowsPerBlk = 1024;  // most rows of C one history-matvec block takes
constexpr int kMaxTaps = 64;     // longest 1-D filter pass (L_s arm: 5 s taps)
constexpr int kMaxFilters = 8;   // distinct (filter, scale) pairs per run

// Device-resident counters and status of one simulation.
struct DevState {
    long long step;        // steps completed
    long long hist_pos;    // LRS history pushes so far
    long long ring_count;  // QoI rows written so far
    long long prof_steps;  // steps summed into the mean profile
    unsigned int status;   // bit 0: unstable seen
    unsigned int pad[3];
};

// One 1-D convolution pass along an axis (0 = x, 1 = y, 2 = z).
struct Taps {
    int radius;     // taps at offsets -radius..radius
    float t[kMaxTaps];
};

// A Gaussian (or binomial) 1-D kernel t of radius R and its self-convolution
// c = t * t (radius 2R): R R along a periodic axis applies c once.
struct GaussTaps {
    int radius;        // R: 1 (binomial), 2, 4 or 6
    float t[13];       // t[0 .. 2R]
    float c[25];       // c[0 .. 4R]
};

// Pointers into the caller's buffer, computed once at create time.
struct Layout {
    void* f[2];          // shifted populations, ping-pong
    float* vps;          // [d][N]  predictor velocity v^{p*} (aliases x6)
    float* vn;           // [3][N]  post-stream velocity (WALE gradients)
    float* kolmo;        // [ny]    Kolmogorov force profile
    float* x6;           // [ncomp][N] stacked (v, omega) filter input
    float* t1;           // [6][N]  pass scratch
    float* t2;           // [6][N]  pass scratch
    float* acc;          // [6][N]  R applied once
    float* rr[kMaxFilters];  // [6][N] R R (v, omega) per filter
    float* vz[kMaxFilters];  // [3][N] curl*(R R omega) per filter
    float* part;         // [nblk_red][npart_all] reduction partials (FP32 block sums, coupling pairs)
    float* plane_part;   // [nzc][ny][1 + n_s] plane-sum partials
    double* plane_sum;   // [ny][1 + n_s] plane sums of v_x and V_k,x
    double* tot;         // [ntot] totals of the reduction partials
    double* hsum;        // [N_Q] known part of the LRS prediction (histories, mu, L z)
    float2* w_mp2;       // [n_mp][ny] band weights as float pairs hi + lo (block couplings)
    double* lrs_part;    // [nblk_lrs][N_Q] LRS history matvec partials
    double* znorm;       // [N_Q] normals of the current step (LRS noise / gamma draws)
    double* lrs_C;       // [(2h+1)N + 1][N]
    double* lrs_mu;      // [N]
    double* lrs_L;       // [N][N] Cholesky factor of Sigma
    double* lrs_sigma;   // [N]
    double* qh;          // [h][N] corrected-QoI ring
    double* qsh;         // [h][N] predictor-QoI ring
    double* track;       // [track_len][N]
    double* w_mp;        // [n_mp][ny] band weights
    double* g_mpmp;      // [n_mp][n_mp]
    double* beta;        // [N_Q] SGS coefficients of the current step (beta = G^-1 dQ)
    double* gfix;        // [N_Q] caller's gamma_i (LBM_TO_FIXED_GAMMA)
    float* betaf;        // [N_Q] beta rounded to FP32 (the collide's SGS corrector)
    float* mprow;        // [ny]  sum_j beta_j w_j(y) of the bands, FP32, per row
    double* ring;        // [ring_cap][row_len]
    double* profile;     // [ny]
    float2* spec;        // [3][ny][nx/2+1] spectrum of (v_x, v_y, omega) (Fourier bands)
    float2* spec_band;   // [3][ny][nx/2+1] one band of it
    void* fft_work;      // cuFFT work area
    DevState* st;
};

// Launch shapes chosen by the autotuner (results do not depend on them).
struct Tune {
    int filter_per_sm[8];  // fused 3-D filter of each distinct filter slot: target blocks per SM (0: default)
    int march_lines;    // 1-D passes along y/z: target threads in flight (line segments)
    int collide_pair;   // node-pair collide when nx is even
    int predict_pair;   // node-pair predictor pass when nx is even
    int one_seg;        // fused 3-D filters: one z segment per block column (least total work)
};

struct Params {
    int dim, q, nx, ny, nz, walls, forcing, substrate, storage, to_mode;
    long long n;         // nodes
    float tau, body[3], kolmo_drag, c_smag2, c_wale2;
    float omega0;        // 1/tau rounded once from double
    float guo_pre0;      // 1 - 1/(2 tau) rounded once from double
    int n_s, n_mp, n_q;  // scale QoIs, bands, total
    int qoi_kind[kMaxQoi];
    int qoi_filter_slot[kMaxQoi];  // which distinct filter each scale QoI uses
    int n_filters;
    int ncomp;           // components filtered: 3 (2-D: vx, vy, w) or 6 (3-D)
    int h, ring_cap, row_len;
    long long track_len;
    long long spinup;    // LRS: steps nudged to the reference first
    double gamma_std;
    double inv_area;     // 1 / (nx nz), rounded once on the host
    unsigned long long seed, member;
    int nblk_red, nzc, npart, nblk_lrs, lrs_rows_per_blk;
    int ntot;            // npart + n_mp (1 + n_s) mean-profile couplings
    int npart_all;       // floats per block partial row: npart + 2 n_mp (1 + n_s) (couplings as float pairs)
    Tune tune;
};

// ---- launchers (stream-ordered; return cudaGetLastError()) ----
cudaError_t launch_init_feq(const Params& p, const Layout& L, const float* rho, const float* u, int which,
                            cudaStream_t s);
// predictor pass: v^{p*} (TO modes) and the post-stream velocity (WALE)
cudaError_t launch_predict(const Params& p, const Layout& L, int src, cudaStream_t s);
// stream-collide from f[src] into f[1 - src], with the SGS corrector of the
// step when corrector_runs(p) (every TO mode but OFF and OBSERVE)
cudaError_t launch_collide(const Params& p, const Layout& L, int src, cudaStream_t s);
bool corrector_runs(const Params& p);
cudaError_t launch_to_curl(const Params& p, const Layout& L, cudaStream_t s);
cudaError_t launch_pass(const Params& p, const float* in, float* out, int ncomp, int axis, const Taps& t,
                        float scale, int accumulate, cudaStream_t s);
cudaError_t launch_pass_fast(const Params& p, const float* in, float* out, int ncomp, int axis, const Taps& t,
                             float scale, int accumulate, cudaStream_t s);
// one fused launch for a whole 2-D filter application on a doubly periodic
// grid (G_s / B3 of radius 1, 4, 12; L_1); cudaErrorNotSupported otherwise
cudaError_t launch_filter2_fused(const Params& p, const float* in, float* out, int ncomp, bool laplacian, int s_scale,
                                 const Taps& t, float scale, int accumulate, cudaStream_t s);
// per_sm: target blocks per SM (z segments); 0 = built-in default
cudaError_t launch_lap3(const Params& p, const float* in, float* out, int ncomp, int s_scale, const Taps& arm,
                        float scale, int accumulate, int per_sm, cudaStream_t s);
inline bool launch_lap3_supported(int s_scale) { return s_scale == 1 || s_scale == 3; }
// L_3 as two launches through a scratch field (box, then cross at stride 3)
bool lap3_split(const Params& p, int s_scale);
// L_3 = c C_3 * B_3 in one pass (nx % 4 == 0, lap3_split): box and cross
// through shared memory, the z arms in registers
cudaError_t launch_lap3_fused(const Params& p, const float* in, float* out, int ncomp, float scale, int per_sm,
                              cudaStream_t s);
// R R of a 3-D Gaussian / binomial filter on ncomp fields is three streaming
// passes: axis 0 (x) and 2 (z) with the composite kernel, then axis 1 (y)
// with the wall projection; any order of the three gives the same operator
bool launch_gauss_rr_supported(int radius);
cudaError_t launch_gauss_pass(const Params& p, int axis, const float* in, float* out, int ncomp, const GaussTaps& gt,
                              DevState* st, cudaStream_t s);
cudaError_t launch_band_mask(const Params& p, const float2* in, float2* out, int ncomp, int lo, int hi,
                             cudaStream_t s);
cudaError_t launch_sens_curl(const Params& p, const float* w, float* out, cudaStream_t s);
cudaError_t launch_reduce(const Params& p, const Layout& L, const float* const* vk, cudaStream_t s);
// LRS history partials and the step's normals (LRS and gamma modes)
cudaError_t launch_lrs_pre(const Params& p, const Layout& L, cudaStream_t s);
cudaError_t launch_totals(const Params& p, const Layout& L, bool with_lrs, cudaStream_t s);
cudaError_t launch_solve(const Params& p, const Layout& L, cudaStream_t s);
cudaError_t launch_macros(const Params& p, const Layout& L, int which, float* drho_out, float* u_out,
                          cudaStream_t s);
// projection phi_m of the stored state onto the nxl x nyl x nzl LF grid
cudaError_t launch_project(const Params& p, const Layout& L, int which, int m, int nxl, int nyl, int nzl,
                           float* drho, float* u, cudaStream_t s);
// the QoIs of a given velocity field: u [3][N] into x6, then q from the totals
cudaError_t launch_load_velocity(const Params& p, const Layout& L, const float* u, cudaStream_t s);
cudaError_t launch_qoi_values(const Params& p, const Layout& L, double* q, cudaStream_t s);

void set_global_error(const char* msg);

}  // namespace lbm
