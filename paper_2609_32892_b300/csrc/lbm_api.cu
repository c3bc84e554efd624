// C ABI of the library (include/lbm.h): configuration checks, placement of
// every device array inside the caller's buffer, the per-step launch
// sequence, CUDA-graph replay and host<->device marshalling.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <memory>
#include <thread>
#if defined(__SSE2__)
#include <emmintrin.h>
#endif
#include <vector>

#include <cufft.h>

#include "batch.cuh"
#include "lbm_common.cuh"

using namespace lbm;

namespace {

thread_local char g_err[256] = "";

struct Filter {
    int kind;   // LBM_FILTER_*
    int scale;  // s, or the lower wavenumber bin of a Fourier band
    int hi;     // upper wavenumber bin of a Fourier band
    bool need_z;
};

}  // namespace

struct lbm_ctx {
    lbm_config cfg;
    Params p;
    Layout L;
    cudaStream_t stream;       // caller's stream
    cudaStream_t cap_stream;   // private stream used only to capture the step graph
    cudaStream_t side;         // branch of the step that runs beside the field kernels
    cudaEvent_t ev_fork, ev_join;
    std::vector<Filter> filters;
    std::vector<Taps> taps1d;  // scratch for building passes
    int cur;                   // which population buffer holds the current state
    int use_graphs;
    int profiling;
    cudaGraphExec_t graph;     // two steps: src 0 -> 1, then 1 -> 0
    long long host_read;       // QoI rows already drained
    long long launches_per_step;
    double filter_flops[LBM_K_COUNT];  // algorithmic flops per step by kernel class
    float* aux;                // [4][N] scratch for macros / init
    float* hpin;               // [4][N] pinned host staging for macros / init (on first use)
    size_t elem;               // bytes per stored population
    char err[256];
    // profiling
    cudaEvent_t ev[2 * 96];
    int ev_used;
    int ev_class[96];
    double prof_ms[LBM_K_COUNT];
    long long prof_n[LBM_K_COUNT];
    int lrs_set;
    int fixed_set;    // LBM_TO_FIXED_GAMMA: gamma_i given
    int autotune;     // tune launch shapes before the first step (default on)
    int branch;       // LRS history / normals on a parallel branch of the step (default on)
    int tuned;
    cufftHandle fft_r2c, fft_c2r;  // Fourier-band filters (3 components batched)
    bool has_fft;
};

static int fail(lbm_ctx* c, int code, const char* fmt, ...) {
    char buf[256];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    snprintf(g_err, sizeof g_err, "%s", buf);
    if (c) snprintf(c->err, sizeof c->err, "%s", buf);
    return code;
}

namespace lbm {
// Record a message as the thread's last error (lbm_last_error(NULL, ...)).
void set_global_error(const char* msg) { snprintf(g_err, sizeof g_err, "%s", msg); }
}  // namespace lbm

#define CK(c, call)                                                                         \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) return fail((c), LBM_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

// ------------------------------------------------------------ validation --
static int qoi_count(const lbm_config* c) { return c->to_mode == LBM_TO_OFF ? 0 : c->n_qoi + c->n_mp; }

static int validate(const lbm_config* c) {
    if (!c) return fail(nullptr, LBM_ERR_ARG, "config is NULL");
    if (c->dim != 2 && c->dim != 3) return fail(nullptr, LBM_ERR_ARG, "dim must be 2 or 3");
    if (c->nx < 3 || c->ny < 3 || c->nz < 1) return fail(nullptr, LBM_ERR_ARG, "grid too small (nx, ny >= 3)");
    if (c->dim == 2 && c->nz != 1) return fail(nullptr, LBM_ERR_ARG, "2-D runs need nz = 1");
    if (c->dim == 3 && c->nz < 3) return fail(nullptr, LBM_ERR_ARG, "3-D runs need nz >= 3");
    if (c->walls && c->ny < 4) return fail(nullptr, LBM_ERR_ARG, "walls need ny >= 4");
    if (!(c->tau > 0.5)) return fail(nullptr, LBM_ERR_ARG, "tau must exceed 1/2");
    if (c->forcing != LBM_FORCING_EDM && c->forcing != LBM_FORCING_GUO) return fail(nullptr, LBM_ERR_ARG, "bad forcing");
    if (c->substrate < 0 || c->substrate > 2) return fail(nullptr, LBM_ERR_ARG, "bad substrate");
    if (c->storage < 0 || c->storage > 2) return fail(nullptr, LBM_ERR_ARG, "bad storage");
    if (c->to_mode < 0 || c->to_mode > 5) return fail(nullptr, LBM_ERR_ARG, "bad to_mode");
    const long long n = (long long)c->nx * c->ny * c->nz;
    // populations are addressed with 64-bit offsets (Q N may exceed 2^31, e.g. the
    // 171 M-node HF channel); node indices and the per-component offsets of the
    // velocity and filter fields (up to 6 N) are 32-bit
    if (n * 6 >= (1LL << 31)) return fail(nullptr, LBM_ERR_ARG, "grid too large (6 N >= 2^31)");
    if (c->to_mode != LBM_TO_OFF) {
        if (c->n_qoi < 0 || c->n_mp < 0 || c->n_qoi + c->n_mp < 1 || c->n_qoi + c->n_mp > LBM_MAX_QOI)
            return fail(nullptr, LBM_ERR_ARG, "need 1..%d QoIs", LBM_MAX_QOI);
        if (c->n_qoi > 8) return fail(nullptr, LBM_ERR_ARG, "at most 8 scale-aware QoIs");
        if (c->n_qoi < 1) return fail(nullptr, LBM_ERR_ARG, "need at least one scale-aware QoI");
        if (c->n_mp > 0 && !c->walls) return fail(nullptr, LBM_ERR_ARG, "mean-profile QoIs need walls");
        if (c->n_mp == 1) return fail(nullptr, LBM_ERR_ARG, "mean-profile bands need n_mp >= 2");
        for (int i = 0; i < c->n_qoi; ++i) {
            const lbm_qoi_spec& s = c->qoi[i];
            if (s.kind != LBM_QOI_ENERGY && s.kind != LBM_QOI_ENSTROPHY) return fail(nullptr, LBM_ERR_ARG, "bad QoI kind");
            if (s.filter < 0 || s.filter > 3) return fail(nullptr, LBM_ERR_ARG, "bad QoI filter");
            if (s.filter == LBM_FILTER_FOURIER) {
                if (c->dim != 2 || c->walls || c->nx != c->ny || c->nx % 2)
                    return fail(nullptr, LBM_ERR_ARG, "Fourier-band QoIs need a periodic 2-D grid with nx = ny even");
                if (s.scale < 0 || s.band_hi < s.scale) return fail(nullptr, LBM_ERR_ARG, "bad Fourier band");
                continue;
            }
            if (s.filter != LBM_FILTER_BINOMIAL && (s.scale < 1 || s.scale % 2 == 0))
                return fail(nullptr, LBM_ERR_ARG, "filter scale must be odd and >= 1");
            const int alpha = c->dim == 2 ? 4 : 2;
            if (s.filter == LBM_FILTER_GAUSS && 2 * alpha * s.scale + 1 > kMaxTaps)
                return fail(nullptr, LBM_ERR_ARG, "Gaussian scale too large");
            if (s.filter == LBM_FILTER_LAPLACE && 5 * s.scale > kMaxTaps)
                return fail(nullptr, LBM_ERR_ARG, "Laplacian scale too large");
        }
        if (c->to_mode == LBM_TO_LRS && (c->h < 1 || c->h > (1 << 20))) return fail(nullptr, LBM_ERR_ARG, "LRS needs 1 <= h <= 2^20");
        if (c->to_mode == LBM_TO_TRACK && c->track_len < 1) return fail(nullptr, LBM_ERR_ARG, "tracking needs track_len >= 1");
        if (c->spinup < 0) return fail(nullptr, LBM_ERR_ARG, "spinup must be >= 0");
        if (c->spinup > 0 && c->to_mode != LBM_TO_LRS) return fail(nullptr, LBM_ERR_ARG, "spinup applies to LBM_TO_LRS");
        if (c->spinup > 0 && c->track_len < 1) return fail(nullptr, LBM_ERR_ARG, "spinup needs track_len >= 1");
    }
    return LBM_OK;
}

static std::vector<Filter> distinct_filters(const lbm_config* c, int* slot) {
    std::vector<Filter> out;
    if (c->to_mode == LBM_TO_OFF) return out;
    for (int i = 0; i < c->n_qoi; ++i) {
        const int kind = c->qoi[i].filter;
        const int s = kind == LBM_FILTER_BINOMIAL ? 1 : c->qoi[i].scale;
        const int hi = kind == LBM_FILTER_FOURIER ? c->qoi[i].band_hi : 0;
        int found = -1;
        for (size_t j = 0; j < out.size(); ++j)
            if (out[j].kind == kind && out[j].scale == s && out[j].hi == hi) found = (int)j;
        if (found < 0) {
            out.push_back({kind, s, hi, false});
            found = (int)out.size() - 1;
        }
        if (c->qoi[i].kind == LBM_QOI_ENSTROPHY) out[found].need_z = true;
        slot[i] = found;
    }
    return out;
}

// ---------------------------------------------------------------- layout --
struct Carver {
    size_t off = 0;
    char* base = nullptr;
    template <typename T> T* take(size_t count) {
        off = (off + 255) & ~(size_t)255;
        T* r = base ? (T*)(base + off) : nullptr;
        off += count * sizeof(T);
        return r;
    }
};

static void make_params(const lbm_config* c, Params* p, std::vector<Filter>* filt) {
    memset(p, 0, sizeof *p);
    p->dim = c->dim;
    p->q = c->dim == 2 ? 9 : 19;
    p->nx = c->nx; p->ny = c->ny; p->nz = c->nz;
    p->walls = c->walls ? 1 : 0;
    p->forcing = c->forcing;
    p->substrate = c->substrate;
    p->storage = c->storage;
    p->to_mode = c->to_mode;
    p->n = (long long)c->nx * c->ny * c->nz;
    p->tau = (float)c->tau;
    p->omega0 = (float)(1.0 / c->tau);
    p->guo_pre0 = (float)(1.0 - 0.5 / c->tau);
    for (int a = 0; a < 3; ++a) p->body[a] = (float)c->body_force[a];
    if (c->dim == 2) p->body[2] = 0.f;
    p->kolmo_drag = (float)c->kolmo_drag;
    p->c_smag2 = (float)(c->c_smag * c->c_smag);
    p->c_wale2 = (float)(c->c_wale * c->c_wale);
    const bool to = c->to_mode != LBM_TO_OFF;
    p->n_s = to ? c->n_qoi : 0;
    p->n_mp = to ? c->n_mp : 0;
    p->n_q = p->n_s + p->n_mp;
    int slot[kMaxQoi] = {0};
    *filt = distinct_filters(c, slot);
    for (int i = 0; i < p->n_s; ++i) {
        p->qoi_kind[i] = c->qoi[i].kind;
        p->qoi_filter_slot[i] = slot[i];
    }
    p->n_filters = (int)filt->size();
    p->ncomp = c->dim == 2 ? 3 : 6;
    p->h = c->to_mode == LBM_TO_LRS ? c->h : 0;
    p->ring_cap = c->qoi_ring > 0 ? c->qoi_ring : 4096;
    p->row_len = 2 + 3 * p->n_q;
    p->spinup = c->to_mode == LBM_TO_LRS ? c->spinup : 0;
    p->track_len = (c->to_mode == LBM_TO_TRACK || p->spinup > 0) ? c->track_len : 0;
    p->gamma_std = c->gamma_std;
    p->inv_area = 1.0 / ((double)c->nx * (double)c->nz);
    p->seed = c->seed;
    p->member = c->member;
    // reduction geometry: one block per (row y, chunk of z planes), ~1200 blocks
    int target = (1184 + c->ny - 1) / c->ny;
    if (target < 1) target = 1;
    if (target > c->nz) target = c->nz;
    const int zper = (c->nz + target - 1) / target;
    p->nzc = (c->nz + zper - 1) / zper;
    p->nblk_red = c->ny * p->nzc;
    p->npart = p->n_s + p->n_s * (p->n_s + 1) / 2;
    p->ntot = p->npart + p->n_mp * (1 + p->n_s);
    p->npart_all = p->npart + 2 * p->n_mp * (1 + p->n_s);
    for (int f = 0; f < 8; ++f) p->tune.filter_per_sm[f] = 0;
    p->tune.march_lines = 148 * 2048;
    p->tune.collide_pair = c->substrate == LBM_SUBSTRATE_WALE ? 0 : 1;
    p->tune.predict_pair = c->substrate == LBM_SUBSTRATE_WALE ? 0 : 1;
    p->tune.one_seg = 0;
    if (p->h > 0) {
        const long long rows = (long long)(2 * p->h + 1) * p->n_q + 1;
        // about 64 blocks (the solve sums their partials two per lane)
        long long rpb = (rows + 63) / 64;
        if (rpb < 256) rpb = 256;
        if (rpb > kLrsRowsPerBlk) rpb = kLrsRowsPerBlk;
        p->lrs_rows_per_blk = (int)rpb;
        p->nblk_lrs = (int)((rows + rpb - 1) / rpb);
    }
}

// cuFFT 2-D transforms of the three filtered components (v_x, v_y, omega),
// batched with component stride N, real <-> half spectrum
static void fft_dims(const Params& p, int n[2], int rin[2], int cout_[2]) {
    n[0] = p.ny; n[1] = p.nx;
    rin[0] = p.ny; rin[1] = p.nx;
    cout_[0] = p.ny; cout_[1] = p.nx / 2 + 1;
}

static size_t fft_work_bytes(const Params& p) {
    int n[2], rin[2], co[2];
    fft_dims(p, n, rin, co);
    const int idist = p.ny * p.nx, odist = p.ny * (p.nx / 2 + 1);
    size_t a = 0, b = 0;
    cufftEstimateMany(2, n, rin, 1, idist, co, 1, odist, CUFFT_R2C, 3, &a);
    cufftEstimateMany(2, n, co, 1, odist, rin, 1, idist, CUFFT_C2R, 3, &b);
    const size_t w = a > b ? a : b;
    return (w + (1 << 20)) & ~(size_t)255;  // estimate plus margin
}

static size_t carve(const lbm_config* c, const Params& p, const std::vector<Filter>& filt, char* base, Layout* L,
                    float** aux) {
    Carver cv;
    cv.base = base;
    Layout l;
    memset(&l, 0, sizeof l);
    const size_t N = (size_t)p.n;
    const size_t elem = c->storage == LBM_STORAGE_FP32 ? 4 : 2;
    l.f[0] = cv.take<char>(elem * p.q * N);
    l.f[1] = cv.take<char>(elem * p.q * N);
    *aux = cv.take<float>(4 * N);
    l.kolmo = cv.take<float>(p.ny);
    if (c->substrate == LBM_SUBSTRATE_WALE) l.vn = cv.take<float>(3 * N);
    if (p.to_mode != LBM_TO_OFF) {
        l.x6 = cv.take<float>(p.ncomp * N);
        l.vps = l.x6;
        l.t1 = cv.take<float>(p.ncomp * N);
        l.t2 = cv.take<float>(p.ncomp * N);
        l.acc = cv.take<float>(p.ncomp * N);
        for (size_t f = 0; f < filt.size(); ++f) {
            l.rr[f] = cv.take<float>(p.ncomp * N);
            l.vz[f] = filt[f].need_z ? cv.take<float>(p.dim * N) : nullptr;
        }
        l.part = cv.take<float>((size_t)p.nblk_red * (p.npart_all > 0 ? p.npart_all : 1));
        l.tot = cv.take<double>(p.ntot > 0 ? p.ntot : 1);
        l.hsum = cv.take<double>(kMaxQoi);
        l.plane_part = cv.take<float>((size_t)p.nzc * p.ny * (1 + p.n_s));
        l.znorm = cv.take<double>(kMaxQoi);
        l.plane_sum = cv.take<double>((size_t)p.ny * (1 + p.n_s));
        if (p.h > 0) {
            const size_t rows = (size_t)(2 * p.h + 1) * p.n_q + 1;
            l.lrs_part = cv.take<double>((size_t)p.nblk_lrs * p.n_q);
            l.lrs_C = cv.take<double>(rows * p.n_q);
            l.lrs_mu = cv.take<double>(p.n_q);
            l.lrs_L = cv.take<double>((size_t)p.n_q * p.n_q);
            l.lrs_sigma = cv.take<double>(p.n_q);
            l.qh = cv.take<double>((size_t)p.h * p.n_q);
            l.qsh = cv.take<double>((size_t)p.h * p.n_q);
        }
        if (p.track_len > 0) l.track = cv.take<double>((size_t)p.track_len * p.n_q);
        l.w_mp = cv.take<double>((size_t)(p.n_mp > 0 ? p.n_mp : 1) * p.ny);
        l.w_mp2 = cv.take<float2>((size_t)(p.n_mp > 0 ? p.n_mp : 1) * p.ny);
        l.g_mpmp = cv.take<double>((size_t)(p.n_mp > 0 ? p.n_mp * p.n_mp : 1));
        bool fourier = false;
        for (const Filter& f : filt) fourier = fourier || f.kind == LBM_FILTER_FOURIER;
        if (fourier) {
            const size_t nspec = (size_t)3 * p.ny * (p.nx / 2 + 1);
            l.spec = cv.take<float2>(nspec);
            l.spec_band = cv.take<float2>(nspec);
            l.fft_work = cv.take<char>(fft_work_bytes(p));
        }
        l.beta = cv.take<double>(kMaxQoi);
        l.betaf = cv.take<float>(kMaxQoi);
        l.mprow = cv.take<float>(p.ny);
        if (p.to_mode == LBM_TO_FIXED_GAMMA) l.gfix = cv.take<double>(kMaxQoi);
        l.ring = cv.take<double>((size_t)p.ring_cap * p.row_len);
        l.profile = cv.take<double>(p.ny);
    }
    l.st = cv.take<DevState>(1);
    if (L) *L = l;
    return (cv.off + 255) & ~(size_t)255;
}

// -------------------------------------------------------- filter passes --
// 1-D factors of the compact filters (Sec. 4.1).
//   G_s: exp(-r^2/(2 s^2)) normalised on |r| <= alpha s (alpha = 4 in 2-D,
//        2 in 3-D); the d-D kernel of Eq. gaussian is the product of these.
//   L_s: sum over axes a of [l dilated by s along a] x [box_s on the other
//        axes], l = [1,-4,6,-4,1], scaled by 1/(8 d s^d) so sum |L_s| = 2
//        (Eq. laplace, Kronecker dilation with the all-ones block).
//   B3 : [1, 2, 1] / 4 on every axis.
static Taps gauss_taps(int s, int dim) {
    Taps t;
    memset(&t, 0, sizeof t);
    const int alpha = dim == 2 ? 4 : 2;
    t.radius = alpha * s;
    double sum = 0.0, v[kMaxTaps];
    for (int r = -t.radius; r <= t.radius; ++r) {
        v[r + t.radius] = exp(-(double)(r * r) / (2.0 * s * s));
        sum += v[r + t.radius];
    }
    for (int i = 0; i <= 2 * t.radius; ++i) t.t[i] = (float)(v[i] / sum);
    return t;
}
static Taps ell_taps(int s) {
    static const double ell[5] = {1.0, -4.0, 6.0, -4.0, 1.0};
    Taps t;
    memset(&t, 0, sizeof t);
    t.radius = (5 * s - 1) / 2;
    for (int m = 0; m < 5 * s; ++m) t.t[m] = (float)ell[m / s];
    return t;
}
static Taps box_taps(int s) {
    Taps t;
    memset(&t, 0, sizeof t);
    t.radius = (s - 1) / 2;
    for (int m = 0; m < s; ++m) t.t[m] = 1.0f;
    return t;
}
// The 3-D Gaussian (alpha = 2) or binomial 1-D kernel t and its
// self-convolution t * t, both from double (the factor R R applies along a
// periodic axis)
static GaussTaps gauss_pair_taps(const Filter& f) {
    GaussTaps g;
    memset(&g, 0, sizeof g);
    double t[13] = {0.0};
    int r = 1;
    if (f.kind == LBM_FILTER_BINOMIAL) {
        t[0] = 0.25; t[1] = 0.5; t[2] = 0.25;
    } else {
        r = 2 * f.scale;
        double sum = 0.0;
        for (int k = -r; k <= r; ++k) {
            t[k + r] = exp(-(double)(k * k) / (2.0 * f.scale * f.scale));
            sum += t[k + r];
        }
        for (int k = 0; k <= 2 * r; ++k) t[k] /= sum;
    }
    g.radius = r;
    for (int k = 0; k <= 2 * r; ++k) g.t[k] = (float)t[k];
    for (int k = 0; k <= 4 * r; ++k) {
        double c = 0.0;
        for (int i = 0; i <= 2 * r; ++i)
            if (k - i >= 0 && k - i <= 2 * r) c += t[i] * t[k - i];
        g.c[k] = (float)c;
    }
    return g;
}

// R R of a Gaussian / binomial filter through launch_gauss_rr (3-D fields)
static bool gauss_rr_path(const Params& p, const Filter& f) {
    if (p.dim != 3 || (f.kind != LBM_FILTER_GAUSS && f.kind != LBM_FILTER_BINOMIAL)) return false;
    return launch_gauss_rr_supported(f.kind == LBM_FILTER_BINOMIAL ? 1 : 2 * f.scale);
}

static Taps binom_taps() {
    Taps t;
    memset(&t, 0, sizeof t);
    t.radius = 1;
    t.t[0] = 0.25f; t.t[1] = 0.5f; t.t[2] = 0.25f;
    return t;
}

// ---------------------------------------------------------- step sequence --
struct Launcher {
    lbm_ctx* c;
    cudaStream_t s;
    bool count_only;
    long long n;
    cudaError_t err = cudaSuccess;
    bool timed;
    void before(int cls) {
        ++n;
        if (timed && c->ev_used < 96) {
            c->ev_class[c->ev_used] = cls;
            cudaEventRecord(c->ev[2 * c->ev_used], s);
        }
    }
    void check(cudaError_t e) {
        if (e != cudaSuccess && err == cudaSuccess) err = e;
    }
    void after(cudaError_t e) {
        check(e);
        if (timed && c->ev_used < 96) {
            cudaEventRecord(c->ev[2 * c->ev_used + 1], s);
            ++c->ev_used;
        }
    }
};

// a library call (cuFFT): timed like a kernel, not counted as one of ours
#define LIBCALL(lc, cls, expr)                                       \
    do {                                                             \
        if (g_rec) rec_refuse("library call in the step");          \
        else if (!(lc).count_only) {                                 \
            const int n_ = (int)(lc).n;                              \
            (lc).before(cls);                                        \
            (lc).n = n_;                                             \
            (lc).after((expr) == CUFFT_SUCCESS ? cudaSuccess : cudaErrorUnknown); \
        }                                                            \
    } while (0)

#define LAUNCH(lc, cls, expr)              \
    do {                                   \
        (lc).before(cls);                  \
        if (!(lc).count_only) (lc).after(expr); \
    } while (0)

// taps of one application of a separable filter per output: G/B d(2R+1);
// L_s d x (5 s arm + (d-1) s box taps, the box omitted when s = 1)
static double filter_taps(const Filter& f, int d) {
    if (f.kind == LBM_FILTER_FOURIER) return 0.0;  // transforms, counted separately
    if (f.kind == LBM_FILTER_GAUSS) return d * (2.0 * (d == 2 ? 4 : 2) * f.scale + 1.0);
    if (f.kind == LBM_FILTER_BINOMIAL) return d * 3.0;
    // L_s = c B_s * C_s: the (4d + 1)-point cross at stride s plus the
    // separable s^d box (d factors of s taps), the factorised form the 3-D
    // kernel evaluates
    return 4.0 * d + 1.0 + (f.scale > 1 ? (double)d * f.scale : 0.0);
}

static void enqueue_filter(Launcher& lc, const Filter& f, int slot, const float* in, float* out) {
    lbm_ctx* c = lc.c;
    const Params& p = c->p;
    const int nc = p.ncomp;
    const int d = p.dim;
    float* t1 = c->L.t1;
    float* t2 = c->L.t2;
    const double flops = 2.0 * filter_taps(f, d) * nc * (double)p.n;
    if (d == 3 && f.kind == LBM_FILTER_LAPLACE && launch_lap3_supported(f.scale)) {
        // fused 3-D kernels: the whole filter in one pass over the field (for
        // L_3 with nx % 4 == 0 in the factorised form c C_3 * B_3)
        const float scale = (float)(1.0 / (8.0 * d * (double)f.scale * f.scale * f.scale));
        const double n = (double)nc * (double)p.n;
        if (lap3_split(p, f.scale)) {
            if (lc.count_only) c->filter_flops[LBM_K_LAP3] += flops;
            LAUNCH(lc, LBM_K_LAP3, launch_lap3_fused(p, in, out, nc, scale, p.tune.filter_per_sm[slot], lc.s));
            return;
        }
        if (lc.count_only) c->filter_flops[LBM_K_LAP1] += flops;
        LAUNCH(lc, LBM_K_LAP1,
               launch_lap3(p, in, out, nc, f.scale, ell_taps(f.scale), scale, 0, p.tune.filter_per_sm[slot], lc.s));
        return;
    }
    if (lc.count_only) c->filter_flops[LBM_K_FILTER] += flops;
    if (d == 2 && !p.walls) {
        // doubly periodic 2-D: one fused launch when a specialised kernel exists
        const bool lap = f.kind == LBM_FILTER_LAPLACE;
        const Taps t = lap ? ell_taps(f.scale) : (f.kind == LBM_FILTER_GAUSS ? gauss_taps(f.scale, d) : binom_taps());
        const float sc = lap ? (float)(1.0 / (8.0 * d * (double)f.scale * f.scale)) : 1.f;
        const bool ok = lap ? (f.scale == 1 && t.radius == 2)
                            : (t.radius == 1 || t.radius == 4 || t.radius == 12);
        if (ok) {
            LAUNCH(lc, LBM_K_FILTER, launch_filter2_fused(p, in, out, nc, lap, f.scale, t, sc, 0, lc.s));
            return;
        }
    }
    if (f.kind == LBM_FILTER_GAUSS || f.kind == LBM_FILTER_BINOMIAL) {
        const Taps t = f.kind == LBM_FILTER_GAUSS ? gauss_taps(f.scale, d) : binom_taps();
        if (d == 2) {
            LAUNCH(lc, LBM_K_FILTER, launch_pass(p, in, t1, nc, 0, t, 1.f, 0, lc.s));
            LAUNCH(lc, LBM_K_FILTER, launch_pass(p, t1, out, nc, 1, t, 1.f, 0, lc.s));
        } else {
            LAUNCH(lc, LBM_K_FILTER, launch_pass(p, in, t1, nc, 0, t, 1.f, 0, lc.s));
            LAUNCH(lc, LBM_K_FILTER, launch_pass(p, t1, t2, nc, 1, t, 1.f, 0, lc.s));
            LAUNCH(lc, LBM_K_FILTER, launch_pass(p, t2, out, nc, 2, t, 1.f, 0, lc.s));
        }
        return;
    }
    // Laplacian high-pass: sum of d separable terms
    const int s = f.scale;
    double sd = 1.0;
    for (int a = 0; a < d; ++a) sd *= s;
    const float scale = (float)(1.0 / (8.0 * d * sd));
    const Taps el = ell_taps(s);
    const Taps bx = box_taps(s);
    for (int a = 0; a < d; ++a) {
        const int acc = a > 0;
        if (s == 1) {
            LAUNCH(lc, LBM_K_FILTER, launch_pass(p, in, out, nc, a, el, scale, acc, lc.s));
            continue;
        }
        int others[2], no = 0;
        for (int b = 0; b < d; ++b)
            if (b != a) others[no++] = b;
        const float* src = in;
        float* bufs[2] = {t1, t2};
        for (int k = 0; k < no; ++k) {
            LAUNCH(lc, LBM_K_FILTER, launch_pass(p, src, bufs[k], nc, others[k], bx, 1.f, 0, lc.s));
            src = bufs[k];
        }
        LAUNCH(lc, LBM_K_FILTER, launch_pass(p, src, out, nc, a, el, scale, acc, lc.s));
    }
}

// curl, filters, sensitivities and the block reduction of the velocity in
// x6: the QoI/Gram part of the TO phase
static void enqueue_fields(Launcher& lc) {
    lbm_ctx* c = lc.c;
    const Params& p = c->p;
    const Layout& L = c->L;
    LAUNCH(lc, LBM_K_CURL, launch_to_curl(p, L, lc.s));
    if (c->has_fft) {
        // one forward transform of (v_x, v_y, omega) serves every Fourier band
        LIBCALL(lc, LBM_K_FFT, (cufftSetStream(c->fft_r2c, lc.s), cufftExecR2C(c->fft_r2c, (cufftReal*)L.x6, (cufftComplex*)L.spec)));
    }
    for (size_t f = 0; f < c->filters.size(); ++f) {
        const Filter& fl = c->filters[f];
        if (fl.kind == LBM_FILTER_FOURIER) {
            // a sharp band is a projection, R R = R: one masked inverse transform
            LAUNCH(lc, LBM_K_FILTER, launch_band_mask(p, L.spec, L.spec_band, 3, fl.scale, fl.hi, lc.s));
            LIBCALL(lc, LBM_K_FFT, (cufftSetStream(c->fft_c2r, lc.s),
                                    cufftExecC2R(c->fft_c2r, (cufftComplex*)L.spec_band, (cufftReal*)L.rr[f])));
        } else if (gauss_rr_path(p, fl)) {
            // R R in three streaming passes with the composite kernel t * t
            const GaussTaps gt = gauss_pair_taps(fl);
            if (lc.count_only) {
                const double fl1 = 2.0 * (4.0 * gt.radius + 1.0) * p.ncomp * (double)p.n;  // one composite pass
                c->filter_flops[LBM_K_GAUSS_X] += fl1;
                c->filter_flops[LBM_K_GAUSS_Z] += fl1;
                c->filter_flops[LBM_K_GAUSS_Y] += fl1;
            }
            LAUNCH(lc, LBM_K_GAUSS_X, launch_gauss_pass(p, 0, L.x6, L.t1, p.ncomp, gt, L.st, lc.s));
            LAUNCH(lc, LBM_K_GAUSS_Z, launch_gauss_pass(p, 2, L.t1, L.t2, p.ncomp, gt, L.st, lc.s));
            LAUNCH(lc, LBM_K_GAUSS_Y, launch_gauss_pass(p, 1, L.t2, L.rr[f], p.ncomp, gt, L.st, lc.s));
        } else {
            enqueue_filter(lc, fl, (int)f, L.x6, L.acc);
            enqueue_filter(lc, fl, (int)f, L.acc, L.rr[f]);
        }
        if (fl.need_z) LAUNCH(lc, LBM_K_SENS, launch_sens_curl(p, L.rr[f] + (size_t)p.dim * p.n, L.vz[f], lc.s));
    }
    const float* vk[kMaxQoi];
    for (int k = 0; k < p.n_s; ++k) {
        const int slot = p.qoi_filter_slot[k];
        vk[k] = p.qoi_kind[k] == LBM_QOI_ENERGY ? L.rr[slot] : L.vz[slot];
    }
    LAUNCH(lc, LBM_K_REDUCE, launch_reduce(p, L, vk, lc.s));
}

// One time step from f[src] into f[1 - src].  TO modes: the predictor pass
// (v^{p*}, and the post-stream velocity for WALE), the QoI/Gram fields, totals
// and the solve, then the stream-collide with the SGS corrector applied in
// registers before the store (Eq. LES-2), so the predictor populations are
// never written.  Substrate-only runs: the collide (after the velocity pass
// WALE needs).
static void enqueue_step(Launcher& lc, int src) {
    lbm_ctx* c = lc.c;
    const Params& p = c->p;
    const Layout& L = c->L;
    // LRS history matvec and the step's normals: inputs from the previous
    // step only, so they run on a branch beside the field kernels and join
    // before the solve (in line when the kernels are timed one by one)
    const bool pre = p.to_mode == LBM_TO_LRS || p.to_mode == LBM_TO_GAMMA;
    const bool fork = pre && c->branch && !lc.timed && !lc.count_only;
    if (fork) {
        lc.check(cudaEventRecord(c->ev_fork, lc.s));
        lc.check(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
        LAUNCH(lc, LBM_K_LRS, launch_lrs_pre(p, L, c->side));
        lc.check(cudaEventRecord(c->ev_join, c->side));
    }
    if (p.to_mode != LBM_TO_OFF || p.substrate == LBM_SUBSTRATE_WALE)
        LAUNCH(lc, LBM_K_MOMENTS, launch_predict(p, L, src, lc.s));
    if (p.to_mode != LBM_TO_OFF) {
        if (pre && !fork) LAUNCH(lc, LBM_K_LRS, launch_lrs_pre(p, L, lc.s));
        enqueue_fields(lc);
        if (fork) lc.check(cudaStreamWaitEvent(lc.s, c->ev_join, 0));
        LAUNCH(lc, LBM_K_TOTALS, launch_totals(p, L, true, lc.s));
        LAUNCH(lc, LBM_K_SOLVE, launch_solve(p, L, lc.s));
    }
    LAUNCH(lc, LBM_K_COLLIDE, launch_collide(p, L, src, lc.s));
}

static void count_launches(lbm_ctx* c) {
    for (int k = 0; k < LBM_K_COUNT; ++k) c->filter_flops[k] = 0.0;
    Launcher lc{c, c->stream, true, 0};
    lc.timed = false;
    enqueue_step(lc, 0);
    c->launches_per_step = lc.n;
}

static int build_graph(lbm_ctx* c) {
    if (c->graph) return LBM_OK;
    CK(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    Launcher lc{c, c->cap_stream, false, 0};
    lc.timed = false;
    enqueue_step(lc, 0);
    enqueue_step(lc, 1);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
    if (lc.err != cudaSuccess || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return fail(c, LBM_ERR_CUDA, "graph capture failed: %s",
                    cudaGetErrorString(lc.err != cudaSuccess ? lc.err : e));
    }
    e = cudaGraphInstantiate(&c->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        c->graph = nullptr;
        return fail(c, LBM_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
    }
    return LBM_OK;
}


static int eager_step(lbm_ctx* c) {
    Launcher lc{c, c->stream, false, 0};
    lc.timed = c->profiling != 0;
    c->ev_used = 0;
    enqueue_step(lc, c->cur);
    if (lc.err != cudaSuccess) return fail(c, LBM_ERR_CUDA, "kernel launch: %s", cudaGetErrorString(lc.err));
    c->cur = 1 - c->cur;
    if (lc.timed) {
        CK(c, cudaEventSynchronize(c->ev[2 * (c->ev_used - 1) + 1]));
        for (int i = 0; i < c->ev_used; ++i) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, c->ev[2 * i], c->ev[2 * i + 1]);
            c->prof_ms[c->ev_class[i]] += ms;
            c->prof_n[c->ev_class[i]] += 1;
        }
    }
    return LBM_OK;
}

// ------------------------------------------------------ host-side tables --
// Mean-profile band weights (Eq. 3d-mp-band-weights) on fluid rows 1..ny-2:
// d_w = min(y - 1/2, 2H - (y - 1/2)), H = (ny - 2)/2; centres log-spaced from
// 0.5 to H; sigma = spacing of ln(centre); each band sums to 1 over fluid rows.
static void band_weights(int ny, int nb, std::vector<double>* w) {
    w->assign((size_t)nb * ny, 0.0);
    const double h = 0.5 * (ny - 2);
    const double l0 = log(0.5), l1 = log(h);
    const double sig = (l1 - l0) / (nb - 1);
    for (int j = 0; j < nb; ++j) {
        const double lc = l0 + (l1 - l0) * j / (nb - 1);
        double sum = 0.0;
        for (int y = 1; y <= ny - 2; ++y) {
            const double yw = y - 0.5;
            const double dw = yw < 2.0 * h - yw ? yw : 2.0 * h - yw;
            const double e = (log(dw) - lc) / sig;
            (*w)[(size_t)j * ny + y] = exp(-0.5 * e * e);
            sum += (*w)[(size_t)j * ny + y];
        }
        for (int y = 1; y <= ny - 2; ++y) (*w)[(size_t)j * ny + y] /= sum;
    }
}

template <typename T> static float to_f(T v);
template <> float to_f<float>(float v) { return v; }
template <> float to_f<__half>(__half v) { return __half2float(v); }
template <> float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

static const double kW2[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
static double lat_w(int dim, int i) {
    if (dim == 2) return kW2[i];
    return i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0);
}

static int sync_check(lbm_ctx* c) {
    CK(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

template <typename T>
static void widen(const std::vector<char>& raw, int dim, int q, size_t N, double* f) {
    const T* g = (const T*)raw.data();
    for (int i = 0; i < q; ++i)
        for (size_t n = 0; n < N; ++n) f[(size_t)i * N + n] = lat_w(dim, i) + (double)to_f<T>(g[(size_t)i * N + n]);
}

// coefficient-source arrays in blob order: the LRS model (C, mu, chol(Sigma),
// sigma_ref) or the fixed gamma_i; unused entries have zero bytes
static void coef_parts(lbm_ctx* c, void* ptr[4], size_t bytes[4]) {
    const Params& p = c->p;
    const size_t nq = (size_t)p.n_q;
    for (int k = 0; k < 4; ++k) {
        ptr[k] = nullptr;
        bytes[k] = 0;
    }
    if (p.h > 0) {
        ptr[0] = c->L.lrs_C;     bytes[0] = sizeof(double) * ((size_t)(2 * p.h + 1) * nq + 1) * nq;
        ptr[1] = c->L.lrs_mu;    bytes[1] = sizeof(double) * nq;
        ptr[2] = c->L.lrs_L;     bytes[2] = sizeof(double) * nq * nq;
        ptr[3] = c->L.lrs_sigma; bytes[3] = sizeof(double) * nq;
    } else if (p.to_mode == LBM_TO_FIXED_GAMMA) {
        ptr[0] = c->L.gfix;      bytes[0] = sizeof(double) * nq;
    }
}

// checkpoint blob: magic, sizes, DevState, populations, histories, ring, profile, cursor
struct BlobHead {
    uint64_t magic, fbytes, hbytes, rbytes, pbytes, cbytes, tbytes;
    int64_t host_read;
};
static const uint64_t kMagic = 0x4c424d544f303031ULL;

static void blob_sizes(lbm_ctx* c, BlobHead* h) {
    const Params& p = c->p;
    h->magic = kMagic;
    h->fbytes = c->elem * p.q * (size_t)p.n;
    h->hbytes = p.h > 0 ? sizeof(double) * (size_t)p.h * p.n_q : 0;
    h->rbytes = c->L.ring ? sizeof(double) * (size_t)p.ring_cap * p.row_len : 0;
    h->pbytes = c->L.profile ? sizeof(double) * (size_t)p.ny : 0;
    // coefficient source: the LRS model (C, mu, chol(Sigma), sigma_ref, the last
    // possibly set from the first step) or the fixed gamma_i
    void* ptr[4];
    size_t nb[4];
    coef_parts(c, ptr, nb);
    h->cbytes = nb[0] + nb[1] + nb[2] + nb[3];
    h->tbytes = p.track_len > 0 ? sizeof(double) * (size_t)p.track_len * p.n_q : 0;
    h->host_read = c->host_read;
}

// ------------------------------------------------------------- autotuner --
// Launch shapes are chosen by timing the candidates on this context's own
// buffers before the first step (CUDA events on its stream).  Only buffers the
// next step overwrites are written: the other population copy, the TO fields
// and the filter scratch.  Choices are cached per grid shape for the process,
// so every context of a shape (ensemble members included) runs the same kernels.
#include <map>
#include <mutex>
#include <tuple>

namespace {
using TuneKey = std::tuple<int, int, int, int, int, int, int, int, int, int>;
std::mutex g_tune_mu;
std::map<TuneKey, Tune> g_tune_cache;

TuneKey tune_key(const Params& p) {
    return TuneKey(p.dim, p.nx, p.ny, p.nz, p.walls, p.storage, p.substrate, p.to_mode != LBM_TO_OFF, p.n_filters,
                   p.tune.one_seg);
}
}  // namespace

template <typename F>
static float time_ms(lbm_ctx* c, F launch, int reps = 3) {
    launch();  // warm-up
    cudaEvent_t a = c->ev[0], b = c->ev[1];
    cudaEventRecord(a, c->stream);
    for (int r = 0; r < reps; ++r) launch();
    cudaEventRecord(b, c->stream);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    return ms / reps;
}

static int autotune(lbm_ctx* c) {
    Params& p = c->p;
    const TuneKey key = tune_key(p);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            p.tune = it->second;
            c->tuned = 1;
            return LBM_OK;
        }
    }
    const int src = c->cur;
    cudaError_t err = cudaSuccess;
    auto chk = [&](cudaError_t e) { if (e != cudaSuccess && err == cudaSuccess) err = e; };
    // collide: node pairs or single nodes
    if (p.nx % 2 == 0) {
        float best = 1e30f;
        int pick = p.tune.collide_pair;
        for (int v = 0; v <= 1; ++v) {
            p.tune.collide_pair = v;
            const float t = time_ms(c, [&] { chk(launch_collide(p, c->L, src, c->stream)); }, 5);
            if (t < best) { best = t; pick = v; }
        }
        p.tune.collide_pair = pick;
    }
    // predictor pass: node pairs or single nodes
    if (p.nx % 2 == 0 && (p.to_mode != LBM_TO_OFF || p.substrate == LBM_SUBSTRATE_WALE)) {
        float best = 1e30f;
        int pick = p.tune.predict_pair;
        for (int v = 0; v <= 1; ++v) {
            p.tune.predict_pair = v;
            const float t = time_ms(c, [&] { chk(launch_predict(p, c->L, src, c->stream)); }, 5);
            if (t < best) { best = t; pick = v; }
        }
        p.tune.predict_pair = pick;
    }
    if (p.to_mode != LBM_TO_OFF) {
        const int nc = p.ncomp;
        if (p.dim == 3 && !p.tune.one_seg) {
            static const int cand[] = {2, 3, 4, 6, 8, 12, 16};
            for (size_t f = 0; f < c->filters.size() && f < 8; ++f) {
                const Filter& fl = c->filters[f];
                // the Gaussian R R streams have fixed shapes; the fused Laplacian
                // kernels choose their z-segment count
                if (fl.kind != LBM_FILTER_LAPLACE || !launch_lap3_supported(fl.scale)) continue;
                const Taps t0 = ell_taps(fl.scale);
                float best = 1e30f;
                int pick = 0;
                for (int v : cand) {
                    const float t = time_ms(c, [&] {
                        if (lap3_split(p, fl.scale)) {
                            chk(launch_lap3_fused(p, c->L.x6, c->L.acc, nc, 1.f, v, c->stream));
                        } else {
                            chk(launch_lap3(p, c->L.x6, c->L.acc, nc, fl.scale, t0, 1.f, 0, v, c->stream));
                        }
                    }, 5);
                    if (t < best) { best = t; pick = v; }
                }
                p.tune.filter_per_sm[f] = pick;
            }
        } else if (p.dim == 2) {
            // 2-D: the y-axis march of the first compact filter
            const Filter* fp = nullptr;
            for (const Filter& f : c->filters)
                if (!fp && f.kind != LBM_FILTER_FOURIER) fp = &f;
            if (!fp) goto tuned;
            const Filter& fl = *fp;
            const Taps t0 = fl.kind == LBM_FILTER_GAUSS ? gauss_taps(fl.scale, 2)
                            : fl.kind == LBM_FILTER_BINOMIAL ? binom_taps() : ell_taps(fl.scale);
            static const int cand[] = {148 * 256, 148 * 512, 148 * 1024, 148 * 2048, 148 * 4096};
            float best = 1e30f;
            int pick = p.tune.march_lines;
            for (int v : cand) {
                p.tune.march_lines = v;
                const float t = time_ms(c, [&] { chk(launch_pass(p, c->L.x6, c->L.t1, nc, 1, t0, 1.f, 0, c->stream)); });
                if (t < best) { best = t; pick = v; }
            }
            p.tune.march_lines = pick;
        }
    }
tuned:
    if (err != cudaSuccess) return fail(c, LBM_ERR_CUDA, "autotune: %s", cudaGetErrorString(err));
    CK(c, cudaStreamSynchronize(c->stream));
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune_cache[key] = p.tune;
    }
    c->tuned = 1;
    return LBM_OK;
}

// Host-side element loops over whole fields (FP64 <-> FP32 conversion for
// uploads and downloads) split over up to 16 threads: for a 23 M-node field
// a single thread spends longer converting than the GPU spends stepping.
template <typename F>
static void parallel_for(size_t n, F body) {
    unsigned t = std::thread::hardware_concurrency();
    if (t > 16) t = 16;
    if (t < 2 || n < ((size_t)1 << 20)) {
        body((size_t)0, n);
        return;
    }
    std::vector<std::thread> pool;
    const size_t chunk = (n + t - 1) / t;
    for (unsigned k = 0; k < t; ++k) {
        const size_t a = k * chunk, b = a + chunk < n ? a + chunk : n;
        if (a >= b) break;
        pool.emplace_back([=] { body(a, b); });
    }
    for (std::thread& th : pool) th.join();
}

// dst[i] = (float)(src[i] - off) for i in [0, n): the same conversion as the
// scalar loop, with 16-byte non-temporal stores where dst is aligned (the
// staging buffer is written once and read by the DMA engine, so the stores
// skip the cache and its read-for-ownership of every line).
static void f64_to_f32(float* dst, const double* src, size_t n, double off) {
    size_t i = 0;
#if defined(__SSE2__)
    while (i < n && ((uintptr_t)(dst + i) & 15)) {
        dst[i] = (float)(src[i] - off);
        ++i;
    }
    const __m128d o = _mm_set1_pd(off);
    for (; i + 4 <= n; i += 4) {
        const __m128 lo = _mm_cvtpd_ps(_mm_sub_pd(_mm_loadu_pd(src + i), o));
        const __m128 hi = _mm_cvtpd_ps(_mm_sub_pd(_mm_loadu_pd(src + i + 2), o));
        _mm_stream_ps(dst + i, _mm_movelh_ps(lo, hi));
    }
#endif
    for (; i < n; ++i) dst[i] = (float)(src[i] - off);
}

// The context's pinned host staging for whole-field transfers ([4][N]
// floats), allocated on first use for fields of 2^20 nodes or more: a
// pageable copy of a 23 M-node field runs at a fraction of the DMA rate.
// Small fields (ensemble members, admitted while others run) keep a
// temporary pageable buffer, since a pinned allocation may synchronise the
// device.  Also the fallback if pinned memory is refused.
static float* host_stage(lbm_ctx* c, std::unique_ptr<float[]>& fallback) {
    if (!c->hpin && c->p.n >= (1LL << 20)) {
        void* ptr = nullptr;
        if (cudaMallocHost(&ptr, sizeof(float) * 4 * (size_t)c->p.n) == cudaSuccess) c->hpin = (float*)ptr;
        else cudaGetLastError();
    }
    if (c->hpin) return c->hpin;
    fallback.reset(new float[4 * (size_t)c->p.n]);
    return fallback.get();
}

// ================================================================== C ABI ==
extern "C" {

int lbm_qoi_row_len(const lbm_config* cfg, int64_t* len) {
    if (!cfg || !len) return fail(nullptr, LBM_ERR_ARG, "NULL argument");
    *len = 2 + 3 * qoi_count(cfg);
    return LBM_OK;
}

int lbm_required_bytes(const lbm_config* cfg, size_t* bytes) {
    int rc = validate(cfg);
    if (rc) return rc;
    if (!bytes) return fail(nullptr, LBM_ERR_ARG, "bytes is NULL");
    Params p;
    std::vector<Filter> f;
    make_params(cfg, &p, &f);
    float* aux;
    *bytes = carve(cfg, p, f, nullptr, nullptr, &aux);
    return LBM_OK;
}

int lbm_create(const lbm_config* cfg, void* dev_buf, size_t bytes, void* cuda_stream, lbm_ctx** out) {
    int rc = validate(cfg);
    if (rc) return rc;
    if (!out || !dev_buf) return fail(nullptr, LBM_ERR_ARG, "NULL argument");
    if (((uintptr_t)dev_buf & 255) != 0) return fail(nullptr, LBM_ERR_ARG, "dev_buf must be 256-byte aligned");
    lbm_ctx* c = new lbm_ctx();
    memset(c->err, 0, sizeof c->err);
    c->cfg = *cfg;
    make_params(cfg, &c->p, &c->filters);
    const size_t need = carve(cfg, c->p, c->filters, (char*)dev_buf, &c->L, &c->aux);
    if (bytes < need) {
        delete c;
        return fail(nullptr, LBM_ERR_BUDGET, "buffer holds %zu bytes, %zu needed", bytes, need);
    }
    c->stream = (cudaStream_t)cuda_stream;
    c->elem = cfg->storage == LBM_STORAGE_FP32 ? 4 : 2;
    c->use_graphs = 1;
    c->branch = 1;
    c->autotune = 1;
    c->has_fft = c->L.spec != nullptr;
    if (c->has_fft) {
        int n[2], rin[2], co[2];
        fft_dims(c->p, n, rin, co);
        const int idist = c->p.ny * c->p.nx, odist = c->p.ny * (c->p.nx / 2 + 1);
        size_t w1 = 0, w2 = 0;
        const size_t avail = fft_work_bytes(c->p);
        bool ok = cufftCreate(&c->fft_r2c) == CUFFT_SUCCESS && cufftCreate(&c->fft_c2r) == CUFFT_SUCCESS &&
                  cufftSetAutoAllocation(c->fft_r2c, 0) == CUFFT_SUCCESS &&
                  cufftSetAutoAllocation(c->fft_c2r, 0) == CUFFT_SUCCESS &&
                  cufftMakePlanMany(c->fft_r2c, 2, n, rin, 1, idist, co, 1, odist, CUFFT_R2C, 3, &w1) == CUFFT_SUCCESS &&
                  cufftMakePlanMany(c->fft_c2r, 2, n, co, 1, odist, rin, 1, idist, CUFFT_C2R, 3, &w2) == CUFFT_SUCCESS;
        ok = ok && w1 <= avail && w2 <= avail && cufftSetWorkArea(c->fft_r2c, c->L.fft_work) == CUFFT_SUCCESS &&
             cufftSetWorkArea(c->fft_c2r, c->L.fft_work) == CUFFT_SUCCESS;
        if (!ok) {
            delete c;
            return fail(nullptr, LBM_ERR_CUDA, "cuFFT plan set-up failed (work area %zu/%zu of %zu bytes)", w1, w2, avail);
        }
    }
    cudaError_t e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete c;
        return fail(nullptr, LBM_ERR_CUDA, "cudaStreamCreate: %s", cudaGetErrorString(e));
    }
    e = cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        lbm_destroy(c);
        return fail(nullptr, LBM_ERR_CUDA, "stream/event create: %s", cudaGetErrorString(e));
    }
    for (int i = 0; i < 2 * 96; ++i) cudaEventCreate(&c->ev[i]);
    // zero everything (rest state: shifted populations g = 0), then tables
    e = cudaMemsetAsync(dev_buf, 0, need, c->stream);
    std::vector<float> kol(cfg->ny);
    for (int y = 0; y < cfg->ny; ++y)
        kol[y] = (float)(cfg->kolmo_amp * sin(2.0 * M_PI * cfg->kolmo_k * (double)y / cfg->ny));
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->L.kolmo, kol.data(), sizeof(float) * cfg->ny, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && c->p.n_mp > 0) {
        std::vector<double> w;
        band_weights(cfg->ny, c->p.n_mp, &w);
        std::vector<double> g((size_t)c->p.n_mp * c->p.n_mp);
        const double area = (double)cfg->nx * cfg->nz;
        for (int i = 0; i < c->p.n_mp; ++i)
            for (int j = 0; j < c->p.n_mp; ++j) {
                double a = 0.0;
                for (int y = 0; y < cfg->ny; ++y) a += w[(size_t)i * cfg->ny + y] * w[(size_t)j * cfg->ny + y];
                g[(size_t)i * c->p.n_mp + j] = area * a;
            }
        e = cudaMemcpyAsync(c->L.w_mp, w.data(), sizeof(double) * w.size(), cudaMemcpyHostToDevice, c->stream);
        std::vector<float2> w2(w.size());
        for (size_t i = 0; i < w.size(); ++i) {
            w2[i].x = (float)w[i];
            w2[i].y = (float)(w[i] - (double)w2[i].x);
        }
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(c->L.w_mp2, w2.data(), sizeof(float2) * w2.size(), cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(c->L.g_mpmp, g.data(), sizeof(double) * g.size(), cudaMemcpyHostToDevice, c->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        lbm_destroy(c);
        return fail(nullptr, LBM_ERR_CUDA, "create: %s", cudaGetErrorString(e));
    }
    count_launches(c);
    *out = c;
    return LBM_OK;
}

int lbm_destroy(lbm_ctx* c) {
    if (!c) return LBM_OK;
    cudaStreamSynchronize(c->stream);
    if (c->graph) cudaGraphExecDestroy(c->graph);
    for (int i = 0; i < 2 * 96; ++i)
        if (c->ev[i]) cudaEventDestroy(c->ev[i]);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->hpin) cudaFreeHost(c->hpin);
    if (c->side) {
        cudaStreamSynchronize(c->side);
        cudaStreamDestroy(c->side);
    }
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->has_fft) {
        cufftDestroy(c->fft_r2c);
        cufftDestroy(c->fft_c2r);
    }
    delete c;
    return LBM_OK;
}

int lbm_last_error(const lbm_ctx* c, char* buf, size_t len) {
    if (!buf || len == 0) return LBM_ERR_ARG;
    snprintf(buf, len, "%s", c ? c->err : g_err);
    return LBM_OK;
}

static int reset_counters(lbm_ctx* c) {
    const Params& p = c->p;
    DevState st;
    memset(&st, 0, sizeof st);
    if (p.h > 0) {
        // keep the LRS history position
        CK(c, cudaMemcpyAsync(&st, c->L.st, sizeof st, cudaMemcpyDeviceToHost, c->stream));
        CK(c, cudaStreamSynchronize(c->stream));
        const long long hp = st.hist_pos;
        memset(&st, 0, sizeof st);
        st.hist_pos = hp;
    }
    CK(c, cudaMemcpyAsync(c->L.st, &st, sizeof st, cudaMemcpyHostToDevice, c->stream));
    if (c->L.ring) CK(c, cudaMemsetAsync(c->L.ring, 0, sizeof(double) * p.ring_cap * p.row_len, c->stream));
    if (c->L.profile) CK(c, cudaMemsetAsync(c->L.profile, 0, sizeof(double) * p.ny, c->stream));
    c->host_read = 0;
    return LBM_OK;
}

int lbm_init_macros(lbm_ctx* c, const double* rho, const double* u) {
    if (!c || !u) return fail(c, LBM_ERR_ARG, "NULL argument");
    const size_t N = (size_t)c->p.n;
    std::unique_ptr<float[]> tmp;
    float* hp = host_stage(c, tmp);
    // without a density field its slot is zeroed on the device (a quarter of
    // the upload saved)
    if (!rho) CK(c, cudaMemsetAsync(c->aux, 0, sizeof(float) * N, c->stream));
    // every conversion thread queues the copy of each 1 MB piece it has
    // written, so the DMA of one piece overlaps the conversion of the next
    // (worker threads select the caller's device first)
    int dev = 0;
    CK(c, cudaGetDevice(&dev));
    std::atomic<int> err{0};
    parallel_for(N, [&](size_t a, size_t b) {
        if (cudaSetDevice(dev) != cudaSuccess) {
            err.store((int)cudaErrorInvalidDevice);
            return;
        }
        constexpr size_t kPiece = (size_t)1 << 18;
        for (size_t q0 = a; q0 < b; q0 += kPiece) {
            const size_t q1 = q0 + kPiece < b ? q0 + kPiece : b;
            if (rho) f64_to_f32(hp + q0, rho + q0, q1 - q0, 1.0);
            for (int k = 0; k < 3; ++k) f64_to_f32(hp + (k + 1) * N + q0, u + k * N + q0, q1 - q0, 0.0);
#if defined(__SSE2__)
            _mm_sfence();  // the streamed stores are visible before the copy is queued
#endif
            for (int sl = rho ? 0 : 1; sl < 4; ++sl) {
                const cudaError_t e = cudaMemcpyAsync(c->aux + sl * N + q0, hp + sl * N + q0, sizeof(float) * (q1 - q0),
                                                      cudaMemcpyHostToDevice, c->stream);
                if (e != cudaSuccess) {
                    int none = 0;
                    err.compare_exchange_strong(none, (int)e);
                }
            }
        }
    });
    if (err.load()) CK(c, (cudaError_t)err.load());
    c->cur = 0;
    CK(c, launch_init_feq(c->p, c->L, c->aux, c->aux + N, 0, c->stream));
    int rc = reset_counters(c);
    if (rc) return rc;
    return sync_check(c);
}

int lbm_set_lrs(lbm_ctx* c, const double* C, const double* mu, const double* Sigma, const double* sigma_ref,
                const double* q_hist, const double* qs_hist) {
    if (!c) return fail(c, LBM_ERR_ARG, "NULL context");
    const Params& p = c->p;
    if (p.to_mode != LBM_TO_LRS) return fail(c, LBM_ERR_STATE, "lbm_set_lrs needs to_mode LBM_TO_LRS");
    if (!C || !mu || !Sigma || !sigma_ref) return fail(c, LBM_ERR_ARG, "NULL coefficient array");
    const int n = p.n_q;
    for (int i = 0; i < n; ++i) {
        if (!(sigma_ref[i] == sigma_ref[i])) return fail(c, LBM_ERR_ARG, "sigma_ref[%d] is NaN", i);
        if (sigma_ref[i] <= 0.0 && (q_hist || qs_hist || p.spinup > 0))
            return fail(c, LBM_ERR_ARG, "sigma_ref <= 0 (taken from the first step) needs zero initial histories and no spin-up");
    }
    // Cholesky of Sigma (symmetric positive definite required)
    std::vector<double> Lh((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            if (fabs(Sigma[i * n + j] - Sigma[j * n + i]) > 1e-12 * (fabs(Sigma[i * n + j]) + fabs(Sigma[j * n + i])) + 1e-300)
                return fail(c, LBM_ERR_ARG, "Sigma is not symmetric");
    for (int k = 0; k < n; ++k) {
        double d = Sigma[k * n + k];
        for (int m = 0; m < k; ++m) d -= Lh[k * n + m] * Lh[k * n + m];
        if (!(d > 0.0)) return fail(c, LBM_ERR_ARG, "Sigma is not positive definite");
        Lh[k * n + k] = sqrt(d);
        for (int i = k + 1; i < n; ++i) {
            double a = Sigma[i * n + k];
            for (int m = 0; m < k; ++m) a -= Lh[i * n + m] * Lh[k * n + m];
            Lh[i * n + k] = a / Lh[k * n + k];
        }
    }
    const size_t rows = (size_t)(2 * p.h + 1) * n + 1;
    CK(c, cudaMemcpyAsync(c->L.lrs_C, C, sizeof(double) * rows * n, cudaMemcpyHostToDevice, c->stream));
    CK(c, cudaMemcpyAsync(c->L.lrs_mu, mu, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
    CK(c, cudaMemcpyAsync(c->L.lrs_L, Lh.data(), sizeof(double) * n * n, cudaMemcpyHostToDevice, c->stream));
    CK(c, cudaMemcpyAsync(c->L.lrs_sigma, sigma_ref, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
    // ring slot of q^{n-k} is (pos - k) mod h with pos = 0
    std::vector<double> qh((size_t)p.h * n, 0.0), qsh((size_t)p.h * n, 0.0);
    for (int k = 1; k <= p.h; ++k)
        for (int i = 0; i < n; ++i) {
            const size_t slot = (size_t)(p.h - k);
            if (q_hist) qh[slot * n + i] = q_hist[(size_t)(k - 1) * n + i];
            if (qs_hist) qsh[slot * n + i] = qs_hist[(size_t)(k - 1) * n + i];
        }
    CK(c, cudaMemcpyAsync(c->L.qh, qh.data(), sizeof(double) * qh.size(), cudaMemcpyHostToDevice, c->stream));
    CK(c, cudaMemcpyAsync(c->L.qsh, qsh.data(), sizeof(double) * qsh.size(), cudaMemcpyHostToDevice, c->stream));
    DevState st;
    CK(c, cudaMemcpyAsync(&st, c->L.st, sizeof st, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    st.hist_pos = 0;
    CK(c, cudaMemcpyAsync(c->L.st, &st, sizeof st, cudaMemcpyHostToDevice, c->stream));
    c->lrs_set = 1;
    return sync_check(c);
}

int lbm_set_to_coeffs(lbm_ctx* c, int mode, int32_t h, const double* C, const double* mu, const double* Sigma,
                      const double* sigma_ref, const double* gamma_fixed) {
    if (!c) return fail(c, LBM_ERR_ARG, "NULL context");
    const Params& p = c->p;
    if (mode < LBM_TO_OFF || mode > LBM_TO_FIXED_GAMMA) return fail(c, LBM_ERR_ARG, "bad mode %d", mode);
    if (mode != p.to_mode)
        return fail(c, LBM_ERR_STATE, "the context was created for to_mode %d, not %d", p.to_mode, mode);
    if (mode == LBM_TO_LRS) {
        if (h != p.h) return fail(c, LBM_ERR_ARG, "h = %d, the context holds h = %d", (int)h, p.h);
        return lbm_set_lrs(c, C, mu, Sigma, sigma_ref, nullptr, nullptr);
    }
    if (mode == LBM_TO_FIXED_GAMMA) {
        if (!gamma_fixed) return fail(c, LBM_ERR_ARG, "gamma_fixed is NULL");
        for (int i = 0; i < p.n_q; ++i)
            if (!isfinite(gamma_fixed[i])) return fail(c, LBM_ERR_ARG, "gamma_fixed[%d] is not finite", i);
        CK(c, cudaMemcpyAsync(c->L.gfix, gamma_fixed, sizeof(double) * p.n_q, cudaMemcpyHostToDevice, c->stream));
        c->fixed_set = 1;
        return sync_check(c);
    }
    return LBM_OK;
}

int lbm_set_track_reference(lbm_ctx* c, const double* qref, int64_t len) {
    if (!c || !qref) return fail(c, LBM_ERR_ARG, "NULL argument");
    if (c->p.track_len < 1) return fail(c, LBM_ERR_STATE, "needs LBM_TO_TRACK or an LRS spin-up (track_len >= 1)");
    if (len < 1 || len > c->p.track_len) return fail(c, LBM_ERR_ARG, "len must be in 1..track_len");
    std::vector<double> buf((size_t)c->p.track_len * c->p.n_q);
    for (long long r = 0; r < c->p.track_len; ++r)
        for (int i = 0; i < c->p.n_q; ++i)
            buf[(size_t)r * c->p.n_q + i] = qref[(size_t)(r < len ? r : len - 1) * c->p.n_q + i];
    CK(c, cudaMemcpyAsync(c->L.track, buf.data(), sizeof(double) * buf.size(), cudaMemcpyHostToDevice, c->stream));
    return sync_check(c);
}

}  // extern "C"

namespace lbm {
// Batched execution (lbm_batch.cu): the checks and the tuning lbm_step does
// before a context's first step, then the launch programs of one step from
// each population buffer.  A program whose launches cannot all be batched
// comes back with ok == false (the member then steps on its own).
int record_step_programs(lbm_ctx* c, Recorder prog[2]) {
    if (!c) return fail(c, LBM_ERR_ARG, "NULL context");
    if (c->p.to_mode == LBM_TO_LRS && !c->lrs_set) return fail(c, LBM_ERR_STATE, "call lbm_set_lrs or lbm_set_to_coeffs first");
    if (c->p.to_mode == LBM_TO_FIXED_GAMMA && !c->fixed_set)
        return fail(c, LBM_ERR_STATE, "call lbm_set_to_coeffs with gamma_fixed first");
    if (c->autotune && !c->tuned) {
        const int rc = autotune(c);
        if (rc) return rc;
    }
    for (int par = 0; par < 2; ++par) {
        prog[par] = Recorder();
        if (c->profiling || c->branch) {
            prog[par].ok = false;
            prog[par].why = c->profiling ? "profiling" : "branched step";
            continue;
        }
        Launcher lc{c, c->stream, false, 0};
        lc.timed = false;
        g_rec = &prog[par];
        enqueue_step(lc, par);
        g_rec = nullptr;
        if (lc.err != cudaSuccess) return fail(c, LBM_ERR_CUDA, "recording a step: %s", cudaGetErrorString(lc.err));
    }
    return LBM_OK;
}
int step_parity(const lbm_ctx* c) { return c->cur; }
void steps_taken(lbm_ctx* c, int64_t n) {
    if (n & 1) c->cur = 1 - c->cur;
}
}  // namespace lbm

extern "C" {

int lbm_step(lbm_ctx* c, int64_t nsteps) {
    if (!c) return fail(c, LBM_ERR_ARG, "NULL context");
    if (nsteps < 0) return fail(c, LBM_ERR_ARG, "nsteps < 0");
    if (c->p.to_mode == LBM_TO_LRS && !c->lrs_set) return fail(c, LBM_ERR_STATE, "call lbm_set_lrs or lbm_set_to_coeffs first");
    if (c->p.to_mode == LBM_TO_FIXED_GAMMA && !c->fixed_set)
        return fail(c, LBM_ERR_STATE, "call lbm_set_to_coeffs with gamma_fixed first");
    if (c->autotune && !c->tuned && nsteps > 0) {
        const int rc = autotune(c);
        if (rc) return rc;
    }
    int64_t left = nsteps;
    const bool graphs = c->use_graphs && !c->profiling;
    if (graphs && left >= 2) {
        if (c->cur == 1) {
            int rc = eager_step(c);
            if (rc) return rc;
            --left;
        }
        if (left >= 2) {
            int rc = build_graph(c);
            if (rc) return rc;
            while (left >= 2) {
                CK(c, cudaGraphLaunch(c->graph, c->stream));
                left -= 2;
            }
        }
    }
    while (left > 0) {
        int rc = eager_step(c);
        if (rc) return rc;
        --left;
    }
    CK(c, cudaGetLastError());
    return LBM_OK;
}

int lbm_sync(lbm_ctx* c) {
    if (!c) return fail(c, LBM_ERR_ARG, "NULL context");
    DevState st;
    CK(c, cudaMemcpyAsync(&st, c->L.st, sizeof st, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    if (st.status & 4u)
        return fail(c, LBM_ERR_TIMEOUT, "a kernel's bounded wait for its bulk copies gave up; results are not valid");
    if (st.status & 1u) return fail(c, LBM_ERR_UNSTABLE, "unstable state (non-finite, rho <= 0 or |v| > c_s)");
    return LBM_OK;
}

int lbm_qoi(lbm_ctx* c, double* out, int64_t capacity, int64_t* n_written, int64_t* n_lost) {
    if (!c || !n_written) return fail(c, LBM_ERR_ARG, "NULL argument");
    *n_written = 0;
    if (n_lost) *n_lost = 0;
    const Params& p = c->p;
    if (p.to_mode == LBM_TO_OFF) return LBM_OK;
    DevState st;
    CK(c, cudaMemcpyAsync(&st, c->L.st, sizeof st, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    long long avail = st.ring_count - c->host_read;
    if (avail > p.ring_cap) {
        if (n_lost) *n_lost = avail - p.ring_cap;
        c->host_read = st.ring_count - p.ring_cap;
        avail = p.ring_cap;
    }
    const long long take = avail < capacity ? avail : capacity;
    if (take <= 0) return LBM_OK;
    if (!out) return fail(c, LBM_ERR_ARG, "out is NULL");
    std::vector<double> ring((size_t)p.ring_cap * p.row_len);
    CK(c, cudaMemcpyAsync(ring.data(), c->L.ring, sizeof(double) * ring.size(), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    for (long long r = 0; r < take; ++r) {
        const long long src = (c->host_read + r) % p.ring_cap;
        memcpy(out + (size_t)r * p.row_len, ring.data() + (size_t)src * p.row_len, sizeof(double) * p.row_len);
    }
    c->host_read += take;
    *n_written = take;
    return LBM_OK;
}

int lbm_get_macros(lbm_ctx* c, double* rho, double* u) {
    if (!c || !rho || !u) return fail(c, LBM_ERR_ARG, "NULL argument");
    const size_t N = (size_t)c->p.n;
    CK(c, launch_macros(c->p, c->L, c->cur, c->aux, c->aux + N, c->stream));
    std::unique_ptr<float[]> tmp;
    float* hp = host_stage(c, tmp);
    CK(c, cudaMemcpyAsync(hp, c->aux, sizeof(float) * 4 * N, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    parallel_for(N, [&](size_t a, size_t b) {
        for (size_t i = a; i < b; ++i) {
            rho[i] = 1.0 + (double)hp[i];
            u[i] = (double)hp[N + i];
            u[N + i] = (double)hp[2 * N + i];
            u[2 * N + i] = (double)hp[3 * N + i];
        }
    });
    return LBM_OK;
}

int lbm_get_populations(lbm_ctx* c, double* f) {
    if (!c || !f) return fail(c, LBM_ERR_ARG, "NULL argument");
    const size_t N = (size_t)c->p.n;
    std::vector<char> raw(c->elem * c->p.q * N);
    CK(c, cudaMemcpyAsync(raw.data(), c->L.f[c->cur], raw.size(), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    if (c->p.storage == LBM_STORAGE_FP16) widen<__half>(raw, c->p.dim, c->p.q, N, f);
    else if (c->p.storage == LBM_STORAGE_BF16) widen<__nv_bfloat16>(raw, c->p.dim, c->p.q, N, f);
    else widen<float>(raw, c->p.dim, c->p.q, N, f);
    return LBM_OK;
}

int lbm_set_populations(lbm_ctx* c, const double* f) {
    if (!c || !f) return fail(c, LBM_ERR_ARG, "NULL argument");
    const size_t N = (size_t)c->p.n;
    const int q = c->p.q;
    std::vector<char> raw(c->elem * q * N);
    for (int i = 0; i < q; ++i)
        for (size_t n = 0; n < N; ++n) {
            const double g = f[(size_t)i * N + n] - lat_w(c->p.dim, i);
            const size_t k = (size_t)i * N + n;
            if (c->p.storage == LBM_STORAGE_FP16) ((__half*)raw.data())[k] = __float2half_rn((float)g);
            else if (c->p.storage == LBM_STORAGE_BF16) ((__nv_bfloat16*)raw.data())[k] = __float2bfloat16_rn((float)g);
            else ((float*)raw.data())[k] = (float)g;
        }
    CK(c, cudaMemcpyAsync(c->L.f[c->cur], raw.data(), raw.size(), cudaMemcpyHostToDevice, c->stream));
    return sync_check(c);
}

int lbm_get_profile(lbm_ctx* c, double* prof, int64_t* nsteps) {
    if (!c || !prof || !nsteps) return fail(c, LBM_ERR_ARG, "NULL argument");
    *nsteps = 0;
    if (!c->L.profile) {
        memset(prof, 0, sizeof(double) * c->p.ny);
        return LBM_OK;
    }
    DevState st;
    CK(c, cudaMemcpyAsync(prof, c->L.profile, sizeof(double) * c->p.ny, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaMemcpyAsync(&st, c->L.st, sizeof st, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    *nsteps = st.prof_steps;
    return LBM_OK;
}

int lbm_get_step(lbm_ctx* c, int64_t* step) {
    if (!c || !step) return fail(c, LBM_ERR_ARG, "NULL argument");
    DevState st;
    CK(c, cudaMemcpyAsync(&st, c->L.st, sizeof st, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    *step = st.step;
    return LBM_OK;
}

int lbm_state_bytes(lbm_ctx* c, size_t* bytes) {
    if (!c || !bytes) return fail(c, LBM_ERR_ARG, "NULL argument");
    BlobHead h;
    blob_sizes(c, &h);
    *bytes = sizeof h + sizeof(DevState) + h.fbytes + 2 * h.hbytes + h.rbytes + h.pbytes + h.cbytes + h.tbytes;
    return LBM_OK;
}

int lbm_save(lbm_ctx* c, void* buf, size_t bytes) {
    size_t need = 0;
    int rc = lbm_state_bytes(c, &need);
    if (rc) return rc;
    if (!buf || bytes < need) return fail(c, LBM_ERR_ARG, "checkpoint buffer too small (%zu < %zu)", bytes, need);
    BlobHead h;
    blob_sizes(c, &h);
    char* o = (char*)buf;
    memcpy(o, &h, sizeof h);
    o += sizeof h;
    CK(c, cudaMemcpyAsync(o, c->L.st, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream));
    o += sizeof(DevState);
    CK(c, cudaMemcpyAsync(o, c->L.f[c->cur], h.fbytes, cudaMemcpyDeviceToHost, c->stream));
    o += h.fbytes;
    if (h.hbytes) {
        CK(c, cudaMemcpyAsync(o, c->L.qh, h.hbytes, cudaMemcpyDeviceToHost, c->stream));
        o += h.hbytes;
        CK(c, cudaMemcpyAsync(o, c->L.qsh, h.hbytes, cudaMemcpyDeviceToHost, c->stream));
        o += h.hbytes;
    }
    if (h.rbytes) {
        CK(c, cudaMemcpyAsync(o, c->L.ring, h.rbytes, cudaMemcpyDeviceToHost, c->stream));
        o += h.rbytes;
    }
    if (h.pbytes) {
        CK(c, cudaMemcpyAsync(o, c->L.profile, h.pbytes, cudaMemcpyDeviceToHost, c->stream));
        o += h.pbytes;
    }
    if (h.cbytes) {
        void* ptr[4];
        size_t nb[4];
        coef_parts(c, ptr, nb);
        for (int k = 0; k < 4; ++k) {
            if (!nb[k]) continue;
            CK(c, cudaMemcpyAsync(o, ptr[k], nb[k], cudaMemcpyDeviceToHost, c->stream));
            o += nb[k];
        }
    }
    if (h.tbytes) CK(c, cudaMemcpyAsync(o, c->L.track, h.tbytes, cudaMemcpyDeviceToHost, c->stream));
    return sync_check(c);
}

int lbm_load(lbm_ctx* c, const void* buf, size_t bytes) {
    size_t need = 0;
    int rc = lbm_state_bytes(c, &need);
    if (rc) return rc;
    if (!buf || bytes < need) return fail(c, LBM_ERR_ARG, "checkpoint buffer too small");
    BlobHead h, mine;
    memcpy(&h, buf, sizeof h);
    blob_sizes(c, &mine);
    if (h.magic != kMagic || h.fbytes != mine.fbytes || h.hbytes != mine.hbytes || h.rbytes != mine.rbytes ||
        h.pbytes != mine.pbytes || h.cbytes != mine.cbytes || h.tbytes != mine.tbytes)
        return fail(c, LBM_ERR_ARG, "checkpoint does not match this configuration");
    const char* o = (const char*)buf + sizeof h;
    CK(c, cudaMemcpyAsync(c->L.st, o, sizeof(DevState), cudaMemcpyHostToDevice, c->stream));
    o += sizeof(DevState);
    c->cur = 0;
    CK(c, cudaMemcpyAsync(c->L.f[0], o, h.fbytes, cudaMemcpyHostToDevice, c->stream));
    o += h.fbytes;
    if (h.hbytes) {
        CK(c, cudaMemcpyAsync(c->L.qh, o, h.hbytes, cudaMemcpyHostToDevice, c->stream));
        o += h.hbytes;
        CK(c, cudaMemcpyAsync(c->L.qsh, o, h.hbytes, cudaMemcpyHostToDevice, c->stream));
        o += h.hbytes;
    }
    if (h.rbytes) {
        CK(c, cudaMemcpyAsync(c->L.ring, o, h.rbytes, cudaMemcpyHostToDevice, c->stream));
        o += h.rbytes;
    }
    if (h.pbytes) {
        CK(c, cudaMemcpyAsync(c->L.profile, o, h.pbytes, cudaMemcpyHostToDevice, c->stream));
        o += h.pbytes;
    }
    if (h.cbytes) {
        void* ptr[4];
        size_t nb[4];
        coef_parts(c, ptr, nb);
        for (int k = 0; k < 4; ++k) {
            if (!nb[k]) continue;
            CK(c, cudaMemcpyAsync(ptr[k], o, nb[k], cudaMemcpyHostToDevice, c->stream));
            o += nb[k];
        }
    }
    if (h.tbytes) CK(c, cudaMemcpyAsync(c->L.track, o, h.tbytes, cudaMemcpyHostToDevice, c->stream));
    c->host_read = h.host_read;
    c->lrs_set = c->lrs_set || c->p.h > 0;
    c->fixed_set = c->fixed_set || c->p.to_mode == LBM_TO_FIXED_GAMMA;
    return sync_check(c);
}

int lbm_set_autotune(lbm_ctx* c, int enable) {
    if (!c) return fail(c, LBM_ERR_ARG, "NULL context");
    if (c->graph) return fail(c, LBM_ERR_STATE, "lbm_set_autotune must precede the first lbm_step");
    c->autotune = enable ? 1 : 0;
    return LBM_OK;
}

int lbm_get_tuning(lbm_ctx* c, int32_t* values, int count) {
    if (!c || !values) return fail(c, LBM_ERR_ARG, "NULL argument");
    int32_t v[14] = {c->tuned, c->p.tune.collide_pair, corrector_runs(c->p) ? 1 : 0, c->p.tune.march_lines};
    for (int f = 0; f < 8; ++f) v[4 + f] = c->p.tune.filter_per_sm[f];
    v[12] = c->p.tune.one_seg;
    v[13] = c->p.tune.predict_pair;
    for (int k = 0; k < count && k < 14; ++k) values[k] = v[k];
    return LBM_OK;
}

int lbm_set_launch_goal(lbm_ctx* c, int goal) {
    if (!c) return fail(c, LBM_ERR_ARG, "NULL context");
    if (goal != LBM_GOAL_LATENCY && goal != LBM_GOAL_THROUGHPUT) return fail(c, LBM_ERR_ARG, "bad launch goal %d", goal);
    if (c->graph || c->tuned) return fail(c, LBM_ERR_STATE, "lbm_set_launch_goal must precede the first lbm_step");
    c->p.tune.one_seg = goal == LBM_GOAL_THROUGHPUT ? 1 : 0;
    return LBM_OK;
}

// ------------------------------------------------------ projection phi_m --
static int lf_dims(const lbm_config* c, int m, int32_t d[3]) {
    if (m < 1) return fail(nullptr, LBM_ERR_ARG, "projection factor m must be >= 1");
    if (c->dim == 2) {
        if (c->walls) return fail(nullptr, LBM_ERR_ARG, "2-D projection (bicubic) needs a doubly periodic grid");
        if (c->nx % m || c->ny % m) return fail(nullptr, LBM_ERR_ARG, "%dx%d does not coarsen by m = %d", c->nx, c->ny, m);
        d[0] = c->nx / m; d[1] = c->ny / m; d[2] = 1;
    } else {
        if (!c->walls) return fail(nullptr, LBM_ERR_ARG, "3-D projection (wall-anchored subsampling) needs the channel walls");
        if (m % 2 == 0) return fail(nullptr, LBM_ERR_ARG, "wall-anchored subsampling needs odd m");
        if (c->nx % m || c->nz % m || (c->ny - 2) % m)
            return fail(nullptr, LBM_ERR_ARG, "%dx%dx%d does not coarsen by m = %d", c->nx, c->ny, c->nz, m);
        d[0] = c->nx / m; d[1] = (c->ny - 2) / m + 2; d[2] = c->nz / m;
    }
    if (d[0] < 3 || d[1] < 3 || (c->dim == 3 && (d[1] < 4 || d[2] < 3)))
        return fail(nullptr, LBM_ERR_ARG, "LF grid %dx%dx%d too small", d[0], d[1], d[2]);
    return LBM_OK;
}

int lbm_project_shape(const lbm_config* cfg, int m, int32_t* lf) {
    if (!cfg || !lf) return fail(nullptr, LBM_ERR_ARG, "NULL argument");
    return lf_dims(cfg, m, lf);
}

int lbm_project(lbm_ctx* c, int m, float* drho, float* u) {
    if (!c || !drho || !u) return fail(c, LBM_ERR_ARG, "NULL argument");
    int32_t d[3] = {0, 0, 0};
    const int rc = lf_dims(&c->cfg, m, d);
    if (rc != LBM_OK) return fail(c, rc, "%s", g_err);
    CK(c, launch_project(c->p, c->L, c->cur, m, d[0], d[1], d[2], drho, u, c->stream));
    return LBM_OK;
}

int lbm_eval_qoi(lbm_ctx* c, const float* u, double* q) {
    if (!c || !u || !q) return fail(c, LBM_ERR_ARG, "NULL argument");
    if (c->p.to_mode == LBM_TO_OFF) return fail(c, LBM_ERR_STATE, "lbm_eval_qoi needs a context with QoIs (to_mode != off)");
    Launcher lc{c, c->stream, false, 0};
    lc.timed = false;
    LAUNCH(lc, LBM_K_CURL, launch_load_velocity(c->p, c->L, u, lc.s));
    enqueue_fields(lc);
    LAUNCH(lc, LBM_K_TOTALS, launch_totals(c->p, c->L, false, lc.s));
    LAUNCH(lc, LBM_K_SOLVE, launch_qoi_values(c->p, c->L, q, lc.s));
    if (lc.err != cudaSuccess) return fail(c, LBM_ERR_CUDA, "lbm_eval_qoi: %s", cudaGetErrorString(lc.err));
    return LBM_OK;
}

int lbm_set_branching(lbm_ctx* c, int enable) {
    if (!c) return fail(c, LBM_ERR_ARG, "NULL context");
    if (c->graph) return fail(c, LBM_ERR_STATE, "lbm_set_branching must precede the first lbm_step");
    c->branch = enable ? 1 : 0;
    return LBM_OK;
}

int lbm_set_graphs(lbm_ctx* c, int enable) {
    if (!c) return fail(c, LBM_ERR_ARG, "NULL context");
    c->use_graphs = enable ? 1 : 0;
    return LBM_OK;
}

int lbm_profile(lbm_ctx* c, int enable) {
    if (!c) return fail(c, LBM_ERR_ARG, "NULL context");
    c->profiling = enable ? 1 : 0;
    for (int k = 0; k < LBM_K_COUNT; ++k) {
        c->prof_ms[k] = 0.0;
        c->prof_n[k] = 0;
    }
    return LBM_OK;
}

int lbm_profile_read(lbm_ctx* c, double* ms, int64_t* launches, int count) {
    if (!c || !ms || !launches) return fail(c, LBM_ERR_ARG, "NULL argument");
    for (int k = 0; k < count && k < LBM_K_COUNT; ++k) {
        ms[k] = c->prof_ms[k];
        launches[k] = c->prof_n[k];
    }
    return LBM_OK;
}

int lbm_launches_per_step(lbm_ctx* c, int64_t* launches) {
    if (!c || !launches) return fail(c, LBM_ERR_ARG, "NULL argument");
    *launches = c->launches_per_step;
    return LBM_OK;
}

int lbm_filter_flops_per_step(lbm_ctx* c, double* flops, int count) {
    if (!c || !flops) return fail(c, LBM_ERR_ARG, "NULL argument");
    for (int k = 0; k < count && k < LBM_K_COUNT; ++k) flops[k] = c->filter_flops[k];
    return LBM_OK;
}

}  // extern "C"
