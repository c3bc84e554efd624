// lbm_qoi_eval_static: the scale-aware QoIs of a caller-supplied velocity
// field, computed with the TO-phase kernels on a scratch array that is
// compiled into the library instead of memory the caller allocates.
#include <mutex>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>
#include <math.h>

#include <cuda.h>  // driver types only: the two driver calls below are fetched at run time

#include "lbm_common.cuh"
#include "dfloat.cuh"

using namespace lbm;

namespace {

// The one scratch array.  Its name is only a host-side stand-in in host code;
// the device address comes from cudaGetSymbolAddress, looked up once per CUDA
// context (the primary context of each device, or any other context the
// caller makes current) and cached under the context's unique id, so a
// context created later (after cudaDeviceReset, say) gets its own lookup.
static __device__ __align__(256) unsigned char g_static_scratch[LBM_STATIC_SCRATCH_BYTES];

constexpr int kMaxContexts = 64;
std::mutex g_mu;
struct CtxEntry {
    unsigned long long id;
    void* ptr;
};
CtxEntry g_ctx_cache[kMaxContexts];
int g_nctx = 0;

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

// unique id of the calling thread's current context (0 if none or unknown)
unsigned long long current_context_id() {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = (CtxGetCurrentFn)f;
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = (CtxGetIdFn)f;
    }
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (get_current && get_id && get_current(&c) == CUDA_SUCCESS && c && get_id(c, &id) == CUDA_SUCCESS) return id;
    return 0;
}

int err(int code, const char* fmt, ...) {
    char buf[256];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    set_global_error(buf);
    return code;
}

// velocity components into the stacked field, zero on solid rows
__global__ void masked_copy_kernel(Params p, const float* __restrict__ u, float* __restrict__ x6) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= p.n) return;
    const int y = (n / p.nx) % p.ny;
    const bool solid = p.walls && (y == 0 || y == p.ny - 1);
    for (int a = 0; a < p.dim; ++a) x6[(size_t)a * p.n + n] = solid ? 0.f : u[(size_t)a * p.n + n];
}

// q_k = (1/2) sum over blocks of <v, V_k> (self-adjointness: E_R = <v, RRv>/2,
// Z_R = <v, curl*(RR omega)>/2), one warp per QoI in a fixed order
__global__ void finish_kernel(Params p, const float* __restrict__ part, double* __restrict__ q) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int k = wid; k < p.n_s; k += blockDim.x >> 5) {
        const double a = df_warp_sum(part + k, p.nblk_red, (size_t)p.npart_all, lane);
        if (lane == 0) q[k] = 0.5 * a;
    }
}

struct Filt {
    int kind, scale;
    bool need_z;
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

Taps taps_gauss(int s, int dim) {
    Taps t;
    memset(&t, 0, sizeof t);
    const int alpha = dim == 2 ? 4 : 2;
    t.radius = alpha * s;
    double sum = 0.0;
    for (int r = -t.radius; r <= t.radius; ++r) sum += exp(-(double)(r * r) / (2.0 * s * s));
    for (int r = -t.radius; r <= t.radius; ++r) t.t[r + t.radius] = (float)(exp(-(double)(r * r) / (2.0 * s * s)) / sum);
    return t;
}
Taps taps_ell(int s) {
    static const double ell[5] = {1.0, -4.0, 6.0, -4.0, 1.0};
    Taps t;
    memset(&t, 0, sizeof t);
    t.radius = (5 * s - 1) / 2;
    for (int m = 0; m < 5 * s; ++m) t.t[m] = (float)ell[m / s];
    return t;
}
Taps taps_box(int s) {
    Taps t;
    memset(&t, 0, sizeof t);
    t.radius = (s - 1) / 2;
    for (int m = 0; m < s; ++m) t.t[m] = 1.0f;
    return t;
}

// R applied to `in` (ncomp components) into `out`, through t1/t2
cudaError_t filter(const Params& p, const Filt& f, const float* in, float* out, float* t1, float* t2,
                   cudaStream_t s) {
    const int nc = p.ncomp, d = p.dim;
    cudaError_t e = cudaSuccess;
    if (f.kind == LBM_FILTER_GAUSS || f.kind == LBM_FILTER_BINOMIAL) {
        Taps t;
        if (f.kind == LBM_FILTER_GAUSS) {
            t = taps_gauss(f.scale, d);
        } else {
            memset(&t, 0, sizeof t);
            t.radius = 1;
            t.t[0] = 0.25f; t.t[1] = 0.5f; t.t[2] = 0.25f;
        }
        if (d == 2) {
            if (!e) e = launch_pass(p, in, t1, nc, 0, t, 1.f, 0, s);
            if (!e) e = launch_pass(p, t1, out, nc, 1, t, 1.f, 0, s);
        } else {
            if (!e) e = launch_pass(p, in, t1, nc, 0, t, 1.f, 0, s);
            if (!e) e = launch_pass(p, t1, t2, nc, 1, t, 1.f, 0, s);
            if (!e) e = launch_pass(p, t2, out, nc, 2, t, 1.f, 0, s);
        }
        return e;
    }
    const int sc = f.scale;
    double sd = 1.0;
    for (int a = 0; a < d; ++a) sd *= sc;
    const float scale = (float)(1.0 / (8.0 * d * sd));
    const Taps el = taps_ell(sc), bx = taps_box(sc);
    for (int a = 0; a < d && !e; ++a) {
        const int acc = a > 0;
        if (sc == 1) {
            e = launch_pass(p, in, out, nc, a, el, scale, acc, s);
            continue;
        }
        const float* src = in;
        float* bufs[2] = {t1, t2};
        int k = 0;
        for (int b = 0; b < d && !e; ++b) {
            if (b == a) continue;
            e = launch_pass(p, src, bufs[k], nc, b, bx, 1.f, 0, s);
            src = bufs[k++];
        }
        if (!e) e = launch_pass(p, src, out, nc, a, el, scale, acc, s);
    }
    return e;
}

}  // namespace

extern "C" int lbm_qoi_eval_static(const lbm_config* cfg, const float* u, double* q, void* cuda_stream) {
    if (!cfg || !u || !q) return err(LBM_ERR_ARG, "lbm_qoi_eval_static: NULL argument");
    if (cfg->dim != 2 && cfg->dim != 3) return err(LBM_ERR_ARG, "lbm_qoi_eval_static: dim must be 2 or 3");
    if (cfg->nx < 3 || cfg->ny < 3 || (cfg->dim == 2 ? cfg->nz != 1 : cfg->nz < 3))
        return err(LBM_ERR_ARG, "lbm_qoi_eval_static: bad grid size");
    if (cfg->walls && cfg->ny < 4) return err(LBM_ERR_ARG, "lbm_qoi_eval_static: walls need ny >= 4");
    if (cfg->n_qoi < 1 || cfg->n_qoi > 8) return err(LBM_ERR_ARG, "lbm_qoi_eval_static: need 1..8 scale-aware QoIs");
    if (cfg->n_mp != 0) return err(LBM_ERR_ARG, "lbm_qoi_eval_static: mean-profile QoIs are not supported (n_mp must be 0)");
    const cudaStream_t s = (cudaStream_t)cuda_stream;

    Params p;
    memset(&p, 0, sizeof p);
    p.dim = cfg->dim;
    p.nx = cfg->nx; p.ny = cfg->ny; p.nz = cfg->nz;
    p.walls = cfg->walls ? 1 : 0;
    p.n = (long long)cfg->nx * cfg->ny * cfg->nz;
    p.n_s = cfg->n_qoi;
    p.n_q = p.n_s;
    p.ncomp = cfg->dim == 2 ? 3 : 6;
    if (p.n * p.ncomp >= (1LL << 31)) return err(LBM_ERR_ARG, "lbm_qoi_eval_static: grid too large");
    Filt filt[kMaxFilters];
    int nf = 0;
    for (int i = 0; i < p.n_s; ++i) {
        const lbm_qoi_spec& sp = cfg->qoi[i];
        if (sp.kind != LBM_QOI_ENERGY && sp.kind != LBM_QOI_ENSTROPHY) return err(LBM_ERR_ARG, "lbm_qoi_eval_static: bad QoI kind");
        if (sp.filter == LBM_FILTER_FOURIER)
            return err(LBM_ERR_ARG, "lbm_qoi_eval_static: Fourier-band QoIs are not supported (Gaussian, Laplacian, binomial only)");
        if (sp.filter < 0 || sp.filter > 2) return err(LBM_ERR_ARG, "lbm_qoi_eval_static: bad filter");
        const int sc = sp.filter == LBM_FILTER_BINOMIAL ? 1 : sp.scale;
        if (sp.filter != LBM_FILTER_BINOMIAL && (sc < 1 || sc % 2 == 0)) return err(LBM_ERR_ARG, "lbm_qoi_eval_static: filter scale must be odd");
        if (sp.filter == LBM_FILTER_GAUSS && 2 * (cfg->dim == 2 ? 4 : 2) * sc + 1 > kMaxTaps) return err(LBM_ERR_ARG, "lbm_qoi_eval_static: Gaussian scale too large");
        if (sp.filter == LBM_FILTER_LAPLACE && 5 * sc > kMaxTaps) return err(LBM_ERR_ARG, "lbm_qoi_eval_static: Laplacian scale too large");
        int found = -1;
        for (int j = 0; j < nf; ++j)
            if (filt[j].kind == sp.filter && filt[j].scale == sc) found = j;
        if (found < 0) {
            filt[nf] = {sp.filter, sc, false};
            found = nf++;
        }
        if (sp.kind == LBM_QOI_ENSTROPHY) filt[found].need_z = true;
        p.qoi_kind[i] = sp.kind;
        p.qoi_filter_slot[i] = found;
    }
    p.n_filters = nf;
    int target = (1184 + p.ny - 1) / p.ny;
    if (target > p.nz) target = p.nz;
    if (target < 1) target = 1;
    const int zper = (p.nz + target - 1) / target;
    p.nzc = (p.nz + zper - 1) / zper;
    p.nblk_red = p.ny * p.nzc;
    p.npart = p.n_s + p.n_s * (p.n_s + 1) / 2;
    p.ntot = p.npart;  // no mean-profile bands
    p.npart_all = p.npart;

    // scratch layout (offsets into the static array)
    const size_t N = (size_t)p.n;
    const size_t field = align256(sizeof(float) * p.ncomp * N);
    size_t need = 4 * field;  // x6, t1, t2, acc
    size_t off_rr[kMaxFilters], off_vz[kMaxFilters];
    for (int f = 0; f < nf; ++f) {
        off_rr[f] = need;
        need += field;
        off_vz[f] = need;
        if (filt[f].need_z) need += align256(sizeof(float) * p.dim * N);
    }
    const size_t off_part = need;
    need += align256(sizeof(float) * (size_t)p.nblk_red * p.npart_all);
    const size_t off_plane = need;
    need += align256(sizeof(float) * (size_t)p.nzc * p.ny * (1 + p.n_s));
    if (need > LBM_STATIC_SCRATCH_BYTES)
        return err(LBM_ERR_BUDGET, "lbm_qoi_eval_static: needs %zu scratch bytes, the static array holds %u", need,
                   (unsigned)LBM_STATIC_SCRATCH_BYTES);

    // set-up once per context: the device address of the static array
    char* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        unsigned long long id = current_context_id();
        for (int i = 0; i < g_nctx && id; ++i)
            if (g_ctx_cache[i].id == id) base = (char*)g_ctx_cache[i].ptr;
        if (!base) {
            void* ptr = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
            if (e != cudaSuccess || !ptr)
                return err(LBM_ERR_CUDA, "lbm_qoi_eval_static: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            base = (char*)ptr;
            if (!id) id = current_context_id();  // the lookup made the primary context current
            if (id && g_nctx < kMaxContexts) g_ctx_cache[g_nctx++] = {id, ptr};
        }
    }
    cudaError_t e = cudaSuccess;

    Layout L;
    memset(&L, 0, sizeof L);
    L.x6 = (float*)base;
    L.vps = L.x6;
    L.t1 = (float*)(base + field);
    L.t2 = (float*)(base + 2 * field);
    L.acc = (float*)(base + 3 * field);
    for (int f = 0; f < nf; ++f) {
        L.rr[f] = (float*)(base + off_rr[f]);
        L.vz[f] = filt[f].need_z ? (float*)(base + off_vz[f]) : nullptr;
    }
    L.part = (float*)(base + off_part);
    L.plane_part = (float*)(base + off_plane);

    // every scratch region below is fully written before it is read:
    // the velocity copy zeroes solid rows, curl/passes/sens write every node,
    // each reduction block writes its own partial slot
    masked_copy_kernel<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(p, u, L.x6);
    e = cudaGetLastError();
    if (!e) e = launch_to_curl(p, L, s);
    for (int f = 0; f < nf && !e; ++f) {
        e = filter(p, filt[f], L.x6, L.acc, L.t1, L.t2, s);
        if (!e) e = filter(p, filt[f], L.acc, L.rr[f], L.t1, L.t2, s);
        if (!e && filt[f].need_z) e = launch_sens_curl(p, L.rr[f] + (size_t)p.dim * N, L.vz[f], s);
    }
    const float* vk[kMaxQoi];
    for (int k = 0; k < p.n_s; ++k)
        vk[k] = p.qoi_kind[k] == LBM_QOI_ENERGY ? L.rr[p.qoi_filter_slot[k]] : L.vz[p.qoi_filter_slot[k]];
    if (!e) e = launch_reduce(p, L, vk, s);
    if (!e) {
        finish_kernel<<<1, 256, 0, s>>>(p, L.part, q);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return err(LBM_ERR_CUDA, "lbm_qoi_eval_static: launch: %s", cudaGetErrorString(e));
    return LBM_OK;
}
