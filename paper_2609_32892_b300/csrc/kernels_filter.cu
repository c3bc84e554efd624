// Fast 1-D filter passes (one separable factor of G_s, L_s or B3, Sec. 4.1).
//
// Strided axes (y, z): each thread owns a segment of one line along the axis
// and marches along it with a register window of 2R+1 values per component,
// so every input element is loaded once per segment (plus a 2R halo) and all
// loads of a warp are coalesced (consecutive threads = consecutive x).
// Contiguous axis (x): one block stages a row chunk plus halo of every
// component in shared memory with coalesced loads and convolves from there.
// Both handle periodic wrap of any length and, along y with walls, the zero
// extension beyond the array with zero output on solid rows.
#include "batch.cuh"
#include "lbm_common.cuh"

namespace lbm {

template <int R> struct TapsR {
    float t[2 * R + 1];
};

__device__ __forceinline__ int posmod(int a, int n) {
    int r = a % n;
    return r < 0 ? r + n : r;
}

template <int R, int NC>
__device__ __forceinline__ void march_kernel_body(const VB& vb, const Params& p, const float* __restrict__ in,
                                                  float* __restrict__ out, int axis, TapsR<R> tp, float scale,
                                                  int accumulate, int seg) {
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const int other = axis == 1 ? nz : ny;
    const int line = vb.x * blockDim.x + threadIdx.x;
    if (line >= nx * other) return;
    const int x = line % nx;
    const int o = line / nx;
    const int L = axis == 1 ? ny : nz;
    const size_t stride = axis == 1 ? (size_t)nx : (size_t)nx * ny;
    const size_t base = axis == 1 ? (size_t)o * ny * nx + x : (size_t)o * nx + x;
    const size_t N = (size_t)p.n;
    const bool zero_pad = axis == 1 && p.walls;
    const int p0 = vb.y * seg;
    const int p1 = min(L, p0 + seg);
    if (p0 >= L) return;
    float w[NC][2 * R + 1];
    // prologue: positions p0-R .. p0+R-1 into slots 0 .. 2R-1
#pragma unroll
    for (int k = 0; k < 2 * R; ++k) {
        const int q = p0 - R + k;
        bool ok = true;
        int qq = q;
        if (zero_pad) ok = (q >= 0 && q < L);
        else qq = posmod(q, L);
#pragma unroll
        for (int c = 0; c < NC; ++c) w[c][k] = ok ? __ldg(in + c * N + base + (size_t)qq * stride) : 0.f;
    }
    for (int pos = p0; pos < p1; ++pos) {
        const int q = pos + R;
        bool ok = true;
        int qq = q;
        if (zero_pad) ok = q < L;
        else qq = posmod(q, L);
        const bool solid = p.walls && axis == 1 && (pos == 0 || pos == L - 1);
        const bool solid_row = p.walls && axis == 2 && (o == 0 || o == ny - 1);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            w[c][2 * R] = ok ? __ldg(in + c * N + base + (size_t)qq * stride) : 0.f;
            // out(pos) = sum_r t(r) in(pos - r); slot k holds in(pos - R + k)
            float s = 0.f;
#pragma unroll
            for (int r = -R; r <= R; ++r) s += tp.t[r + R] * w[c][R - r];
            float* op = out + c * N + base + (size_t)pos * stride;
            const float v = (solid || solid_row) ? 0.f : scale * s;
            *op = accumulate ? (*op + v) : v;
#pragma unroll
            for (int k = 0; k < 2 * R; ++k) w[c][k] = w[c][k + 1];
        }
    }
}
template <int R, int NC>
struct march_kernel_op {
    static constexpr int NT = 128, MINB = 1;
    template <class... B>
    static __device__ __forceinline__ void run(const VB& vb, const B&... b) {
        march_kernel_body<R, NC>(vb, b...);
    }
};
template <int R, int NC>
__global__ void __launch_bounds__(128) march_kernel(Params p, const float* __restrict__ in, float* __restrict__ out,
                                                    int axis, TapsR<R> tp, float scale, int accumulate, int seg) {
    march_kernel_body<R, NC>(vb_hw(), p, in, out, axis, tp, scale, accumulate, seg);
}

constexpr int kTX = 128;

template <int R, int NC>
__device__ __forceinline__ void xpass_kernel_body(const VB& vb, const Params& p, const float* __restrict__ in,
                                                  float* __restrict__ out, TapsR<R> tp, float scale, int accumulate) {
    __shared__ float sm[NC][kTX + 2 * R];
    const int nx = p.nx, ny = p.ny;
    const int row = vb.y;  // z * ny + y
    const int y = row % ny;
    const int x0 = vb.x * kTX;
    const size_t N = (size_t)p.n;
    const size_t rbase = (size_t)row * nx;
    const int x = x0 + threadIdx.x;
    if (p.walls && (y == 0 || y == ny - 1)) {
        if (x < nx)
#pragma unroll
            for (int c = 0; c < NC; ++c) out[c * N + rbase + x] = 0.f;
        return;
    }
    for (int i = threadIdx.x; i < NC * (kTX + 2 * R); i += kTX) {
        const int c = i / (kTX + 2 * R), k = i % (kTX + 2 * R);
        const int xs = posmod(x0 - R + k, nx);
        sm[c][k] = __ldg(in + c * N + rbase + xs);
    }
    __syncthreads();
    if (x >= nx) return;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        float s = 0.f;
#pragma unroll
        for (int r = -R; r <= R; ++r) s += tp.t[r + R] * sm[c][threadIdx.x + R - r];
        float* op = out + c * N + rbase + x;
        const float v = scale * s;
        *op = accumulate ? (*op + v) : v;
    }
}
template <int R, int NC>
struct xpass_kernel_op {
    static constexpr int NT = kTX, MINB = 1;
    template <class... B>
    static __device__ __forceinline__ void run(const VB& vb, const B&... b) {
        xpass_kernel_body<R, NC>(vb, b...);
    }
};
template <int R, int NC>
__global__ void __launch_bounds__(kTX) xpass_kernel(Params p, const float* __restrict__ in, float* __restrict__ out,
                                                    TapsR<R> tp, float scale, int accumulate) {
    xpass_kernel_body<R, NC>(vb_hw(), p, in, out, tp, scale, accumulate);
}

template <int R, int NC>
static cudaError_t run(const Params& p, const float* in, float* out, int axis, const Taps& t, float scale,
                       int accumulate, cudaStream_t s) {
    TapsR<R> tr;
    for (int i = 0; i < 2 * R + 1; ++i) tr.t[i] = t.t[i];
    if (axis == 0) {
        dim3 grid((p.nx + kTX - 1) / kTX, p.ny * p.nz);
        go<xpass_kernel_op<R, NC>>(xpass_kernel<R, NC>, grid, kTX, 0, s, p, in, out, tr, scale, accumulate);
    } else {
        const int L = axis == 1 ? p.ny : p.nz;
        const int lines = p.nx * (axis == 1 ? p.nz : p.ny);
        // split lines into segments so that ~tune.march_lines threads are in flight
        int nseg = (int)(((long long)p.tune.march_lines + lines - 1) / lines);
        if (nseg < 1) nseg = 1;
        int seg = (L + nseg - 1) / nseg;
        if (seg < 4 * R) seg = 4 * R;
        if (seg > L) seg = L;
        nseg = (L + seg - 1) / seg;
        dim3 grid((lines + 127) / 128, nseg);
        go<march_kernel_op<R, NC>>(march_kernel<R, NC>, grid, 128, 0, s, p, in, out, axis, tr, scale, accumulate,
                                   seg);
    }
    return cudaGetLastError();
}

// Returns cudaErrorNotSupported when no specialised instance exists.
cudaError_t launch_pass_fast(const Params& p, const float* in, float* out, int ncomp, int axis, const Taps& t,
                             float scale, int accumulate, cudaStream_t s) {
#define LBM_CASE(RR)                                                                  \
    case RR:                                                                          \
        if (ncomp == 3) return run<RR, 3>(p, in, out, axis, t, scale, accumulate, s); \
        if (ncomp == 6) return run<RR, 6>(p, in, out, axis, t, scale, accumulate, s); \
        break;
    switch (t.radius) {
        LBM_CASE(1)
        LBM_CASE(2)
        LBM_CASE(4)
        LBM_CASE(6)
        LBM_CASE(7)
        LBM_CASE(12)
        default: break;
    }
#undef LBM_CASE
    return cudaErrorNotSupported;
}

// ------------------------------------------------------ fused 2-D filters --
// One launch per application on a doubly periodic 2-D grid (the separate x
// and y passes cost two launches and a round trip of the intermediate field,
// which dominates small members).  A block stages a (TY + 2R) x (TX + 2R)
// tile of one component in shared memory with periodic wrap, applies the x
// factor into a second array (8 consecutive outputs per task from 8 + 2R
// staged values) and the y factor from there (4 rows per thread); the L_1
// cross reads the tile directly.
namespace f2 {
constexpr int TX = 32, TY = 32, NT = 256;
}

template <int R>
__device__ __forceinline__ void gauss2_kernel_body(const VB& vb, const Params& p, const float* __restrict__ in,
                                                   float* __restrict__ out, TapsR<R> tp, float scale,
                                                   int accumulate) {
    constexpr int TX = f2::TX, TY = f2::TY, NT = f2::NT, W = TX + 2 * R, H = TY + 2 * R;
    __shared__ float tile[H * W];
    __shared__ float xt[H * TX];
    const size_t N = (size_t)p.n;
    const float* a = in + vb.z * N;
    float* o = out + vb.z * N;
    const int x0 = vb.x * TX, y0 = vb.y * TY;
    for (int i = threadIdx.x; i < H * W; i += NT) {
        const int ly = i / W, lx = i - ly * W;
        const int gx = posmod(x0 - R + lx, p.nx), gy = posmod(y0 - R + ly, p.ny);
        tile[i] = __ldg(a + (size_t)gy * p.nx + gx);
    }
    __syncthreads();
    for (int task = threadIdx.x; task < H * (TX / 8); task += NT) {
        const int ry = task / (TX / 8), k = task - ry * (TX / 8);
        const float* row = tile + ry * W + 8 * k;
        float v[8 + 2 * R];
#pragma unroll
        for (int m = 0; m < 8 + 2 * R; ++m) v[m] = row[m];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            float sx = 0.f;
#pragma unroll
            for (int r = -R; r <= R; ++r) sx = fmaf(tp.t[r + R], v[j + R - r], sx);
            xt[ry * TX + 8 * k + j] = sx;
        }
    }
    __syncthreads();
    const int lx = threadIdx.x & (TX - 1), r0 = (threadIdx.x / TX) * 4;
    float col[4 + 2 * R];
#pragma unroll
    for (int m = 0; m < 4 + 2 * R; ++m) col[m] = xt[(r0 + m) * TX + lx];
    const int x = x0 + lx;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int y = y0 + r0 + j;
        if (x < p.nx && y < p.ny) {
            float sy = 0.f;
#pragma unroll
            for (int r = -R; r <= R; ++r) sy = fmaf(tp.t[r + R], col[j + R - r], sy);
            float* op = o + (size_t)y * p.nx + x;
            const float v = scale * sy;
            *op = accumulate ? *op + v : v;
        }
    }
}
template <int R>
struct gauss2_kernel_op {
    static constexpr int NT = 256, MINB = 1;
    template <class... B>
    static __device__ __forceinline__ void run(const VB& vb, const B&... b) {
        gauss2_kernel_body<R>(vb, b...);
    }
};
template <int R>
__global__ void __launch_bounds__(256) gauss2_kernel(Params p, const float* __restrict__ in, float* __restrict__ out,
                                                     TapsR<R> tp, float scale, int accumulate) {
    gauss2_kernel_body<R>(vb_hw(), p, in, out, tp, scale, accumulate);
}

// L_1 in 2-D: the 9-point cross of l = [1, -4, 6, -4, 1] along x and y
__device__ __forceinline__ void cross2_kernel_body(const VB& vb, const Params& p, const float* __restrict__ in,
                                                   float* __restrict__ out, TapsR<2> ell, float scale,
                                                   int accumulate) {
    constexpr int R = 2, TX = f2::TX, TY = f2::TY, NT = f2::NT, W = TX + 2 * R, H = TY + 2 * R;
    __shared__ float tile[H * W];
    const size_t N = (size_t)p.n;
    const float* a = in + vb.z * N;
    float* o = out + vb.z * N;
    const int x0 = vb.x * TX, y0 = vb.y * TY;
    for (int i = threadIdx.x; i < H * W; i += NT) {
        const int ly = i / W, lx = i - ly * W;
        const int gx = posmod(x0 - R + lx, p.nx), gy = posmod(y0 - R + ly, p.ny);
        tile[i] = __ldg(a + (size_t)gy * p.nx + gx);
    }
    __syncthreads();
    const int lx = threadIdx.x & (TX - 1), r0 = (threadIdx.x / TX) * 4;
    const int x = x0 + lx;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int y = y0 + r0 + j;
        if (x < p.nx && y < p.ny) {
            const float* c = tile + (r0 + j + R) * W + lx + R;
            float s2 = 2.f * ell.t[R] * c[0];
#pragma unroll
            for (int r = 1; r <= R; ++r) s2 = fmaf(ell.t[R + r], (c[-r] + c[r]) + (c[-r * W] + c[r * W]), s2);
            float* op = o + (size_t)y * p.nx + x;
            const float v = scale * s2;
            *op = accumulate ? *op + v : v;
        }
    }
}
struct cross2_kernel_op {
    static constexpr int NT = 256, MINB = 1;
    template <class... B>
    static __device__ __forceinline__ void run(const VB& vb, const B&... b) {
        cross2_kernel_body(vb, b...);
    }
};
__global__ void __launch_bounds__(256) cross2_kernel(Params p, const float* __restrict__ in, float* __restrict__ out,
                                                     TapsR<2> ell, float scale, int accumulate) {
    cross2_kernel_body(vb_hw(), p, in, out, ell, scale, accumulate);
}

template <int R>
static cudaError_t run_gauss2(const Params& p, const float* in, float* out, int ncomp, const Taps& t, float scale,
                              int accumulate, cudaStream_t s) {
    TapsR<R> tr;
    for (int i = 0; i < 2 * R + 1; ++i) tr.t[i] = t.t[i];
    const dim3 grid((p.nx + f2::TX - 1) / f2::TX, (p.ny + f2::TY - 1) / f2::TY, ncomp);
    go<gauss2_kernel_op<R>>(gauss2_kernel<R>, grid, f2::NT, 0, s, p, in, out, tr, scale, accumulate);
    return cudaGetLastError();
}

// Returns cudaErrorNotSupported unless the grid is 2-D and doubly periodic and
// a specialised instance exists (the separable passes serve the rest).
cudaError_t launch_filter2_fused(const Params& p, const float* in, float* out, int ncomp, bool laplacian, int s_scale,
                                 const Taps& t, float scale, int accumulate, cudaStream_t s) {
    if (p.dim != 2 || p.walls) return cudaErrorNotSupported;
    if (laplacian) {
        if (s_scale != 1 || t.radius != 2) return cudaErrorNotSupported;
        TapsR<2> tr;
        for (int i = 0; i < 5; ++i) tr.t[i] = t.t[i];
        const dim3 grid((p.nx + f2::TX - 1) / f2::TX, (p.ny + f2::TY - 1) / f2::TY, ncomp);
        go<cross2_kernel_op>(cross2_kernel, grid, f2::NT, 0, s, p, in, out, tr, scale, accumulate);
        return cudaGetLastError();
    }
    switch (t.radius) {
        case 1: return run_gauss2<1>(p, in, out, ncomp, t, scale, accumulate, s);
        case 4: return run_gauss2<4>(p, in, out, ncomp, t, scale, accumulate, s);
        case 12: return run_gauss2<12>(p, in, out, ncomp, t, scale, accumulate, s);
        default: return cudaErrorNotSupported;
    }
}

}  // namespace lbm
