// Tau-orthogonal phase kernels (Sec. 4, App. A): vorticity, separable filter
// passes, enstrophy sensitivities, the QoI / Gram block reduction, the LRS
// history matvec and the single-block FP64 coefficient solve.
//
// Fields are FP32 structure-of-arrays [comp][nz][ny][nx].  Every field is
// zero on solid rows, which is exactly the zero extension the filters and the
// central differences use beyond the walls (Sec. 4.1).
#include "batch.cuh"
#include "lbm_common.cuh"
#include "rng.cuh"
#include "dfloat.cuh"

namespace lbm {

__device__ __forceinline__ int wrapi(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }
__device__ __forceinline__ int modp(int a, int n) {
    int r = a % n;
    return r < 0 ? r + n : r;
}

// ------------------------------------------------------------ vorticity --
// omega = curl v* by central differences: 3-D (d_y v_z - d_z v_y, d_z v_x -
// d_x v_z, d_x v_y - d_y v_x); 2-D the scalar d_x v_y - d_y v_x.  Written
// after the d velocity components of the stacked field x6.
__device__ __forceinline__ void curl_kernel_body(const VB& vb, const Params& p, float* __restrict__ x6) {
    const int n = vb.x * blockDim.x + threadIdx.x;
    if (n >= p.n) return;
    const int N = (int)p.n, nx = p.nx, ny = p.ny, nz = p.nz;
    const int x = n % nx;
    const int t = n / nx;
    const int y = t % ny;
    const int z = t / ny;
    const int d = p.dim;
    if (p.walls && (y == 0 || y == ny - 1)) {
        for (int c = d; c < p.ncomp; ++c) x6[(size_t)c * N + n] = 0.f;
        return;
    }
    const int xm = wrapi(x - 1, nx), xp = wrapi(x + 1, nx);
    const int ym = wrapi(y - 1, ny), yp = wrapi(y + 1, ny);
    const size_t r0 = ((size_t)z * ny + y) * nx;
    const size_t iym = ((size_t)z * ny + ym) * nx + x, iyp = ((size_t)z * ny + yp) * nx + x;
    const float* vx = x6;
    const float* vy = x6 + N;
    if (d == 2) {
        const float dxvy = 0.5f * (vy[r0 + xp] - vy[r0 + xm]);
        const float dyvx = 0.5f * (vx[iyp] - vx[iym]);
        x6[(size_t)2 * N + n] = dxvy - dyvx;
        return;
    }
    const float* vz = x6 + 2 * (size_t)N;
    const int zm = wrapi(z - 1, nz), zp = wrapi(z + 1, nz);
    const size_t izm = ((size_t)zm * ny + y) * nx + x, izp = ((size_t)zp * ny + y) * nx + x;
    const float dyvz = 0.5f * (vz[iyp] - vz[iym]), dzvy = 0.5f * (vy[izp] - vy[izm]);
    const float dzvx = 0.5f * (vx[izp] - vx[izm]), dxvz = 0.5f * (vz[r0 + xp] - vz[r0 + xm]);
    const float dxvy = 0.5f * (vy[r0 + xp] - vy[r0 + xm]), dyvx = 0.5f * (vx[iyp] - vx[iym]);
    x6[(size_t)3 * N + n] = dyvz - dzvy;
    x6[(size_t)4 * N + n] = dzvx - dxvz;
    x6[(size_t)5 * N + n] = dxvy - dyvx;
}
struct curl_kernel_op {
    static constexpr int NT = 256, MINB = 1;
    template <class... B>
    static __device__ __forceinline__ void run(const VB& vb, const B&... b) {
        curl_kernel_body(vb, b...);
    }
};
__global__ void __launch_bounds__(256) curl_kernel(Params p, float* __restrict__ x6) {
    curl_kernel_body(vb_hw(), p, x6);
}

// --------------------------------------------------------- filter pass --
// out(x) = [out(x) +] scale * sum_r t(r) in(x - r e_axis) for every component:
// one 1-D factor of a separable filter.  Periodic along x and z (and y without
// walls, any radius); along y with walls, rows outside the array contribute
// nothing and solid rows hold zero, and the output is zero on solid rows.
__device__ __forceinline__ void pass_kernel_body(const VB& vb, const Params& p, const float* __restrict__ in,
                                                 float* __restrict__ out, int ncomp, int axis, const Taps& tp,
                                                 float scale, int accumulate) {
    const int n = vb.x * blockDim.x + threadIdx.x;
    if (n >= p.n) return;
    const size_t N = (size_t)p.n;
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const int x = n % nx;
    const int t = n / nx;
    const int y = t % ny;
    const int z = t / ny;
    if (p.walls && (y == 0 || y == ny - 1)) {
        for (int c = 0; c < ncomp; ++c) out[c * N + n] = 0.f;
        return;
    }
    const int R = tp.radius;
    for (int c = 0; c < ncomp; ++c) {
        const float* a = in + c * N;
        float s = 0.f;
        if (axis == 0) {
            const size_t row = ((size_t)z * ny + y) * nx;
            for (int r = -R; r <= R; ++r) s += tp.t[r + R] * a[row + modp(x - r, nx)];
        } else if (axis == 1) {
            if (p.walls) {
                for (int r = -R; r <= R; ++r) {
                    const int ys = y - r;
                    if (ys >= 0 && ys < ny) s += tp.t[r + R] * a[((size_t)z * ny + ys) * nx + x];
                }
            } else {
                for (int r = -R; r <= R; ++r) s += tp.t[r + R] * a[((size_t)z * ny + modp(y - r, ny)) * nx + x];
            }
        } else {
            for (int r = -R; r <= R; ++r) s += tp.t[r + R] * a[((size_t)modp(z - r, nz) * ny + y) * nx + x];
        }
        float* o = out + c * N + n;
        *o = accumulate ? (*o + scale * s) : scale * s;
    }
}
struct pass_kernel_op {
    static constexpr int NT = 256, MINB = 1;
    template <class... B>
    static __device__ __forceinline__ void run(const VB& vb, const B&... b) {
        pass_kernel_body(vb, b...);
    }
};
__global__ void __launch_bounds__(256) pass_kernel(Params p, const float* __restrict__ in, float* __restrict__ out,
                                                   int ncomp, int axis, Taps tp, float scale, int accumulate) {
    pass_kernel_body(vb_hw(), p, in, out, ncomp, axis, tp, scale, accumulate);
}

// ------------------------------------------------------- Fourier bands --
// out = in * (1/(nx ny) if lo - 1/2 <= |k| < hi + 1/2 else 0) on the R2C half
// spectrum [c][ky][kx] (kx = 0..nx/2, ky folded to -ny/2..ny/2-1): the sharp
// filter R_[lo,hi] of Sec. 4.1 with the inverse transform's normalisation.
// The band edges sit at half-integers, so the test on the integer |k|^2 is exact.
__global__ void __launch_bounds__(256) band_mask_kernel(Params p, const float2* __restrict__ in,
                                                        float2* __restrict__ out, int ncomp, int lo, int hi) {
    const int nxh = p.nx / 2 + 1;
    const long long per = (long long)p.ny * nxh;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= per * ncomp) return;
    const long long e = i % per;
    const int kx = (int)(e % nxh);
    const int jy = (int)(e / nxh);
    const int ky = jy <= p.ny / 2 ? jy : jy - p.ny;
    const long long k2 = (long long)kx * kx + (long long)ky * ky;
    // lo - 1/2 <= |k|  <=>  k2 >= lo^2 - lo + 1 (lo >= 1);  |k| < hi + 1/2  <=>  k2 <= hi^2 + hi
    const bool keep = (lo == 0 || k2 >= (long long)lo * lo - lo + 1) && k2 <= (long long)hi * hi + hi;
    const float sc = keep ? 1.0f / ((float)p.nx * (float)p.ny) : 0.f;
    const float2 v = in[i];
    out[i] = make_float2(v.x * sc, v.y * sc);
}

// ---------------------------------------------- enstrophy sensitivities --
// V_Z = curl*(W), W = R R omega (App. A): 2-D (d_y W, -d_x W); 3-D curl W.
__device__ __forceinline__ void sens_curl_kernel_body(const VB& vb, const Params& p, const float* __restrict__ w,
                                                      float* __restrict__ out) {
    const int n = vb.x * blockDim.x + threadIdx.x;
    if (n >= p.n) return;
    const int N = (int)p.n, nx = p.nx, ny = p.ny, nz = p.nz;
    const int x = n % nx;
    const int t = n / nx;
    const int y = t % ny;
    const int z = t / ny;
    const int d = p.dim;
    if (p.walls && (y == 0 || y == ny - 1)) {
        for (int c = 0; c < d; ++c) out[(size_t)c * N + n] = 0.f;
        return;
    }
    const int xm = wrapi(x - 1, nx), xp = wrapi(x + 1, nx);
    const int ym = wrapi(y - 1, ny), yp = wrapi(y + 1, ny);
    const size_t r0 = ((size_t)z * ny + y) * nx;
    const size_t iym = ((size_t)z * ny + ym) * nx + x, iyp = ((size_t)z * ny + yp) * nx + x;
    if (d == 2) {
        out[n] = 0.5f * (w[iyp] - w[iym]);
        out[(size_t)N + n] = -0.5f * (w[r0 + xp] - w[r0 + xm]);
        return;
    }
    const float* wx = w;
    const float* wy = w + N;
    const float* wz = w + 2 * (size_t)N;
    const int zm = wrapi(z - 1, nz), zp = wrapi(z + 1, nz);
    const size_t izm = ((size_t)zm * ny + y) * nx + x, izp = ((size_t)zp * ny + y) * nx + x;
    out[n] = 0.5f * (wz[iyp] - wz[iym]) - 0.5f * (wy[izp] - wy[izm]);
    out[(size_t)N + n] = 0.5f * (wx[izp] - wx[izm]) - 0.5f * (wz[r0 + xp] - wz[r0 + xm]);
    out[(size_t)2 * N + n] = 0.5f * (wy[r0 + xp] - wy[r0 + xm]) - 0.5f * (wx[iyp] - wx[iym]);
}
struct sens_curl_kernel_op {
    static constexpr int NT = 256, MINB = 1;
    template <class... B>
    static __device__ __forceinline__ void run(const VB& vb, const B&... b) {
        sens_curl_kernel_body(vb, b...);
    }
};
__global__ void __launch_bounds__(256) sens_curl_kernel(Params p, const float* __restrict__ w, float* __restrict__ out) {
    sens_curl_kernel_body(vb_hw(), p, w, out);
}

// ------------------------------------------- four nodes per thread --
// The same central differences for nx % 4 == 0, four x-consecutive nodes per
// thread: float4 loads of the centre and the y and z neighbour quads, two
// scalar loads for the x neighbours past the quad's ends, float4 stores.  The
// index arithmetic runs once per quad, and a 3-D quad takes 14 load
// instructions where four one-node threads take 48.  Every difference is taken
// in the order of the one-node kernels above (halving is exact), so the
// results are bit-identical.
enum { kCurl3 = 0, kVort2 = 1, kSens2 = 2 };

__device__ __forceinline__ float4 ld4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ void st4(float* p, float a, float b, float c, float d) {
    *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
}

struct Q4 {
    float v[4];
};
// half central difference along x of the row quad at c + r (+ x)
__device__ __forceinline__ Q4 dx4(const float* __restrict__ c, size_t r, int x, int xl, int xr) {
    const float4 m = ld4(c + r + x);
    const float l = __ldg(c + r + xl), h = __ldg(c + r + xr);
    return Q4{{0.5f * (m.y - l), 0.5f * (m.z - m.x), 0.5f * (m.w - m.y), 0.5f * (h - m.z)}};
}
// half difference of the quads at c + ip and c + im
__device__ __forceinline__ Q4 dq4(const float* __restrict__ c, size_t ip, size_t im) {
    const float4 a = ld4(c + ip), b = ld4(c + im);
    return Q4{{0.5f * (a.x - b.x), 0.5f * (a.y - b.y), 0.5f * (a.z - b.z), 0.5f * (a.w - b.w)}};
}

// kCurl3: out = curl a (3-D, a and out three components; curl* = curl for
// the periodic central-difference operator).  kVort2: out = d_x a_y - d_y a_x.
// kSens2: out = (d_y a, -d_x a) of the scalar a.  Wall rows are zero.
template <int MODE>
__device__ __forceinline__ void curl4_kernel_body(const VB& vb, const Params& p, const float* __restrict__ a,
                                                  float* __restrict__ out) {
    const int nq = p.nx >> 2;
    const long long q = (long long)vb.x * blockDim.x + threadIdx.x;
    if (q >= p.n >> 2) return;
    const int N = (int)p.n, nx = p.nx, ny = p.ny, nz = p.nz;
    const int x = (int)(q % nq) * 4;
    const int t = (int)(q / nq);  // z * ny + y
    const int y = t % ny, z = t / ny;
    const size_t r0 = (size_t)t * nx;
    constexpr int NOUT = MODE == kCurl3 ? 3 : (MODE == kVort2 ? 1 : 2);
    if (p.walls && (y == 0 || y == ny - 1)) {
#pragma unroll
        for (int c = 0; c < NOUT; ++c) st4(out + (size_t)c * N + r0 + x, 0.f, 0.f, 0.f, 0.f);
        return;
    }
    const int xl = x == 0 ? nx - 1 : x - 1, xr = x + 4 == nx ? 0 : x + 4;
    const int ym = wrapi(y - 1, ny), yp = wrapi(y + 1, ny);
    const size_t iym = ((size_t)z * ny + ym) * nx + x, iyp = ((size_t)z * ny + yp) * nx + x;
    if (MODE == kSens2) {
        const Q4 dy = dq4(a, iyp, iym), dx = dx4(a, r0, x, xl, xr);
        st4(out + r0 + x, dy.v[0], dy.v[1], dy.v[2], dy.v[3]);
        st4(out + (size_t)N + r0 + x, -dx.v[0], -dx.v[1], -dx.v[2], -dx.v[3]);
        return;
    }
    const float* ax = a;
    const float* ay = a + N;
    if (MODE == kVort2) {
        const Q4 dxay = dx4(ay, r0, x, xl, xr), dyax = dq4(ax, iyp, iym);
        st4(out + r0 + x, dxay.v[0] - dyax.v[0], dxay.v[1] - dyax.v[1], dxay.v[2] - dyax.v[2],
            dxay.v[3] - dyax.v[3]);
        return;
    }
    const float* az = a + 2 * (size_t)N;
    const int zm = wrapi(z - 1, nz), zp = wrapi(z + 1, nz);
    const size_t izm = ((size_t)zm * ny + y) * nx + x, izp = ((size_t)zp * ny + y) * nx + x;
    const Q4 dyaz = dq4(az, iyp, iym), dzay = dq4(ay, izp, izm);
    const Q4 dzax = dq4(ax, izp, izm), dxaz = dx4(az, r0, x, xl, xr);
    const Q4 dxay = dx4(ay, r0, x, xl, xr), dyax = dq4(ax, iyp, iym);
    float* o = out + r0 + x;
    st4(o, dyaz.v[0] - dzay.v[0], dyaz.v[1] - dzay.v[1], dyaz.v[2] - dzay.v[2], dyaz.v[3] - dzay.v[3]);
    o += N;
    st4(o, dzax.v[0] - dxaz.v[0], dzax.v[1] - dxaz.v[1], dzax.v[2] - dxaz.v[2], dzax.v[3] - dxaz.v[3]);
    o += N;
    st4(o, dxay.v[0] - dyax.v[0], dxay.v[1] - dyax.v[1], dxay.v[2] - dyax.v[2], dxay.v[3] - dyax.v[3]);
}
template <int MODE>
struct curl4_kernel_op {
    static constexpr int NT = 256, MINB = 1;
    template <class... B>
    static __device__ __forceinline__ void run(const VB& vb, const B&... b) {
        curl4_kernel_body<MODE>(vb, b...);
    }
};
template <int MODE>
__global__ void __launch_bounds__(256) curl4_kernel(Params p, const float* __restrict__ a, float* __restrict__ out) {
    curl4_kernel_body<MODE>(vb_hw(), p, a, out);
}

// ------------------------------------------------------ block reduction --
// Per block (one y row, a chunk of z planes): <v*, V_k> and <V_i, V_j> (i <= j)
// over its fluid nodes, the row sums P_k of v*_x and V_k,x, and the
// mean-profile couplings w_j(y) P_k.  FP32 throughout the block (per thread
// over a few nodes, then a warp tree); the totals kernel sums the partials
// with compensation.  No double-precision arithmetic here: on this GPU an
// FP64 warp tree over the values of every block costs more than the whole
// field traversal.
__device__ __forceinline__ float lane4(const float4& v, int c) { return c == 0 ? v.x : (c == 1 ? v.y : (c == 2 ? v.z : v.w)); }

struct RedPtrs {
    const float* v[kMaxQoi];
};

template <int NS>
__device__ __forceinline__ void reduce_kernel_body(const VB& vb, const Params& p, const float* __restrict__ vps,
                                                   RedPtrs vk, const float2* __restrict__ w_mp2,
                                                   float* __restrict__ part, float* __restrict__ plane_part) {
    constexpr int NG = NS * (NS + 1) / 2;
    constexpr int NV = NS + NG + 1 + NS;  // <v,V_k>, Gram, row sums (v_x, V_k,x)
    const int y = vb.x;
    const int zc = vb.y;
    const int zper = (p.nz + p.nzc - 1) / p.nzc;
    const int z0 = zc * zper;
    const int z1 = min(p.nz, z0 + zper);
    const size_t N = (size_t)p.n;
    const int d = p.dim;
    float acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = 0.f;
    const bool solid = p.walls && (y == 0 || y == p.ny - 1);
    // one node's contributions from its velocity u and sensitivities w
    auto add_node = [&](const float (&u)[3], const float (&w)[NS][3]) {
        int idx = 0;
#pragma unroll
        for (int k = 0; k < NS; ++k) acc[idx++] += u[0] * w[k][0] + u[1] * w[k][1] + u[2] * w[k][2];
#pragma unroll
        for (int i = 0; i < NS; ++i)
#pragma unroll
            for (int j = i; j < NS; ++j) acc[idx++] += w[i][0] * w[j][0] + w[i][1] * w[j][1] + w[i][2] * w[j][2];
        acc[idx++] += u[0];
#pragma unroll
        for (int k = 0; k < NS; ++k) acc[idx++] += w[k][0];
    };
    if (p.nx % 4 == 0) {
        // four x-consecutive nodes per iteration: 16-byte loads, one index
        // division per quad
        const int nq = p.nx >> 2;
        const int cnt = solid ? 0 : (z1 - z0) * nq;
        for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
            const int zz = e / nq;
            const size_t n = ((size_t)(z0 + zz) * p.ny + y) * p.nx + 4 * (e - zz * nq);
            const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 u0 = ld4(vps + n), u1 = ld4(vps + N + n), u2 = d == 3 ? ld4(vps + 2 * N + n) : zero;
            float4 w4[NS][3];
#pragma unroll
            for (int k = 0; k < NS; ++k) {
                w4[k][0] = ld4(vk.v[k] + n);
                w4[k][1] = ld4(vk.v[k] + N + n);
                w4[k][2] = d == 3 ? ld4(vk.v[k] + 2 * N + n) : zero;
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                float u[3] = {lane4(u0, c), lane4(u1, c), lane4(u2, c)};
                float w[NS][3];
#pragma unroll
                for (int k = 0; k < NS; ++k)
#pragma unroll
                    for (int a = 0; a < 3; ++a) w[k][a] = lane4(w4[k][a], c);
                add_node(u, w);
            }
        }
    } else {
        const int cnt = solid ? 0 : (z1 - z0) * p.nx;
        for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
            const int z = z0 + e / p.nx;
            const int x = e % p.nx;
            const size_t n = ((size_t)z * p.ny + y) * p.nx + x;
            float u[3], w[NS][3];
            u[0] = vps[n]; u[1] = vps[N + n]; u[2] = d == 3 ? vps[2 * N + n] : 0.f;
#pragma unroll
            for (int k = 0; k < NS; ++k) {
                w[k][0] = vk.v[k][n];
                w[k][1] = vk.v[k][N + n];
                w[k][2] = d == 3 ? vk.v[k][2 * N + n] : 0.f;
            }
            add_node(u, w);
        }
    }
    __shared__ float sh[4][NV];
    __shared__ float tot[NV];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        float a = acc[v];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        if (lane == 0) sh[wid][v] = a;
    }
    __syncthreads();
    const int blk = vb.y * vb.gx + vb.x;
    const size_t row = (size_t)blk * p.npart_all;
    for (int v = threadIdx.x; v < NV; v += blockDim.x) {
        const float s = (sh[0][v] + sh[1][v]) + (sh[2][v] + sh[3][v]);
        tot[v] = s;
        if (v < NS + NG) part[row + v] = s;
        else plane_part[((size_t)zc * p.ny + y) * (1 + NS) + (v - NS - NG)] = s;
    }
    __syncthreads();
    // couplings w_j(y) P_k of this block's row sums, j < n_mp, k = 0..NS, as
    // unevaluated float pairs: with w = w_hi + w_lo (the FP64 weight split in
    // two floats) the products are exact up to w_lo P_k's rounding, so the
    // couplings keep FP64 accuracy (the mean-profile QoIs are large and the
    // LRS corrects them by small differences)
    for (int t = threadIdx.x; t < p.n_mp * (1 + NS); t += blockDim.x) {
        const int j = t / (1 + NS), k = t - j * (1 + NS);
        const float2 w = w_mp2[(size_t)j * p.ny + y];
        const float r = tot[NS + NG + k];
        const float hi = w.x * r;
        const float lo = fmaf(w.y, r, fmaf(w.x, r, -hi));
        part[row + NS + NG + 2 * t] = hi;
        part[row + NS + NG + 2 * t + 1] = lo;
    }
}
template <int NS>
struct reduce_kernel_op {
    static constexpr int NT = 128, MINB = 1;
    template <class... B>
    static __device__ __forceinline__ void run(const VB& vb, const B&... b) {
        reduce_kernel_body<NS>(vb, b...);
    }
};
template <int NS>
__global__ void __launch_bounds__(128) reduce_kernel(Params p, const float* __restrict__ vps, RedPtrs vk,
                                                     const float2* __restrict__ w_mp2, float* __restrict__ part,
                                                     float* __restrict__ plane_part) {
    reduce_kernel_body<NS>(vb_hw(), p, vps, vk, w_mp2, part, plane_part);
}

// ------------------------------------------------------------ totals --
// Sums the reduction partials across blocks, one block per value (the solve
// is a single block: reading every partial there would serialise a few
// hundred KB of L2 reads on one SM).  Compensated FP32 (TwoSum) per thread and
// across the block, widened to double once.  Further blocks: the plane sums
// P_k(y) over the z chunks (one warp per (y, k)) and, in LRS mode, the known
// part of the LRS prediction (history partials + mu + L z, Eq. LRS).
__device__ __forceinline__ DF df_block_sum(DF a, DF* sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a = df_add(a, df_shfl_down(a, o));
    if (lane == 0) sh[wid] = a;
    __syncthreads();
    DF t = {0.f, 0.f};
    if (wid == 0) {
        if (lane < (int)(blockDim.x >> 5)) t = sh[lane];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t = df_add(t, df_shfl_down(t, o));
    }
    return t;  // valid in thread 0
}

__device__ __forceinline__ void totals_kernel_body(const VB& vb, const Params& p, const Layout& L, int nplane_blk) {
    __shared__ DF sh[8];
    const int b = vb.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (b < p.npart) {
        DF a = {0.f, 0.f};
        int i = threadIdx.x;
        // four loads in flight per thread
        for (; i + 3 * 256 < p.nblk_red; i += 4 * 256) {
            const float x0 = L.part[(size_t)i * p.npart_all + b];
            const float x1 = L.part[(size_t)(i + 256) * p.npart_all + b];
            const float x2 = L.part[(size_t)(i + 512) * p.npart_all + b];
            const float x3 = L.part[(size_t)(i + 768) * p.npart_all + b];
            a = df_add(df_add(a, x0), df_add(df_two_sum(x1, x2), x3));
        }
        for (; i < p.nblk_red; i += 256) a = df_add(a, L.part[(size_t)i * p.npart_all + b]);
        const DF t = df_block_sum(a, sh);
        if (threadIdx.x == 0) L.tot[b] = (double)t.hi + (double)t.lo;
        return;
    }
    if (b < p.ntot) {
        // a coupling: float pairs (hi, lo) per block
        const size_t off = (size_t)p.npart + 2 * (size_t)(b - p.npart);
        DF a = {0.f, 0.f};
        int i = threadIdx.x;
        // (hi, lo) need not be 8-byte aligned: two scalar loads each
        for (; i + 256 < p.nblk_red; i += 2 * 256) {
            const float* r0 = L.part + (size_t)i * p.npart_all + off;
            const float* r1 = L.part + (size_t)(i + 256) * p.npart_all + off;
            const DF x0 = {r0[0], r0[1]}, x1 = {r1[0], r1[1]};
            a = df_add(df_add(a, x0), x1);
        }
        for (; i < p.nblk_red; i += 256) {
            const float* r0 = L.part + (size_t)i * p.npart_all + off;
            a = df_add(a, DF{r0[0], r0[1]});
        }
        const DF t = df_block_sum(a, sh);
        if (threadIdx.x == 0) L.tot[b] = (double)t.hi + (double)t.lo;
        return;
    }
    const int np1 = 1 + p.n_s;
    if (b < p.ntot + nplane_blk) {
        const int e = (b - p.ntot) * 8 + wid;
        if (e >= p.ny * np1) return;
        DF a = {0.f, 0.f};
        for (int zc = lane; zc < p.nzc; zc += 32) a = df_add(a, L.plane_part[(size_t)zc * p.ny * np1 + e]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a = df_add(a, df_shfl_down(a, o));
        if (lane == 0) L.plane_sum[e] = (double)a.hi + (double)a.lo;
        return;
    }
    // LRS: hsum_k = sum of the history partials + mu_k + (L z)_k, one block
    // (one warp: FP64 instructions are slow, spread them over SMs) per k
    const int nq = p.n_q;
    const int k = b - p.ntot - nplane_blk;
    if (wid != 0 || k >= nq) return;
    double a = lane < nq ? L.lrs_L[(size_t)k * nq + lane] * L.znorm[lane] : 0.0;
    if (lane == 0) a += L.lrs_mu[k];
    for (int bb = lane; bb < p.nblk_lrs; bb += 32) a += L.lrs_part[(size_t)bb * nq + k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    if (lane == 0) L.hsum[k] = a;
}
struct totals_kernel_op {
    static constexpr int NT = 256, MINB = 1;
    template <class... B>
    static __device__ __forceinline__ void run(const VB& vb, const B&... b) {
        totals_kernel_body(vb, b...);
    }
};
__global__ void __launch_bounds__(256) totals_kernel(Params p, Layout L, int nplane_blk) {
    totals_kernel_body(vb_hw(), p, L, nplane_blk);
}

// ------------------------------------------- LRS history matvec, normals --
// Runs on a side branch of the step (it needs only the previous step's
// histories and the step counter), so its latency hides behind the field
// kernels.  Blocks 0..nblk_lrs-1: partial sums of x_r C[r][:] over the rows of
// C whose inputs are known before the current QoIs: the histories
// q^{n-1..n-h} and q^{n-1*..n-h*} (scaled by sigma_ref) and the bias 1
// (Eq. LRS); the q^{n*} block is added in the solve.  A block first forms its
// rows' inputs x_r in shared memory (one division each, as in the model),
// then thread (j, k) accumulates rows j, j + per, ... of column k, so a warp
// reads consecutive elements of C.  The last block draws the step's normals
// (the LRS noise or the gamma draws).
__device__ __forceinline__ void lrs_pre_kernel_body(const VB& vb, const Params& p, const Layout& L, int nb) {
    const int nq = p.n_q;
    const long long step = L.st->step;
    if (vb.x == (unsigned)nb) {
        const int stream = p.to_mode == LBM_TO_GAMMA ? kStreamGamma : kStreamLrs;
        if (threadIdx.x < (unsigned)nq) L.znorm[threadIdx.x] = philox_normal(p.seed, p.member, step, stream, threadIdx.x);
        return;
    }
    const int h = p.h;
    const int rows = (2 * h + 1) * nq + 1;
    const int r0 = vb.x * p.lrs_rows_per_blk;
    const int r1 = min(rows, r0 + p.lrs_rows_per_blk);
    const int posm = (int)(L.st->hist_pos % h);
    __shared__ double xs[kLrsRowsPerBlk];
    __shared__ double sh[256];
    for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
        double xr = 0.0;
        if (r < h * nq || (r >= (h + 1) * nq && r < rows - 1)) {
            const bool corrected = r < h * nq;
            const int rr = corrected ? r : r - (h + 1) * nq;
            const int kk = rr / nq + 1, i = rr - (kk - 1) * nq;
            int slot = posm - kk;
            if (slot < 0) slot += h;
            const double sg = L.lrs_sigma[i];
            const double qv = corrected ? L.qh[(size_t)slot * nq + i] : L.qsh[(size_t)slot * nq + i];
            xr = sg > 0.0 ? qv / sg : 0.0;  // sigma <= 0: not yet set, the histories are zero
        } else if (r == rows - 1) {
            xr = 1.0;
        }  // rows of the q^{n*} block: added in the solve
        xs[r - r0] = xr;
    }
    __syncthreads();
    const int per = blockDim.x / nq;
    const int j = threadIdx.x / nq, k = threadIdx.x - j * nq;
    double acc = 0.0;
    if (j < per)
        for (int r = r0 + j; r < r1; r += per) acc = fma(xs[r - r0], L.lrs_C[(size_t)r * nq + k], acc);
    sh[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x < (unsigned)nq) {
        double s = 0.0;
        for (int jj = 0; jj < per; ++jj) s += sh[jj * nq + threadIdx.x];
        L.lrs_part[(size_t)vb.x * nq + threadIdx.x] = s;
    }
}
struct lrs_pre_kernel_op {
    static constexpr int NT = 256, MINB = 1;
    template <class... B>
    static __device__ __forceinline__ void run(const VB& vb, const B&... b) {
        lrs_pre_kernel_body(vb, b...);
    }
};
__global__ void __launch_bounds__(256) lrs_pre_kernel(Params p, Layout L, int nb) {
    lrs_pre_kernel_body(vb_hw(), p, L, nb);
}

// ------------------------------------------------------------- solve --
// One block: assemble q^{n*} and the Gram matrix G from the totals, evaluate
// the coefficient source, invert G and form beta = G^-1 dQ (dv_SGS = sum_k
// beta_k V_k equals sum_i gamma_i O_i with c_ij and gamma_i of Sec. 4.2-4.3)
// and gamma_i = dQ_i (G^-1)_ii.  Then write the QoI block row, push the LRS
// histories, add the mean profile and advance the step counter.
//
// Cost model (measured on this GPU): a double-precision warp instruction
// occupies the FP64 unit of its SM sub-partition for about 64 cycles and is
// not pipelined, whatever the number of active lanes; four sub-partitions per
// SM; a division costs about ten such instructions.  This kernel is on the
// critical path of every step, so it counts FP64 warp instructions per
// sub-partition rather than flops:
//  * G is equilibrated by exact powers of two, G~ = S G S, S = diag(s_i) with
//    s_i^2 G_ii in [1, 4) (integer operations on the exponent field);
//  * G~ is inverted by Gauss-Jordan elimination on [G~ | I] without pivoting
//    (G is symmetric positive definite when not singular) in fraction-free
//    form: row i <- a'_k R_i - (a_ik 2^-e_k) R_k with a_kk = a'_k 2^e_k,
//    a'_k in [1, 2): two FP64 instructions per element and step, no
//    division, one element per thread on the active columns only.  The left
//    block ends diagonal, d_i, and G~^-1 = diag(d)^-1 B;
//  * Sec. 4.3's singular test (Cholesky pivot D_k > 1e-14 max_i G_ii) is
//    taken after the elimination on the same pivots: the fraction-free pivot
//    is a_kk = m_k s_k^2 D_k, m_k = a'_0 ... a'_(k-1) the factor of row k;
//  * dot products over the QoIs run on groups of 8 lanes (3 warps for 12
//    QoIs), and the two divisions on different warps.
__device__ __forceinline__ int exp2_of(double a) {  // floor(log2 |a|) for a normal a
    return (int)((__double_as_longlong(a) >> 52) & 0x7ff) - 1023;
}
__device__ __forceinline__ double pow2(int e) {  // 2^e, -1022 <= e <= 1023
    return __longlong_as_double((long long)(e + 1023) << 52);
}
// x 2^e on the exponent field (integer operations only): exact for normal x
// and a normal result; zero and subnormal x give a signed zero, a result
// outside the normal range a signed zero or infinity
__device__ __forceinline__ double scale2(double x, int e) {
    const long long b = __double_as_longlong(x);
    const long long sign = b & (long long)0x8000000000000000ULL;
    const int ex = (int)((b >> 52) & 0x7ff);
    const int en = ex + e;
    if (ex == 0 || en <= 0) return __longlong_as_double(sign);
    if (en >= 2047 || ex == 2047) return __longlong_as_double(sign | 0x7ff0000000000000LL);
    return __longlong_as_double(b + ((long long)e << 52));
}
// the mantissa of a as a value in [1, 2) (a normal)
__device__ __forceinline__ double mant(double a) {
    return __longlong_as_double((__double_as_longlong(a) & 0x000FFFFFFFFFFFFFLL) | 0x3FF0000000000000LL);
}
// sum over groups of 8 consecutive lanes (every lane gets its group's sum)
__device__ __forceinline__ double group8_sum(double a) {
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    return a;
}
// G_ij from the totals (scale block, couplings) and the fixed band block
__device__ __forceinline__ double gram_entry(const Params& p, const Layout& L, int i, int j) {
    const int ns = p.n_s, np1 = 1 + ns, cpl = ns + ns * (ns + 1) / 2;
    if (i < ns && j < ns) {
        const int a = min(i, j), b = max(i, j);
        return L.tot[ns + a * ns - a * (a - 1) / 2 + (b - a)];
    }
    if (i >= ns && j >= ns) return L.g_mpmp[(size_t)(i - ns) * p.n_mp + (j - ns)];
    if (i >= ns) return L.tot[cpl + (i - ns) * np1 + 1 + j];
    return L.tot[cpl + (j - ns) * np1 + 1 + i];
}
// half the binary exponent of a diagonal entry (its scale is 2^-half)
__device__ __forceinline__ int half_exp(double gii) {
    const int e = gii > 1e-300 && gii < 1e300 ? exp2_of(gii) : 0;
    return e >> 1;  // floor(e / 2)
}

constexpr int kSolveThreads = 320;  // >= 16 x 17 + 15 active elements, plus a spare warp

__device__ __forceinline__ void solve_kernel_body(const VB& vb, const Params& p, const Layout& L) {
    constexpr int MQ = kMaxQoi;
    constexpr int MW = 2 * MQ + 1;
    const int ns = p.n_s, nmp = p.n_mp, nq = p.n_q;
    const int np1 = 1 + ns;
    const int cpl = ns + ns * (ns + 1) / 2;  // offset of the couplings in the totals
    __shared__ double M[2][MQ][MW];  // [G~ | I], ping-pong
    __shared__ double q[MQ], xq[MQ], dq[MQ], gam[MQ], ginv[MQ], wv[MQ], beta[MQ], qnew[MQ], rs[MQ];
    __shared__ double piv[MQ], mkv[MQ + 1];
    __shared__ long long diagbits[MQ];
    __shared__ int hexp[MQ];
    __shared__ int singular;
    const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
    const int gi = tid >> 3, gl = tid & 7;  // group of 8 lanes gi (output), lane gl
    const long long step = L.st->step;
    const bool lrs = p.to_mode == LBM_TO_LRS;
    const bool lrs_pred = lrs && step >= p.spinup;
    // loads needed late, issued now: the q^{n*} block of C (terms j = gl, gl + 8)
    double c_q0 = 0.0, c_q1 = 0.0;
    if (lrs_pred && gi < nq) {
        const size_t base = (size_t)p.h * nq;
        if (gl < nq) c_q0 = L.lrs_C[(base + gl) * nq + gi];
        if (gl + 8 < nq) c_q1 = L.lrs_C[(base + gl + 8) * nq + gi];
    }

    // 1. q^{n*} and G~ = S G S (one element per thread)
    for (int e = tid; e < nq * nq; e += blockDim.x) {
        const int i = e / nq, j = e - i * nq;
        const double gij = gram_entry(p, L, i, j);
        const double gii = i == j ? gij : gram_entry(p, L, i, i);
        const double gjj = i == j ? gij : gram_entry(p, L, j, j);
        M[0][i][j] = scale2(gij, -half_exp(gii) - half_exp(gjj));
        if (i == j) {
            diagbits[i] = __double_as_longlong(gij);
            hexp[i] = half_exp(gij);
        }
    }
    if (tid == 0) mkv[0] = 1.0;
    double sig = 0.0;
    if (tid < nq) {
        const int i = tid;
        q[i] = i < ns ? scale2(L.tot[i], -1) : L.tot[cpl + (i - ns) * np1];
        if (lrs) {
            // a reference scale <= 0 is taken from this step's predictor QoI
            sig = L.lrs_sigma[i];
            if (!(sig > 0.0)) {
                sig = fabs(q[i]) > 0.0 ? fabs(q[i]) : 1.0;
                L.lrs_sigma[i] = sig;
            }
        }
    }
    __syncthreads();

    // 2. fraction-free Gauss-Jordan on [G~ | I].  At step k only the active
    //    part is touched: the left columns k.., the right columns ..k and the
    //    left diagonal entries (i, i), i < k (their columns are eliminated,
    //    so they are only scaled).  Right column k enters as e_k times the
    //    factor m_k of row k.  The last warp carries m_k and the pivots.
    int cur = 0;
    for (int k = 0; k < nq; ++k) {
        const double akk = M[cur][k][k];
        const int ek = exp2_of(akk);
        const double ap = mant(akk);  // akk 2^-ek, in [1, 2)
        const int act = nq * (nq + 1);
        if (tid < act + k) {
            int i, j;
            if (tid < act) {
                i = tid / (nq + 1);
                const int c = tid - i * (nq + 1);
                j = c < nq - k ? k + c : nq + (c - (nq - k));
            } else {
                i = j = tid - act;
            }
            const bool fresh = j == nq + k;  // right column entering the active set
            const double mk = mkv[k];
            const double mij = fresh ? (i == k ? mk : 0.0) : M[cur][i][j];
            double r = mij;
            if (tid >= act) {
                r = ap * mij;  // eliminated column: row k holds 0 there
            } else if (i != k) {
                const double mkj = fresh ? mk : M[cur][k][j];
                r = fma(-scale2(M[cur][i][k], -ek), mkj, ap * mij);
            }
            M[cur ^ 1][i][j] = r;
        }
        if (tid == kSolveThreads - 32) {
            piv[k] = akk;
            mkv[k + 1] = mkv[k] * ap;
        }
        cur ^= 1;
        __syncthreads();
    }

    // 3. the singular test on the pivots (warp 0); the two divisions
    //    1 / d_i (warp 0) and q_i / sigma_i (warp 1) on different warps
    if (wid == 0) {
        long long dmb = 0;  // max_i G_ii on the bit patterns: non-negative doubles
        for (int i = 0; i < nq; ++i) dmb = max(dmb, diagbits[i]);  // order as integers; NaN propagates
        const double dmax = __longlong_as_double(dmb);
        bool bad = false;
        if (lane < nq) {
            const double a = piv[lane];
            bad = !(a > scale2(1e-14 * dmax, -2 * hexp[lane]) * mkv[lane]) || !(a < 1e300);
        }
        const bool sing = __any_sync(0xffffffffu, bad) || !(dmax > 0.0) || isinf(dmax);
        if (lane == 0) singular = sing;
        if (lane < nq && !sing) {
            const int i = lane;
            const double invd = 1.0 / M[cur][i][i];
            rs[i] = scale2(invd, -hexp[i]);
            ginv[i] = scale2(M[cur][i][nq + i] * invd, -2 * hexp[i]);
        }
    } else if (wid == 1 && lrs_pred && lane < nq) {
        xq[lane] = q[lane] / L.lrs_sigma[lane];
    }
    __syncthreads();
    const bool sing = singular;
    // 4. coefficient source -> dQ, gamma (group gi forms the LRS product of QoI gi)
    if (lrs_pred) {
        double t = 0.0;
        // lanes past the last QoI read nothing (shared memory there is not initialised)
        if (gi < nq && gl < nq) t = xq[gl] * c_q0 + (gl + 8 < nq ? xq[gl + 8] * c_q1 : 0.0);
        t = group8_sum(t);
        if (gl == 0 && gi < nq) qnew[gi] = L.lrs_sigma[gi] * (L.hsum[gi] + t);  // corrected QoI for the history
    }
    __syncthreads();
    if (tid < nq) {
        const int i = tid;
        const double gii = sing ? 0.0 : ginv[i];
        double d = 0.0, g = 0.0;
        if (lrs && step < p.spinup) {
            // spin-up: nudged to the reference, which enters the history
            const long long row = step < p.track_len ? step : p.track_len - 1;
            const double qref = L.track[(size_t)row * nq + i];
            d = qref - q[i];
            qnew[i] = qref;
            g = d * gii;
        } else if (lrs) {
            d = qnew[i] - q[i];
            g = d * gii;
        } else if (p.to_mode == LBM_TO_GAMMA) {
            if (!sing) {
                g = p.gamma_std * L.znorm[i];
                d = g / gii;
            }
        } else if (p.to_mode == LBM_TO_FIXED_GAMMA) {
            if (!sing) {
                g = L.gfix[i];
                d = g / gii;
            }
        } else if (p.to_mode == LBM_TO_TRACK) {
            const long long row = step < p.track_len ? step : p.track_len - 1;
            d = L.track[(size_t)row * nq + i] - q[i];
            g = d * gii;
        }
        dq[i] = d;
        gam[i] = g;
        wv[i] = sing ? 0.0 : scale2(d, -hexp[i]);
    }
    __syncthreads();
    // 5. beta = G^-1 dQ = (s_i / d_i) sum_j B_ij s_j dQ_j (group gi forms beta_gi)
    const bool skip = sing || p.to_mode == LBM_TO_OBSERVE;
    if (!skip) {
        double t = 0.0;
        if (gi < nq && gl < nq) {
            t = M[cur][gi][nq + gl] * wv[gl];
            if (gl + 8 < nq) t = fma(M[cur][gi][nq + gl + 8], wv[gl + 8], t);
        }
        t = group8_sum(t);
        if (gl == 0 && gi < nq) beta[gi] = rs[gi] * t;
    } else if (tid < nq) {
        beta[tid] = 0.0;
    }
    __syncthreads();
    // 6. QoI block row and histories (thread i = QoI i)
    const long long rc = L.st->ring_count;
    double* row = L.ring + (size_t)(rc % p.ring_cap) * p.row_len;
    if (tid < nq) {
        const int i = tid;
        L.beta[i] = beta[i];
        row[1 + i] = q[i];
        row[1 + nq + i] = dq[i];
        row[1 + 2 * nq + i] = gam[i];
        if (lrs) {
            const long long slot = L.st->hist_pos % p.h;
            L.qh[slot * nq + i] = qnew[i];
            L.qsh[slot * nq + i] = q[i];
        }
    }
    if (tid == 32) {
        row[0] = (double)step;
        unsigned fl = sing ? LBM_FLAG_SINGULAR : 0u;
        if (L.st->status & 1u) fl |= LBM_FLAG_UNSTABLE;
        row[1 + 3 * nq] = (double)fl;
    }
    // 7. mean profile of the corrected velocity: P_v + sum_k beta_k P_k + nx nz sum_j beta_mp_j w_j;
    //    the corrector's inputs in FP32: beta_k and, per row, sum_j beta_j w_j(y)
    if (tid < nq) L.betaf[tid] = (float)beta[tid];
    for (int y = tid; y < p.ny; y += blockDim.x) {
        const double* ps = L.plane_sum + (size_t)y * np1;
        double a = ps[0], b = 0.0;
        float mp = 0.f;
        for (int k = 0; k < ns; ++k) a = fma(beta[k], ps[1 + k], a);
        for (int j = 0; j < nmp; ++j) {
            const double wb = beta[ns + j] * L.w_mp[(size_t)j * p.ny + y];
            b = fma(beta[ns + j], L.w_mp[(size_t)j * p.ny + y], b);
            mp += (float)wb;
        }
        L.profile[y] += fma(a, p.inv_area, b);
        L.mprow[y] = mp;
    }
    __syncthreads();
    if (tid == 0) {
        L.st->ring_count = rc + 1;
        if (lrs) L.st->hist_pos += 1;
        L.st->prof_steps += 1;
        L.st->step = step + 1;
    }
}
struct solve_kernel_op {
    static constexpr int NT = kSolveThreads, MINB = 1;
    template <class... B>
    static __device__ __forceinline__ void run(const VB& vb, const B&... b) {
        solve_kernel_body(vb, b...);
    }
};
__global__ void __launch_bounds__(kSolveThreads) solve_kernel(Params p, Layout L) {
    solve_kernel_body(vb_hw(), p, L);
}

// ------------------------------------------------- QoIs of a given field --
// The QoI path on a velocity field supplied by the caller (a projected HF
// field): u [3][N] into the filter input with the solid rows zeroed, then,
// after the filters, reduction and totals, q_i = Q_i(u) (Eqs. scale-aware-
// energy / enstrophy: half the squared norms; the bands: sum_y w_j(y) P_0(y)).
__global__ void __launch_bounds__(256) load_velocity_kernel(Params p, const float* __restrict__ u,
                                                            float* __restrict__ x6) {
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= p.n) return;
    const size_t N = (size_t)p.n;
    const int y = (int)((n / p.nx) % p.ny);
    const bool solid = p.walls && (y == 0 || y == p.ny - 1);
    for (int c = 0; c < p.dim; ++c) x6[c * N + n] = solid ? 0.f : u[c * N + n];
}

__global__ void qoi_values_kernel(Params p, Layout L, double* __restrict__ q) {
    const int i = threadIdx.x;
    const int ns = p.n_s, np1 = 1 + ns, cpl = ns + ns * (ns + 1) / 2;
    if (i < p.n_q) q[i] = i < ns ? 0.5 * L.tot[i] : L.tot[cpl + (i - ns) * np1];
}

// ------------------------------------------------------------ launchers --
static inline unsigned gridn(long long n, int b) { return (unsigned)((n + b - 1) / b); }

static bool quads_ok(const Params& p, const float* a, const float* b) {
    return p.nx % 4 == 0 && ((uintptr_t)a & 15) == 0 && ((uintptr_t)b & 15) == 0;
}
cudaError_t launch_to_curl(const Params& p, const Layout& L, cudaStream_t s) {
    float* om = L.x6 + (size_t)p.dim * p.n;
    if (quads_ok(p, L.x6, om)) {
        if (p.dim == 3)
            go<curl4_kernel_op<kCurl3>>(curl4_kernel<kCurl3>, gridn(p.n / 4, 256), 256, 0, s, p, L.x6, om);
        else
            go<curl4_kernel_op<kVort2>>(curl4_kernel<kVort2>, gridn(p.n / 4, 256), 256, 0, s, p, L.x6, om);
        return cudaGetLastError();
    }
    go<curl_kernel_op>(curl_kernel, gridn(p.n, 256), 256, 0, s, p, L.x6);
    return cudaGetLastError();
}
cudaError_t launch_pass(const Params& p, const float* in, float* out, int ncomp, int axis, const Taps& t, float scale,
                        int accumulate, cudaStream_t s) {
    const cudaError_t e = launch_pass_fast(p, in, out, ncomp, axis, t, scale, accumulate, s);
    if (e != cudaErrorNotSupported) return e;
    go<pass_kernel_op>(pass_kernel, gridn(p.n, 256), 256, 0, s, p, in, out, ncomp, axis, t, scale, accumulate);
    return cudaGetLastError();
}
cudaError_t launch_band_mask(const Params& p, const float2* in, float2* out, int ncomp, int lo, int hi,
                             cudaStream_t s) {
    if (g_rec) {  // the transforms around it are library calls: not batched
        rec_refuse("Fourier band mask");
        return cudaSuccess;
    }
    const long long n = (long long)p.ny * (p.nx / 2 + 1) * ncomp;
    band_mask_kernel<<<gridn(n, 256), 256, 0, s>>>(p, in, out, ncomp, lo, hi);
    return cudaGetLastError();
}
cudaError_t launch_sens_curl(const Params& p, const float* w, float* out, cudaStream_t s) {
    if (quads_ok(p, w, out)) {
        if (p.dim == 3)
            go<curl4_kernel_op<kCurl3>>(curl4_kernel<kCurl3>, gridn(p.n / 4, 256), 256, 0, s, p, w, out);
        else
            go<curl4_kernel_op<kSens2>>(curl4_kernel<kSens2>, gridn(p.n / 4, 256), 256, 0, s, p, w, out);
        return cudaGetLastError();
    }
    go<sens_curl_kernel_op>(sens_curl_kernel, gridn(p.n, 256), 256, 0, s, p, w, out);
    return cudaGetLastError();
}
template <int NS>
static void go_reduce(const Params& p, const Layout& L, const RedPtrs& r, dim3 grid, cudaStream_t s) {
    go<reduce_kernel_op<NS>>(reduce_kernel<NS>, grid, 128, 0, s, p, L.vps, r, L.w_mp2, L.part, L.plane_part);
}
cudaError_t launch_reduce(const Params& p, const Layout& L, const float* const* vk, cudaStream_t s) {
    RedPtrs r;
    for (int k = 0; k < kMaxQoi; ++k) r.v[k] = k < p.n_s ? vk[k] : nullptr;
    dim3 grid(p.ny, p.nzc);
    switch (p.n_s) {
        case 1: go_reduce<1>(p, L, r, grid, s); break;
        case 2: go_reduce<2>(p, L, r, grid, s); break;
        case 3: go_reduce<3>(p, L, r, grid, s); break;
        case 4: go_reduce<4>(p, L, r, grid, s); break;
        case 5: go_reduce<5>(p, L, r, grid, s); break;
        case 6: go_reduce<6>(p, L, r, grid, s); break;
        case 7: go_reduce<7>(p, L, r, grid, s); break;
        case 8: go_reduce<8>(p, L, r, grid, s); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}
cudaError_t launch_lrs_pre(const Params& p, const Layout& L, cudaStream_t s) {
    const int nb = p.to_mode == LBM_TO_LRS ? p.nblk_lrs : 0;
    go<lrs_pre_kernel_op>(lrs_pre_kernel, nb + 1, 256, 0, s, p, L, nb);
    return cudaGetLastError();
}
cudaError_t launch_totals(const Params& p, const Layout& L, bool with_lrs, cudaStream_t s) {
    const int nplane_blk = (p.ny * (1 + p.n_s) + 7) / 8;
    const int nb = p.ntot + nplane_blk + (with_lrs && p.to_mode == LBM_TO_LRS ? p.n_q : 0);
    go<totals_kernel_op>(totals_kernel, nb, 256, 0, s, p, L, nplane_blk);
    return cudaGetLastError();
}
cudaError_t launch_solve(const Params& p, const Layout& L, cudaStream_t s) {
    go<solve_kernel_op>(solve_kernel, 1, kSolveThreads, 0, s, p, L);
    return cudaGetLastError();
}

}  // namespace lbm

namespace lbm {
cudaError_t launch_load_velocity(const Params& p, const Layout& L, const float* u, cudaStream_t s) {
    load_velocity_kernel<<<(unsigned)((p.n + 255) / 256), 256, 0, s>>>(p, u, L.x6);
    return cudaGetLastError();
}
cudaError_t launch_qoi_values(const Params& p, const Layout& L, double* q, cudaStream_t s) {
    qoi_values_kernel<<<1, 32, 0, s>>>(p, L, q);
    return cudaGetLastError();
}
}  // namespace lbm
