// Fused 3-D compact filters (Sec. 4.1): one kernel applies a whole filter.
//
// A block owns a TX x TY tile of (x, y) and marches along a segment of z.
// For every input plane it stages the tile plus halo in shared memory
// (coalesced loads, prefetched into registers one plane ahead), applies the
// x and y factors in shared memory, and pushes the result into per-thread
// register rings along z, from which the z factor produces one output plane
// per step.  Each input element is read from DRAM about once per application
// (halo re-reads hit L2) and each output written once, instead of one read and
// one write per 1-D factor.
//
//   gauss3_kernel<R>      G_s (or B3): the same (2R+1)-tap factor on x, y, z
//   lap3_kernel<RA, RB>   L_s = c sum_a [l dilated along a] x [box_s on the
//                         other two axes], arm radius RA = (5s-1)/2, box
//                         radius RB = (s-1)/2 (RB = 0: the box is the identity)
//
// Periodic along x and z; along y with walls the halo outside the array reads
// zero (solid rows already hold zero), and outputs on solid rows are zero, so
// the kernel applies P K P exactly.  One component per blockIdx.z slice.
#include "lbm_common.cuh"

namespace lbm {

namespace {
constexpr int TX = 32, TY = 16, NT = TX * TY;

template <int R> struct T3 {
    float t[2 * R + 1];
};

__device__ __forceinline__ int pm(int a, int n) {
    int r = a % n;
    return r < 0 ? r + n : r;
}

// global -> register prefetch of one (TY + 2H) x (TX + 2H) plane tile
template <int H>
struct TileLoader {
    static constexpr int W = TX + 2 * H, HH = TY + 2 * H, SZ = W * HH, PER = (SZ + NT - 1) / NT;
    float r[PER];
    __device__ __forceinline__ void load(const Params& p, const float* __restrict__ a, int x0, int y0, int zq) {
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int i = threadIdx.x + k * NT;
            float v = 0.f;
            if (i < SZ) {
                const int ly = i / W, lx = i % W;
                int gy = y0 - H + ly;
                const int gx = pm(x0 - H + lx, p.nx);
                bool ok = true;
                if (p.walls) ok = gy >= 0 && gy < p.ny;
                else gy = pm(gy, p.ny);
                if (ok) v = __ldg(a + ((size_t)zq * p.ny + gy) * p.nx + gx);
            }
            r[k] = v;
        }
    }
    __device__ __forceinline__ void store(float* tile) {
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int i = threadIdx.x + k * NT;
            if (i < SZ) tile[i] = r[k];
        }
    }
};

template <int R>
__global__ void __launch_bounds__(NT) gauss3_kernel(Params p, const float* __restrict__ in, float* __restrict__ out,
                                                    T3<R> tp, float scale, int accumulate, int ncomp, int seg) {
    constexpr int W = TX + 2 * R, HH = TY + 2 * R;
    __shared__ float tile[HH * W];
    __shared__ float txs[HH * TX];
    const int c = blockIdx.z % ncomp, zs = blockIdx.z / ncomp;
    const int nz = p.nz;
    const int z0 = zs * seg, z1 = min(nz, z0 + seg);
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int lx = threadIdx.x % TX, ly = threadIdx.x / TX;
    const int x = x0 + lx, y = y0 + ly;
    const size_t N = (size_t)p.n;
    const float* a = in + c * N;
    float* o = out + c * N;
    const bool live = x < p.nx && y < p.ny;
    const bool solid = p.walls && (y == 0 || y == p.ny - 1);
    float ring[2 * R + 1];
#pragma unroll
    for (int k = 0; k < 2 * R + 1; ++k) ring[k] = 0.f;
    TileLoader<R> ld;
    ld.load(p, a, x0, y0, pm(z0 - R, nz));
    for (int q = z0 - R; q < z1 + R; ++q) {
        ld.store(tile);
        __syncthreads();
        if (q + 1 < z1 + R) ld.load(p, a, x0, y0, pm(q + 1, nz));
        // x factor on all tile rows
        for (int i = threadIdx.x; i < HH * TX; i += NT) {
            const int ry = i / TX, rx = i % TX;
            float s = 0.f;
#pragma unroll
            for (int r = -R; r <= R; ++r) s += tp.t[r + R] * tile[ry * W + rx + R - r];
            txs[i] = s;
        }
        __syncthreads();
        // y factor for this thread's point
        float s = 0.f;
#pragma unroll
        for (int r = -R; r <= R; ++r) s += tp.t[r + R] * txs[(ly + R - r) * TX + lx];
#pragma unroll
        for (int k = 0; k < 2 * R; ++k) ring[k] = ring[k + 1];
        ring[2 * R] = s;
        // z factor: ring[k] holds plane q - 2R + k; output plane z = q - R
        const int zo = q - R;
        if (zo >= z0 && live) {
            float v = 0.f;
#pragma unroll
            for (int r = -R; r <= R; ++r) v += tp.t[r + R] * ring[R - r];
            v = solid ? 0.f : scale * v;
            float* op = o + ((size_t)zo * p.ny + y) * p.nx + x;
            *op = accumulate ? (*op + v) : v;
        }
        __syncthreads();
    }
}

template <int RA, int RB>
__global__ void __launch_bounds__(NT) lap3_kernel(Params p, const float* __restrict__ in, float* __restrict__ out,
                                                  T3<RA> arm, float scale, int accumulate, int ncomp, int seg) {
    constexpr int W = TX + 2 * RA, HH = TY + 2 * RA;
    __shared__ float tile[HH * W];
    __shared__ float by[TY * W];   // box along y on the output rows, all tile columns
    __shared__ float bx[HH * TX];  // box along x on all tile rows, output columns
    const int c = blockIdx.z % ncomp, zs = blockIdx.z / ncomp;
    const int nz = p.nz;
    const int z0 = zs * seg, z1 = min(nz, z0 + seg);
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int lx = threadIdx.x % TX, ly = threadIdx.x / TX;
    const int x = x0 + lx, y = y0 + ly;
    const size_t N = (size_t)p.n;
    const float* a = in + c * N;
    float* o = out + c * N;
    const bool live = x < p.nx && y < p.ny;
    const bool solid = p.walls && (y == 0 || y == p.ny - 1);
    // rings along z: rx = l_x(B_y plane), ry = l_y(B_x plane), rz = B_y(B_x plane)
    float rx[2 * RA + 1], ry[2 * RA + 1], rz[2 * RA + 1];
#pragma unroll
    for (int k = 0; k < 2 * RA + 1; ++k) rx[k] = ry[k] = rz[k] = 0.f;
    TileLoader<RA> ld;
    ld.load(p, a, x0, y0, pm(z0 - RA, nz));
    for (int q = z0 - RA; q < z1 + RA; ++q) {
        ld.store(tile);
        __syncthreads();
        if (q + 1 < z1 + RA) ld.load(p, a, x0, y0, pm(q + 1, nz));
        for (int i = threadIdx.x; i < TY * W; i += NT) {
            const int ry_ = i / W, rx_ = i % W;
            float s = 0.f;
#pragma unroll
            for (int r = -RB; r <= RB; ++r) s += tile[(ry_ + RA - r) * W + rx_];
            by[i] = s;
        }
        for (int i = threadIdx.x; i < HH * TX; i += NT) {
            const int ry_ = i / TX, rx_ = i % TX;
            float s = 0.f;
#pragma unroll
            for (int r = -RB; r <= RB; ++r) s += tile[ry_ * W + rx_ + RA - r];
            bx[i] = s;
        }
        __syncthreads();
        float ax = 0.f, ay = 0.f, az = 0.f;
#pragma unroll
        for (int r = -RA; r <= RA; ++r) {
            ax += arm.t[r + RA] * by[ly * W + lx + RA - r];
            ay += arm.t[r + RA] * bx[(ly + RA - r) * TX + lx];
        }
#pragma unroll
        for (int r = -RB; r <= RB; ++r) az += bx[(ly + RA - r) * TX + lx];
#pragma unroll
        for (int k = 0; k < 2 * RA; ++k) {
            rx[k] = rx[k + 1];
            ry[k] = ry[k + 1];
            rz[k] = rz[k + 1];
        }
        rx[2 * RA] = ax;
        ry[2 * RA] = ay;
        rz[2 * RA] = az;
        const int zo = q - RA;
        if (zo >= z0 && live) {
            float v = 0.f;
#pragma unroll
            for (int r = -RB; r <= RB; ++r) v += rx[RA - r] + ry[RA - r];
#pragma unroll
            for (int r = -RA; r <= RA; ++r) v += arm.t[r + RA] * rz[RA - r];
            v = solid ? 0.f : scale * v;
            float* op = o + ((size_t)zo * p.ny + y) * p.nx + x;
            *op = accumulate ? (*op + v) : v;
        }
        __syncthreads();
    }
}

int seg_len(const Params& p, int blocks_xy, int ncomp, int R) {
    // enough z segments for ~4 blocks per SM; each segment re-reads 2R planes
    const long long want = 148LL * 4;
    long long nseg = (want + (long long)blocks_xy * ncomp - 1) / ((long long)blocks_xy * ncomp);
    if (nseg < 1) nseg = 1;
    int seg = (int)((p.nz + nseg - 1) / nseg);
    if (seg < 4 * R) seg = 4 * R;
    if (seg > p.nz) seg = p.nz;
    return seg;
}

template <int R>
cudaError_t run_gauss(const Params& p, const float* in, float* out, int ncomp, const Taps& t, float scale, int acc,
                      cudaStream_t s) {
    T3<R> tp;
    for (int i = 0; i < 2 * R + 1; ++i) tp.t[i] = t.t[i];
    const int bx = (p.nx + TX - 1) / TX, by = (p.ny + TY - 1) / TY;
    const int seg = seg_len(p, bx * by, ncomp, R);
    const int nseg = (p.nz + seg - 1) / seg;
    gauss3_kernel<R><<<dim3(bx, by, ncomp * nseg), NT, 0, s>>>(p, in, out, tp, scale, acc, ncomp, seg);
    return cudaGetLastError();
}

template <int RA, int RB>
cudaError_t run_lap(const Params& p, const float* in, float* out, int ncomp, const Taps& arm, float scale, int acc,
                    cudaStream_t s) {
    T3<RA> tp;
    for (int i = 0; i < 2 * RA + 1; ++i) tp.t[i] = arm.t[i];
    const int bx = (p.nx + TX - 1) / TX, by = (p.ny + TY - 1) / TY;
    const int seg = seg_len(p, bx * by, ncomp, RA);
    const int nseg = (p.nz + seg - 1) / seg;
    lap3_kernel<RA, RB><<<dim3(bx, by, ncomp * nseg), NT, 0, s>>>(p, in, out, tp, scale, acc, ncomp, seg);
    return cudaGetLastError();
}
}  // namespace

// G_s / B3 in 3-D with the same 1-D taps on every axis.
cudaError_t launch_gauss3(const Params& p, const float* in, float* out, int ncomp, const Taps& t, float scale,
                          int accumulate, cudaStream_t s) {
    switch (t.radius) {
        case 1: return run_gauss<1>(p, in, out, ncomp, t, scale, accumulate, s);
        case 2: return run_gauss<2>(p, in, out, ncomp, t, scale, accumulate, s);
        case 4: return run_gauss<4>(p, in, out, ncomp, t, scale, accumulate, s);
        case 6: return run_gauss<6>(p, in, out, ncomp, t, scale, accumulate, s);
        default: return cudaErrorNotSupported;
    }
}

// L_s in 3-D for s = 1 (arm radius 2, no box) and s = 3 (arm 7, box 1).
cudaError_t launch_lap3(const Params& p, const float* in, float* out, int ncomp, int s_scale, const Taps& arm,
                        float scale, int accumulate, cudaStream_t s) {
    if (s_scale == 1 && arm.radius == 2) return run_lap<2, 0>(p, in, out, ncomp, arm, scale, accumulate, s);
    if (s_scale == 3 && arm.radius == 7) return run_lap<7, 1>(p, in, out, ncomp, arm, scale, accumulate, s);
    return cudaErrorNotSupported;
}

}  // namespace lbm
