// Fused 3-D compact filters (Sec. 4.1): one kernel applies a whole filter.
//
// A block owns a TX x TY tile of (x, y) and marches along a segment of z.
// For every input plane it stages the tile plus halo in shared memory
// (coalesced loads, prefetched into registers one plane ahead), applies the
// x and y factors with register sliding windows (a thread produces 8 x-values
// of a row from 8 + 2R staged values, or RPT y-values of a column from
// RPT + 2R), and pushes the result into per-thread register rings along z,
// from which the z factor produces one output plane per step.  Each input
// element is read from DRAM about once per application (halo re-reads hit L2)
// and each output written once.
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
constexpr int TX = 32, TY = 16;

template <int R> struct T3 {
    float t[2 * R + 1];
};

__device__ __forceinline__ int pm(int a, int n) {
    int r = a % n;
    return r < 0 ? r + n : r;
}

__host__ __device__ constexpr int round4(int v) { return (v + 3) & ~3; }

// global -> register prefetch of one (TY + 2H) x Wp plane tile (Wp = TX + 2H
// rounded up to a multiple of 4 so that rows are 16-byte aligned).  The
// in-plane offset of every staged element (or -1 for the zero extension) is
// computed once per block: only the plane offset changes along z.
template <int H, int NT>
struct TileLoader {
    static constexpr int W = TX + 2 * H, WP = round4(W), HH = TY + 2 * H, SZ = WP * HH, PER = (SZ + NT - 1) / NT;
    float r[PER];
    int off[PER];
    __device__ __forceinline__ void init(const Params& p, int x0, int y0) {
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int i = threadIdx.x + k * NT;
            int o = -1;
            if (i < SZ) {
                const int ly = i / WP, lx = i % WP;
                if (lx < W) {
                    int gy = y0 - H + ly;
                    const int gx = pm(x0 - H + lx, p.nx);
                    bool ok = true;
                    if (p.walls) ok = gy >= 0 && gy < p.ny;
                    else gy = pm(gy, p.ny);
                    if (ok) o = gy * p.nx + gx;
                }
            }
            off[k] = o;
        }
    }
    __device__ __forceinline__ void load(const Params& p, const float* __restrict__ a, int zq) {
        const float* plane = a + (size_t)zq * p.ny * p.nx;
#pragma unroll
        for (int k = 0; k < PER; ++k) r[k] = off[k] >= 0 ? __ldg(plane + off[k]) : 0.f;
    }
    __device__ __forceinline__ void store(float* tile) {
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int i = threadIdx.x + k * NT;
            if (i < SZ) tile[i] = r[k];
        }
    }
};

// 8 consecutive outputs of a 1-D convolution along a shared-memory row:
// out[j] = sum_r t(r) row[j + R - r], row 16-byte aligned, 8 + 2R values used.
template <int R>
__device__ __forceinline__ void conv8(const float* row, const float* t, float* out) {
    constexpr int NV = round4(8 + 2 * R);
    float v[NV];
#pragma unroll
    for (int k = 0; k < NV; k += 4) {
        const float4 q = *reinterpret_cast<const float4*>(row + k);
        v[k] = q.x; v[k + 1] = q.y; v[k + 2] = q.z; v[k + 3] = q.w;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        float s = 0.f;
#pragma unroll
        for (int r = -R; r <= R; ++r) s += t[r + R] * v[j + R - r];
        out[j] = s;
    }
}

template <int R>
__global__ void __launch_bounds__(128) gauss3_kernel(Params p, const float* __restrict__ in, float* __restrict__ out,
                                                     T3<R> tp, float scale, int accumulate, int ncomp, int seg) {
    constexpr int NT = 128, RPT = TY / (NT / TX);  // 4 output rows per thread
    using LD = TileLoader<R, NT>;
    constexpr int WP = LD::WP, HH = LD::HH;
    __shared__ __align__(16) float tile[HH * WP];
    __shared__ __align__(16) float xt[HH * TX];
    const int c = blockIdx.z % ncomp, zs = blockIdx.z / ncomp;
    const int nz = p.nz;
    const int z0 = zs * seg, z1 = min(nz, z0 + seg);
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int lx = threadIdx.x % TX, yr = threadIdx.x / TX;
    const int x = x0 + lx;
    const size_t N = (size_t)p.n;
    const float* a = in + c * N;
    float* o = out + c * N;
    float ring[RPT][2 * R + 1];
#pragma unroll
    for (int j = 0; j < RPT; ++j)
#pragma unroll
        for (int k = 0; k < 2 * R + 1; ++k) ring[j][k] = 0.f;
    LD ld;
    ld.init(p, x0, y0);
    ld.load(p, a, pm(z0 - R, nz));
    // Two barriers per plane: the x factor reads `tile` only before the second
    // barrier and the y factor reads `xt` only before the next plane's first,
    // so the next plane's stores cannot overtake a reader.
    for (int q = z0 - R; q < z1 + R; ++q) {
        ld.store(tile);
        __syncthreads();
        if (q + 1 < z1 + R) ld.load(p, a, pm(q + 1, nz));
        // x factor: task = (tile row, 8-wide segment)
        for (int task = threadIdx.x; task < HH * (TX / 8); task += NT) {
            const int ry = task / (TX / 8), k = task % (TX / 8);
            float r8[8];
            conv8<R>(tile + ry * WP + 8 * k, tp.t, r8);
            float4* dst = reinterpret_cast<float4*>(xt + ry * TX + 8 * k);
            dst[0] = make_float4(r8[0], r8[1], r8[2], r8[3]);
            dst[1] = make_float4(r8[4], r8[5], r8[6], r8[7]);
        }
        __syncthreads();
        // y factor: RPT consecutive rows of column lx from RPT + 2R values
        float col[RPT + 2 * R];
#pragma unroll
        for (int m = 0; m < RPT + 2 * R; ++m) col[m] = xt[(yr * RPT + m) * TX + lx];
        const int zo = q - R;
#pragma unroll
        for (int j = 0; j < RPT; ++j) {
            float s = 0.f;
#pragma unroll
            for (int r = -R; r <= R; ++r) s += tp.t[r + R] * col[j + R - r];
#pragma unroll
            for (int k = 0; k < 2 * R; ++k) ring[j][k] = ring[j][k + 1];
            ring[j][2 * R] = s;
            const int y = y0 + yr * RPT + j;
            if (zo >= z0 && x < p.nx && y < p.ny) {
                float v = 0.f;
#pragma unroll
                for (int r = -R; r <= R; ++r) v += tp.t[r + R] * ring[j][R - r];
                const bool solid = p.walls && (y == 0 || y == p.ny - 1);
                v = solid ? 0.f : scale * v;
                float* op = o + ((size_t)zo * p.ny + y) * p.nx + x;
                *op = accumulate ? (*op + v) : v;
            }
        }
    }
}

// L_s with a box (s > 1): double-buffered shared arrays, two barriers per
// plane.  Phase A (after the tile of plane q is stored): box along y on the
// output rows and box along x on every tile row.  Phase B: the three terms of
// this thread's points, pushed into the z rings.  A buffer written in phase A
// of plane q was last read in phase B of plane q-2, which every thread left
// before the first barrier of plane q-1.
template <int RA, int RB>
__global__ void __launch_bounds__(256) lap3_kernel(Params p, const float* __restrict__ in, float* __restrict__ out,
                                                   T3<RA> arm, float scale, int accumulate, int ncomp, int seg) {
    constexpr int NT = 256, RPT = TY / (NT / TX);  // 2 output rows per thread
    using LD = TileLoader<RA, NT>;
    constexpr int WP = LD::WP, HH = LD::HH, W = LD::W;
    constexpr int KXY = RA + RB + 1;  // ring of l_x B_y + l_y B_x (box along z later)
    constexpr int KZ = 2 * RA + 1;    // ring of B_x B_y (arm along z later)
    __shared__ __align__(16) float tile[2][HH * WP];
    __shared__ __align__(16) float by[2][TY * WP];  // box along y on the output rows, every tile column
    __shared__ __align__(16) float bx[2][HH * TX];  // box along x on every tile row, output columns
    const int c = blockIdx.z % ncomp, zs = blockIdx.z / ncomp;
    const int nz = p.nz;
    const int z0 = zs * seg, z1 = min(nz, z0 + seg);
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int lx = threadIdx.x % TX, yr = threadIdx.x / TX;
    const int x = x0 + lx;
    const size_t N = (size_t)p.n;
    const float* a = in + c * N;
    float* o = out + c * N;
    float rxy[RPT][KXY], rz[RPT][KZ];
#pragma unroll
    for (int j = 0; j < RPT; ++j) {
#pragma unroll
        for (int k = 0; k < KXY; ++k) rxy[j][k] = 0.f;
#pragma unroll
        for (int k = 0; k < KZ; ++k) rz[j][k] = 0.f;
    }
    LD ld;
    ld.init(p, x0, y0);
    ld.load(p, a, pm(z0 - RA, nz));
    int b = 0;
    for (int q = z0 - RA; q < z1 + RA; ++q, b ^= 1) {
        ld.store(tile[b]);
        __syncthreads();
        if (q + 1 < z1 + RA) ld.load(p, a, pm(q + 1, nz));
        const float* tl = tile[b];
        for (int task = threadIdx.x; task < W * (TY / 4); task += NT) {
            const int cx = task % W, run = task / W;
            float v[4 + 2 * RB];
#pragma unroll
            for (int m = 0; m < 4 + 2 * RB; ++m) v[m] = tl[(run * 4 + RA - RB + m) * WP + cx];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float s = 0.f;
#pragma unroll
                for (int r = 0; r <= 2 * RB; ++r) s += v[j + r];
                by[b][(run * 4 + j) * WP + cx] = s;
            }
        }
        for (int task = threadIdx.x; task < HH * (TX / 8); task += NT) {
            const int ry = task / (TX / 8), k = task % (TX / 8);
            const float* row = tl + ry * WP + 8 * k + RA - RB;
            float v[8 + 2 * RB];
#pragma unroll
            for (int m = 0; m < 8 + 2 * RB; ++m) v[m] = row[m];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                float s = 0.f;
#pragma unroll
                for (int r = 0; r <= 2 * RB; ++r) s += v[j + r];
                bx[b][ry * TX + 8 * k + j] = s;
            }
        }
        __syncthreads();
        const float* byb = by[b];
        const float* bxb = bx[b];
        float col[RPT + 2 * RA];
#pragma unroll
        for (int m = 0; m < RPT + 2 * RA; ++m) col[m] = bxb[(yr * RPT + m) * TX + lx];
        const int zo = q - RA;
#pragma unroll
        for (int j = 0; j < RPT; ++j) {
            // arm along x of by at (row, lx) and along y of bx, symmetric taps
            const float* br = byb + (yr * RPT + j) * WP + lx;
            float ax = arm.t[RA] * br[RA];
            float ay = arm.t[RA] * col[j + RA];
#pragma unroll
            for (int r = 1; r <= RA; ++r) {
                ax += arm.t[RA + r] * (br[RA - r] + br[RA + r]);
                ay += arm.t[RA + r] * (col[j + RA - r] + col[j + RA + r]);
            }
            float az = 0.f;
#pragma unroll
            for (int r = -RB; r <= RB; ++r) az += col[j + RA - r];
#pragma unroll
            for (int k = 0; k < KXY - 1; ++k) rxy[j][k] = rxy[j][k + 1];
            rxy[j][KXY - 1] = ax + ay;
#pragma unroll
            for (int k = 0; k < KZ - 1; ++k) rz[j][k] = rz[j][k + 1];
            rz[j][KZ - 1] = az;
            const int y = y0 + yr * RPT + j;
            if (zo >= z0 && x < p.nx && y < p.ny) {
                // rxy[k] holds plane q - RA - RB + k, rz[k] plane q - 2 RA + k; output z = q - RA
                float v = 0.f;
#pragma unroll
                for (int r = -RB; r <= RB; ++r) v += rxy[j][RB - r];
                float vz = arm.t[RA] * rz[j][RA];
#pragma unroll
                for (int r = 1; r <= RA; ++r) vz += arm.t[RA + r] * (rz[j][RA - r] + rz[j][RA + r]);
                v += vz;
                const bool solid = p.walls && (y == 0 || y == p.ny - 1);
                v = solid ? 0.f : scale * v;
                float* op = o + ((size_t)zo * p.ny + y) * p.nx + x;
                *op = accumulate ? (*op + v) : v;
            }
        }
    }
}

// L_1 (no box): the 13-point cross l_x + l_y + l_z read straight from the
// double-buffered tile, one barrier per plane.
template <int RA>
__global__ void __launch_bounds__(256) cross3_kernel(Params p, const float* __restrict__ in, float* __restrict__ out,
                                                     T3<RA> arm, float scale, int accumulate, int ncomp, int seg) {
    constexpr int NT = 256, RPT = TY / (NT / TX);
    using LD = TileLoader<RA, NT>;
    constexpr int WP = LD::WP, HH = LD::HH;
    constexpr int KZ = 2 * RA + 1;
    __shared__ __align__(16) float tile[2][HH * WP];
    const int c = blockIdx.z % ncomp, zs = blockIdx.z / ncomp;
    const int nz = p.nz;
    const int z0 = zs * seg, z1 = min(nz, z0 + seg);
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int lx = threadIdx.x % TX, yr = threadIdx.x / TX;
    const int x = x0 + lx;
    const size_t N = (size_t)p.n;
    const float* a = in + c * N;
    float* o = out + c * N;
    float rxy[RPT][RA + 1], rz[RPT][KZ];
#pragma unroll
    for (int j = 0; j < RPT; ++j) {
#pragma unroll
        for (int k = 0; k < RA + 1; ++k) rxy[j][k] = 0.f;
#pragma unroll
        for (int k = 0; k < KZ; ++k) rz[j][k] = 0.f;
    }
    LD ld;
    ld.init(p, x0, y0);
    ld.load(p, a, pm(z0 - RA, nz));
    int b = 0;
    for (int q = z0 - RA; q < z1 + RA; ++q, b ^= 1) {
        ld.store(tile[b]);
        __syncthreads();
        if (q + 1 < z1 + RA) ld.load(p, a, pm(q + 1, nz));
        const float* tl = tile[b];
        const int zo = q - RA;
#pragma unroll
        for (int j = 0; j < RPT; ++j) {
            const int ry = yr * RPT + j + RA;
            const float* row = tl + ry * WP + lx + RA;
            const float ctr = row[0];
            float axy = 2.f * arm.t[RA] * ctr;
#pragma unroll
            for (int r = 1; r <= RA; ++r)
                axy += arm.t[RA + r] * ((row[-r] + row[r]) + (row[-r * WP] + row[r * WP]));
#pragma unroll
            for (int k = 0; k < RA; ++k) rxy[j][k] = rxy[j][k + 1];
            rxy[j][RA] = axy;
#pragma unroll
            for (int k = 0; k < KZ - 1; ++k) rz[j][k] = rz[j][k + 1];
            rz[j][KZ - 1] = ctr;
            const int y = y0 + yr * RPT + j;
            if (zo >= z0 && x < p.nx && y < p.ny) {
                // rxy[k] holds plane q - RA + k, so the current output plane is rxy[0]
                float v = rxy[j][0] + arm.t[RA] * rz[j][RA];
#pragma unroll
                for (int r = 1; r <= RA; ++r) v += arm.t[RA + r] * (rz[j][RA - r] + rz[j][RA + r]);
                const bool solid = p.walls && (y == 0 || y == p.ny - 1);
                v = solid ? 0.f : scale * v;
                float* op = o + ((size_t)zo * p.ny + y) * p.nx + x;
                *op = accumulate ? (*op + v) : v;
            }
        }
    }
}

int seg_len(const Params& p, int blocks_xy, int ncomp, int R, int per_sm) {
    // enough z segments for `per_sm` blocks per SM; each segment re-reads 2R planes
    const long long want = 148LL * per_sm;
    long long nseg = (want + (long long)blocks_xy * ncomp - 1) / ((long long)blocks_xy * ncomp);
    if (nseg < 1) nseg = 1;
    int seg = (int)((p.nz + nseg - 1) / nseg);
    if (seg < 4 * R) seg = 4 * R;
    if (seg > p.nz) seg = p.nz;
    return seg;
}

template <int R>
cudaError_t run_gauss(const Params& p, const float* in, float* out, int ncomp, const Taps& t, float scale, int acc,
                      int per_sm, cudaStream_t s) {
    T3<R> tp;
    for (int i = 0; i < 2 * R + 1; ++i) tp.t[i] = t.t[i];
    const int bx = (p.nx + TX - 1) / TX, by = (p.ny + TY - 1) / TY;
    const int seg = seg_len(p, bx * by, ncomp, R, per_sm > 0 ? per_sm : 8);
    const int nseg = (p.nz + seg - 1) / seg;
    gauss3_kernel<R><<<dim3(bx, by, ncomp * nseg), 128, 0, s>>>(p, in, out, tp, scale, acc, ncomp, seg);
    return cudaGetLastError();
}

template <int RA, int RB>
cudaError_t run_lap(const Params& p, const float* in, float* out, int ncomp, const Taps& arm, float scale, int acc,
                    int per_sm, cudaStream_t s) {
    T3<RA> tp;
    for (int i = 0; i < 2 * RA + 1; ++i) tp.t[i] = arm.t[i];
    const int bx = (p.nx + TX - 1) / TX, by = (p.ny + TY - 1) / TY;
    const int seg = seg_len(p, bx * by, ncomp, RA, per_sm > 0 ? per_sm : 4);
    const int nseg = (p.nz + seg - 1) / seg;
    if (RB == 0)
        cross3_kernel<RA><<<dim3(bx, by, ncomp * nseg), 256, 0, s>>>(p, in, out, tp, scale, acc, ncomp, seg);
    else
        lap3_kernel<RA, RB><<<dim3(bx, by, ncomp * nseg), 256, 0, s>>>(p, in, out, tp, scale, acc, ncomp, seg);
    return cudaGetLastError();
}
}  // namespace

// G_s / B3 in 3-D with the same 1-D taps on every axis.
cudaError_t launch_gauss3(const Params& p, const float* in, float* out, int ncomp, const Taps& t, float scale,
                          int accumulate, int per_sm, cudaStream_t s) {
    switch (t.radius) {
        case 1: return run_gauss<1>(p, in, out, ncomp, t, scale, accumulate, per_sm, s);
        case 2: return run_gauss<2>(p, in, out, ncomp, t, scale, accumulate, per_sm, s);
        case 4: return run_gauss<4>(p, in, out, ncomp, t, scale, accumulate, per_sm, s);
        case 6: return run_gauss<6>(p, in, out, ncomp, t, scale, accumulate, per_sm, s);
        default: return cudaErrorNotSupported;
    }
}

// L_s in 3-D for s = 1 (arm radius 2, no box) and s = 3 (arm 7, box 1).
cudaError_t launch_lap3(const Params& p, const float* in, float* out, int ncomp, int s_scale, const Taps& arm,
                        float scale, int accumulate, int per_sm, cudaStream_t s) {
    if (s_scale == 1 && arm.radius == 2) return run_lap<2, 0>(p, in, out, ncomp, arm, scale, accumulate, per_sm, s);
    if (s_scale == 3 && arm.radius == 7) return run_lap<7, 1>(p, in, out, ncomp, arm, scale, accumulate, per_sm, s);
    return cudaErrorNotSupported;
}

}  // namespace lbm
