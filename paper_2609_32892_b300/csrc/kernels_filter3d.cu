// Fused 3-D Laplacian filters L_s (Sec. 4.1, Eq. laplace): one kernel (or,
// for L_3, two streams) per filter application.  The Gaussian and binomial
// filters are applied twice at once by the streaming passes of kernels_gauss.cu.
//
// A block owns a TX x TY tile of (x, y) and marches along a segment of z.
// For every input plane it stages the tile plus halo in shared memory
// (coalesced loads, prefetched into registers one plane ahead), applies the
// in-plane terms, and pushes the result into per-thread register rings along
// z, from which the z terms produce one output plane per step.  Each input
// element is read from DRAM about once per application (halo re-reads hit L2)
// and each output written once.
//
//   lap3_kernel<RA, RB>   L_s = c sum_a [l dilated along a] x [box_s on the
//                         other two axes], arm radius RA = (5s-1)/2, box
//                         radius RB = (s-1)/2 (RB = 0: the box is the identity;
//                         cross3_kernel<RA>); used when nx % 4 != 0
//
// With nx % 4 == 0 the Laplacian class has its own kernels, one thread per
// output quad with 16-byte accesses: crossq3_kernel (L_1, planes staged by
// asynchronous copies and kept in a ring) and, for L_3, the fused box and
// stride-3 cross of kernels_lap3.cu.
//
// Periodic along x and z; along y with walls the halo outside the array reads
// zero (solid rows already hold zero), and outputs on solid rows are zero, so
// the kernel applies P K P exactly.  One component per blockIdx.z slice.
#include "batch.cuh"
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

// L_s with a box (s > 1): double-buffered shared arrays, two barriers per
// plane.  Phase A (after the tile of plane q is stored): box along y on the
// output rows and box along x on every tile row.  Phase B: the three terms of
// this thread's points, pushed into the z rings.  A buffer written in phase A
// of plane q was last read in phase B of plane q-2, which every thread left
// before the first barrier of plane q-1.
template <int RA, int RB>
__device__ __forceinline__ void lap3_kernel_body(const VB& vb, const Params& p, const float* __restrict__ in,
                                                 float* __restrict__ out, T3<RA> arm, float scale, int accumulate,
                                                 int ncomp, int seg) {
    constexpr int NT = 256, RPT = TY / (NT / TX);  // 2 output rows per thread
    using LD = TileLoader<RA, NT>;
    constexpr int WP = LD::WP, HH = LD::HH, W = LD::W;
    constexpr int KXY = RA + RB + 1;  // ring of l_x B_y + l_y B_x (box along z later)
    constexpr int KZ = 2 * RA + 1;    // ring of B_x B_y (arm along z later)
    __shared__ __align__(16) float tile[2][HH * WP];
    __shared__ __align__(16) float by[2][TY * WP];  // box along y on the output rows, every tile column
    __shared__ __align__(16) float bx[2][HH * TX];  // box along x on every tile row, output columns
    const int c = vb.z % ncomp, zs = vb.z / ncomp;
    const int nz = p.nz;
    const int z0 = zs * seg, z1 = min(nz, z0 + seg);
    const int x0 = vb.x * TX, y0 = vb.y * TY;
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
    int zq = pm(z0 - RA, nz);  // z index of the plane loaded last (advanced by one per plane)
    ld.load(p, a, zq);
    int b = 0;
    for (int q = z0 - RA; q < z1 + RA; ++q, b ^= 1) {
        ld.store(tile[b]);
        __syncthreads();
        zq = zq + 1 == nz ? 0 : zq + 1;
        if (q + 1 < z1 + RA) ld.load(p, a, zq);
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
template <int RA, int RB>
struct lap3_kernel_op {
    static constexpr int NT = 256, MINB = 1;
    template <class... B>
    static __device__ __forceinline__ void run(const VB& vb, const B&... b) {
        lap3_kernel_body<RA, RB>(vb, b...);
    }
};
template <int RA, int RB>
__global__ void __launch_bounds__(256) lap3_kernel(Params p, const float* __restrict__ in, float* __restrict__ out,
                                                   T3<RA> arm, float scale, int accumulate, int ncomp, int seg) {
    lap3_kernel_body<RA, RB>(vb_hw(), p, in, out, arm, scale, accumulate, ncomp, seg);
}

// L_1 (no box): the 13-point cross l_x + l_y + l_z read straight from the
// double-buffered tile, one barrier per plane.
template <int RA>
__device__ __forceinline__ void cross3_kernel_body(const VB& vb, const Params& p, const float* __restrict__ in,
                                                   float* __restrict__ out, T3<RA> arm, float scale, int accumulate,
                                                   int ncomp, int seg) {
    constexpr int NT = 256, RPT = TY / (NT / TX);
    using LD = TileLoader<RA, NT>;
    constexpr int WP = LD::WP, HH = LD::HH;
    constexpr int KZ = 2 * RA + 1;
    __shared__ __align__(16) float tile[2][HH * WP];
    const int c = vb.z % ncomp, zs = vb.z / ncomp;
    const int nz = p.nz;
    const int z0 = zs * seg, z1 = min(nz, z0 + seg);
    const int x0 = vb.x * TX, y0 = vb.y * TY;
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
    int zq = pm(z0 - RA, nz);  // z index of the plane loaded last (advanced by one per plane)
    ld.load(p, a, zq);
    int b = 0;
    for (int q = z0 - RA; q < z1 + RA; ++q, b ^= 1) {
        ld.store(tile[b]);
        __syncthreads();
        zq = zq + 1 == nz ? 0 : zq + 1;
        if (q + 1 < z1 + RA) ld.load(p, a, zq);
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
template <int RA>
struct cross3_kernel_op {
    static constexpr int NT = 256, MINB = 1;
    template <class... B>
    static __device__ __forceinline__ void run(const VB& vb, const B&... b) {
        cross3_kernel_body<RA>(vb, b...);
    }
};
template <int RA>
__global__ void __launch_bounds__(256) cross3_kernel(Params p, const float* __restrict__ in, float* __restrict__ out,
                                                     T3<RA> arm, float scale, int accumulate, int ncomp, int seg) {
    cross3_kernel_body<RA>(vb_hw(), p, in, out, arm, scale, accumulate, ncomp, seg);
}

// asynchronous 16-byte global -> shared copies (zero-fill when src_bytes = 0)
__device__ __forceinline__ void cp_async16(float* smem, const float* gmem, int src_bytes) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

int seg_len(const Params& p, int blocks_xy, int ncomp, int R, int per_sm) {
    // enough z segments for `per_sm` blocks per SM; each segment re-reads 2R
    // planes.  Short segments (down to R planes) serve small grids, where the
    // sequential march of one block, not the halo work, sets the time.
    if (p.tune.one_seg) return p.nz;  // throughput goal: no halo planes re-read
    const long long want = 148LL * per_sm;
    long long nseg = (want + (long long)blocks_xy * ncomp - 1) / ((long long)blocks_xy * ncomp);
    if (nseg < 1) nseg = 1;
    int seg = (int)((p.nz + nseg - 1) / nseg);
    if (seg < R) seg = R;
    if (seg > p.nz) seg = p.nz;
    return seg;
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
        go<cross3_kernel_op<RA>>(cross3_kernel<RA>, dim3(bx, by, ncomp * nseg), 256, 0, s, p, in, out, tp, scale, acc,
                                 ncomp, seg);
    else
        go<lap3_kernel_op<RA, RB>>(lap3_kernel<RA, RB>, dim3(bx, by, ncomp * nseg), 256, 0, s, p, in, out, tp, scale,
                                   acc, ncomp, seg);
    return cudaGetLastError();
}
// L_1 (the 13-point cross, arm radius 2) with planes staged by asynchronous
// 16-byte copies (nx % 4 == 0).  A thread produces the 4 consecutive x outputs
// of one row from 16-byte shared loads: its row's quads at x - 4 .. x + 7 for
// the x arm, the output quad of rows y +- 1, y +- 2 for the y arm and of
// planes z +- 1, z +- 2 for the z arm.  The five planes an output plane reads
// stay staged in a ring of eight plane buffers (five read, two in flight, one
// being refilled), so nothing is carried in registers from plane to plane.
// One barrier per plane: after it every thread has left the previous output
// plane, the last reader of plane z - 3, whose buffer takes plane z + 5.
namespace cq3 {
constexpr int TX = 32, TY = 16, RA = 2, HX = 4, HY = 2;
constexpr int WP = TX + 2 * HX;    // 40 floats per staged row
constexpr int NQ = WP / 4;         // 10 chunks per row
constexpr int TH = TY + 2 * HY;    // 20 staged rows
constexpr int NT = (TX / 4) * TY;  // 128: one thread per output quad
constexpr int SZ = TH * WP;        // 800 floats per plane
constexpr int NB = 8;              // plane buffers (a power of two)
}  // namespace cq3

__device__ __forceinline__ void cp_async_wait2() { asm volatile("cp.async.wait_group 2;\n" ::: "memory"); }

__device__ __forceinline__ void crossq3_kernel_body(const VB& vb, const Params& p, const float* __restrict__ in,
                                                    float* __restrict__ out, T3<2> arm, float scale, int accumulate,
                                                    int ncomp, int seg) {
    constexpr int TX = cq3::TX, TY = cq3::TY, RA = cq3::RA, HX = cq3::HX, HY = cq3::HY;
    constexpr int NQ = cq3::NQ, TH = cq3::TH, NT = cq3::NT, SZ = cq3::SZ, NB = cq3::NB;
    __shared__ __align__(16) float tile[NB][SZ];
    __shared__ int coff[TH * NQ];
    const int c = vb.z % ncomp, zs = vb.z / ncomp;
    const int nz = p.nz;
    const int z0 = zs * seg, z1 = min(nz, z0 + seg);
    const int x0 = vb.x * TX, y0 = vb.y * TY;
    const int qx = threadIdx.x & 7, ry = threadIdx.x >> 3;
    const int gx0 = x0 + 4 * qx, y = y0 + ry;
    const size_t N = (size_t)p.n;
    const float* a = in + c * N;
    float* o = out + c * N;
    // chunk k: staged row k / NQ <-> y0 - HY + row, columns 4 (k % NQ) .. + 3
    // <-> x0 - HX + 4 (k % NQ) .. (periodic in x; a chunk never straddles the
    // period).  Offsets (-1: beyond a wall, zero-filled) are the same for
    // every plane.
    for (int k = threadIdx.x; k < TH * NQ; k += NT) {
        const int ly = k / NQ, m = k - ly * NQ;
        int gy = y0 - HY + ly;
        const int gx = pm(x0 - HX + 4 * m, p.nx);
        bool ok = true;
        if (p.walls) ok = gy >= 0 && gy < p.ny;
        else gy = pm(gy, p.ny);
        coff[k] = ok ? gy * p.nx + gx : -1;
    }
    __syncthreads();
    // plane q (z0 - RA <= q <= z1 + RA - 1) goes to buffer q mod NB; every
    // call commits one group, empty past the last plane needed
    int zq = pm(z0 - RA, nz);  // z index of the next plane staged (calls come in plane order)
    auto issue = [&](int q) {
        if (q < z1 + RA) {
            float* t = tile[q & (NB - 1)];
            const float* plane = a + (size_t)zq * p.ny * p.nx;
            zq = zq + 1 == nz ? 0 : zq + 1;
            for (int k = threadIdx.x; k < TH * NQ; k += NT) {
                const int ofs = coff[k];
                cp_async16(t + 4 * k, ofs >= 0 ? plane + ofs : plane, ofs >= 0 ? 16 : 0);
            }
        }
        cp_async_commit();
    };
    for (int q = z0 - RA; q <= z0 + RA + 2; ++q) issue(q);  // planes z0 - 2 .. z0 + 4
    const bool live = gx0 < p.nx && y < p.ny;
    const bool solid = p.walls && (y == 0 || y == p.ny - 1);
    const int rq = (ry + HY) * NQ + qx + 1;  // the output quad in a staged plane
    // this thread's column: the quad of planes zo - 2 .. zo + 2 in a register
    // ring (plane q in slot (q - z0) mod 5; the plane loop is unrolled by 5,
    // so every slot index is a constant); each plane adds one 16-byte load
    float4 ring[5];
    for (int zb = z0; zb < z1; zb += 5) {
#pragma unroll
        for (int u = 0; u < 5; ++u) {
            const int zo = zb + u;
            if (zo >= z1) break;  // uniform over the block
            cp_async_wait2();  // planes up to zo + 2 have landed (zo + 3, zo + 4 may be in flight)
            __syncthreads();
            issue(zo + RA + 3);
            const float* t0 = tile[zo & (NB - 1)];
            if (zb == z0 && u == 0) {
                ring[3] = reinterpret_cast<const float4*>(tile[(zo - 2) & (NB - 1)])[rq];
                ring[4] = reinterpret_cast<const float4*>(tile[(zo - 1) & (NB - 1)])[rq];
                ring[0] = reinterpret_cast<const float4*>(t0)[rq];
                ring[1] = reinterpret_cast<const float4*>(tile[(zo + 1) & (NB - 1)])[rq];
            }
            ring[(u + 2) % 5] = reinterpret_cast<const float4*>(tile[(zo + 2) & (NB - 1)])[rq];
            const float4 xc = ring[u % 5];
            const float2 xl = reinterpret_cast<const float2*>(t0)[2 * rq - 1];  // x - 2, x - 1
            const float2 xr = reinterpret_cast<const float2*>(t0)[2 * rq + 2];  // x + 4, x + 5
            const float v[8] = {xl.x, xl.y, xc.x, xc.y, xc.z, xc.w, xr.x, xr.y};  // x - 2 .. x + 5
            const float4* t4 = reinterpret_cast<const float4*>(t0);
            const float4 a1 = t4[rq - NQ], b1 = t4[rq + NQ], a2 = t4[rq - 2 * NQ], b2 = t4[rq + 2 * NQ];
            const float ym1[4] = {a1.x, a1.y, a1.z, a1.w}, yp1[4] = {b1.x, b1.y, b1.z, b1.w};
            const float ym2[4] = {a2.x, a2.y, a2.z, a2.w}, yp2[4] = {b2.x, b2.y, b2.z, b2.w};
            const float4 c1 = ring[(u + 4) % 5], d1 = ring[(u + 1) % 5], c2 = ring[(u + 3) % 5],
                         d2 = ring[(u + 2) % 5];
            const float zm1[4] = {c1.x, c1.y, c1.z, c1.w}, zp1[4] = {d1.x, d1.y, d1.z, d1.w};
            const float zm2[4] = {c2.x, c2.y, c2.z, c2.w}, zp2[4] = {d2.x, d2.y, d2.z, d2.w};
            float res[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float ctr = v[2 + j];
                float axy = 2.f * arm.t[RA] * ctr;
                axy += arm.t[RA + 1] * ((v[1 + j] + v[3 + j]) + (ym1[j] + yp1[j]));
                axy += arm.t[RA + 2] * ((v[0 + j] + v[4 + j]) + (ym2[j] + yp2[j]));
                float w = axy + arm.t[RA] * ctr;
                w += arm.t[RA + 1] * (zm1[j] + zp1[j]);
                w += arm.t[RA + 2] * (zm2[j] + zp2[j]);
                res[j] = solid ? 0.f : scale * w;
            }
            if (live) {
                float4* op = reinterpret_cast<float4*>(o + ((size_t)zo * p.ny + y) * p.nx + gx0);
                float4 w = make_float4(res[0], res[1], res[2], res[3]);
                if (accumulate) {
                    const float4 old = *op;
                    w.x += old.x; w.y += old.y; w.z += old.z; w.w += old.w;
                }
                *op = w;
            }
        }
    }
    cp_async_wait0();
}
struct crossq3_kernel_op {
    static constexpr int NT = 128, MINB = 1;
    template <class... B>
    static __device__ __forceinline__ void run(const VB& vb, const B&... b) {
        crossq3_kernel_body(vb, b...);
    }
};
__global__ void __launch_bounds__(128) crossq3_kernel(Params p, const float* __restrict__ in, float* __restrict__ out,
                                                      T3<2> arm, float scale, int accumulate, int ncomp, int seg) {
    crossq3_kernel_body(vb_hw(), p, in, out, arm, scale, accumulate, ncomp, seg);
}

// L_1 with asynchronously staged planes; needs nx % 4 == 0
cudaError_t run_crossq3(const Params& p, const float* in, float* out, int ncomp, const Taps& arm, float scale, int acc,
                        int per_sm, cudaStream_t s) {
    T3<2> tp;
    for (int i = 0; i < 5; ++i) tp.t[i] = arm.t[i];
    const int bx = (p.nx + cq3::TX - 1) / cq3::TX, by = (p.ny + cq3::TY - 1) / cq3::TY;
    const int seg = seg_len(p, bx * by, ncomp, 2, per_sm > 0 ? per_sm : 8);
    const int nseg = (p.nz + seg - 1) / seg;
    go<crossq3_kernel_op>(crossq3_kernel, dim3(bx, by, ncomp * nseg), cq3::NT, 0, s, p, in, out, tp, scale, acc, ncomp,
                          seg);
    return cudaGetLastError();
}

}  // namespace

// L_3 when nx % 4 == 0 runs as one fused kernel (kernels_lap3.cu) in the
// factorised form L_s = c C_s * B_s: L_s is L_1 dilated by the Kronecker
// product with the s^3 block of ones, so B_s is the s x s x s box and C_s the
// cross of l = [1, -4, 6, -4, 1] at stride s along every axis (centre 3 x 6);
// for s = 3 a 27-point box and a 13-point cross instead of the 3 x 21 taps of
// the separable-sum form (lap3_kernel<7, 1>).
bool lap3_split(const Params& p, int s_scale) { return s_scale == 3 && p.nx % 4 == 0; }

// L_s in 3-D for s = 1 (arm radius 2, no box) and s = 3 (arm 7, box 1).
cudaError_t launch_lap3(const Params& p, const float* in, float* out, int ncomp, int s_scale, const Taps& arm,
                        float scale, int accumulate, int per_sm, cudaStream_t s) {
    if (s_scale == 1 && arm.radius == 2) {
        if (p.nx % 4 == 0) return run_crossq3(p, in, out, ncomp, arm, scale, accumulate, per_sm, s);
        return run_lap<2, 0>(p, in, out, ncomp, arm, scale, accumulate, per_sm, s);
    }
    // L_3 with nx % 4 == 0 goes through lap3_split (the fused kernel of kernels_lap3.cu)
    if (s_scale == 3 && arm.radius == 7) return run_lap<7, 1>(p, in, out, ncomp, arm, scale, accumulate, per_sm, s);
    return cudaErrorNotSupported;
}

}  // namespace lbm
