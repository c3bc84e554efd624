// The Gaussian (and binomial) filter applied twice, R R, on 3-D fields (Sec.
// 4.1, Eq. gaussian; the sensitivities R R v and R R omega of App. A).
//
// G_s is the product of one 1-D kernel t (2R + 1 taps) along each axis, and
// the filter acts on the fluid nodes: R = P (Kx Ky Kz) P with P the
// projection onto the fluid rows (zero extension beyond the walls).  Along the
// periodic axes x and z, R R therefore applies the composite kernel t * t
// (4R + 1 taps) once.  Along y with walls the middle projection matters near
// the walls: where every intermediate row y'' in [y - R, y + R] is fluid the
// composite kernel is exact, elsewhere the y factor runs as two stages with
// the projection between them.
//
// Three streaming passes, each reading and writing the field once:
//   gx_kernel  composite along x: a warp stages a 256-node row chunk plus
//              halo in shared memory, each lane produces 8 outputs from a
//              register window (16-byte shared loads);
//   gz_kernel  composite along z: each thread owns a column strip of M
//              outputs and holds its M + 4R inputs in registers (static
//              indices, no ring shifting); the strip index is the fastest
//              grid dimension, so the strips that share halo planes run
//              together and the halo re-reads hit L2;
//   gy_kernel  along y in the same strip form, composite or two-stage.
// Lanes of a warp own consecutive x, so every global access is coalesced.
//
// When rows (and planes) hold whole 16-byte groups (nx % 4 == 0), the passes
// stage their inputs with bulk asynchronous copies (cp.async.bulk, one per
// row or plane piece, completion on an mbarrier): a block's whole input is
// in flight at once and the per-element address arithmetic disappears; each
// thread then reads its column from shared memory with immediate offsets.
// Other shapes take the direct-load kernels.
#include "batch.cuh"
#include "lbm_common.cuh"
#include "tma.cuh"

namespace lbm {

namespace {

constexpr int kGxChunk = 256;  // outputs per warp in the x pass (8 per lane)
constexpr int kStripZ = 16;    // outputs per thread in the z and y passes

__host__ __device__ constexpr int rup4(int v) { return (v + 3) & ~3; }

// x pass: out(x) = sum_k c[k] in(x + k - RC), periodic in x.
template <int RC>
__device__ __forceinline__ void gx_kernel_body(const VB& vb, const Params& p, const float* __restrict__ in,
                                               float* __restrict__ out, const GaussTaps& gt, int chunks_per_row,
                                               long long nchunks) {
    constexpr int RCP = rup4(RC);
    constexpr int SW = kGxChunk + 2 * RCP;  // staged values per warp
    constexpr int NW = 8 + 2 * RC;          // window of one lane (even; a multiple of 4 when RC is)
    __shared__ __align__(16) float sm[4][SW];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long ch = (long long)vb.x * 4 + warp;
    if (ch >= nchunks) return;  // whole warp leaves together
    const int nx = p.nx;
    const long long row = ch / chunks_per_row;  // (comp, z, y) row
    const int x0 = (int)(ch - row * chunks_per_row) * kGxChunk;
    const float* src = in + row * nx;
    float* s = sm[warp];
    // stage x0 - RCP .. x0 + 256 + RCP - 1, periodic (one wrap suffices on
    // rows at least as long as the staged span, otherwise a modulo)
    const bool wide = nx >= SW;
    float st[(SW + 31) / 32];  // every load of the lane in flight before the stores
#pragma unroll
    for (int k = 0; k < (SW + 31) / 32; ++k) {
        const int i = lane + 32 * k;
        int xs = x0 - RCP + i;
        if (wide) {
            xs = xs < 0 ? xs + nx : (xs >= nx ? xs - nx : xs);
        } else {
            xs %= nx;
            if (xs < 0) xs += nx;
        }
        st[k] = i < SW ? __ldg(src + xs) : 0.f;
    }
#pragma unroll
    for (int k = 0; k < (SW + 31) / 32; ++k)
        if (lane + 32 * k < SW) s[lane + 32 * k] = st[k];
    __syncwarp();
    const int xl = x0 + lane * 8;
    if (xl >= nx) return;
    // window: s[lane*8 + RCP - RC + m], m = 0 .. NW - 1: 16-byte aligned when
    // RC % 4 == 0, else (RC = 2) 8-byte aligned; it ends inside the staged row.
    // Scatter form: each window value adds to the outputs it reaches, so
    // only the 8 accumulators stay live.
    const int base = lane * 8 + (RCP - RC);
    float o[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) o[j] = 0.f;
    constexpr int VW = RC % 4 == 0 ? 4 : 2;
#pragma unroll
    for (int m0 = 0; m0 < NW; m0 += VW) {
        float w[VW];
        if constexpr (VW == 4) {
            const float4 q = *reinterpret_cast<const float4*>(s + base + m0);
            w[0] = q.x; w[1] = q.y; w[2] = q.z; w[3] = q.w;
        } else {
            const float2 q = *reinterpret_cast<const float2*>(s + base + m0);
            w[0] = q.x; w[1] = q.y;
        }
#pragma unroll
        for (int e = 0; e < VW; ++e) {
            const int m = m0 + e;
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (m - j >= 0 && m - j <= 2 * RC) o[j] = fmaf(gt.c[m - j], w[e], o[j]);
        }
    }
    float* dst = out + row * nx + xl;
    if ((nx & 3) == 0 && xl + 8 <= nx) {
        reinterpret_cast<float4*>(dst)[0] = make_float4(o[0], o[1], o[2], o[3]);
        reinterpret_cast<float4*>(dst)[1] = make_float4(o[4], o[5], o[6], o[7]);
    } else {
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (xl + j < nx) dst[j] = o[j];
    }
}
template <int RC>
struct gx_kernel_op {
    static constexpr int NT = 128, MINB = 1;
    template <class... B>
    static __device__ __forceinline__ void run(const VB& vb, const B&... b) {
        gx_kernel_body<RC>(vb, b...);
    }
};
template <int RC>
__global__ void __launch_bounds__(128) gx_kernel(Params p, const float* __restrict__ in, float* __restrict__ out,
                                                 GaussTaps gt, int chunks_per_row, long long nchunks) {
    gx_kernel_body<RC>(vb_hw(), p, in, out, gt, chunks_per_row, nchunks);
}

// z pass: out(z) = sum_k c[k] in(z + k - RC), periodic in z; one thread per
// (x, y) node of the plane and strip of kStripZ outputs.
template <int RC>
__device__ __forceinline__ void gz_kernel_body(const VB& vb, const Params& p, const float* __restrict__ in,
                                               float* __restrict__ out, const GaussTaps& gt) {
    constexpr int M = kStripZ, NV = M + 2 * RC;
    const int nz = p.nz;
    const long long plane = (long long)p.nx * p.ny;
    const long long nxy = (long long)vb.y * blockDim.x + threadIdx.x;
    if (nxy >= plane) return;
    const int z0 = vb.x * M;
    const size_t N = (size_t)p.n;
    const float* a = in + (size_t)vb.z * N + nxy;
    float* o = out + (size_t)vb.z * N + nxy;
    float v[NV];
    if (z0 - RC >= 0 && z0 + M + RC <= nz) {
        // interior strip: consecutive planes, no wrap
        const float* q = a + (size_t)(z0 - RC) * plane;
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] = __ldg(q + (size_t)k * plane);
    } else {
        int zk = (z0 - RC) % nz;
        if (zk < 0) zk += nz;
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            v[k] = __ldg(a + (size_t)zk * plane);
            zk = zk + 1 == nz ? 0 : zk + 1;
        }
    }
    // scatter form: input k adds c[k - j] v[k] to each output j it reaches
    float r[M];
#pragma unroll
    for (int j = 0; j < M; ++j) r[j] = 0.f;
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
        for (int j = 0; j < M; ++j)
            if (k - j >= 0 && k - j <= 2 * RC) r[j] = fmaf(gt.c[k - j], v[k], r[j]);
#pragma unroll
    for (int j = 0; j < M; ++j)
        if (z0 + j < nz) o[(size_t)(z0 + j) * plane] = r[j];
}
template <int RC>
struct gz_kernel_op {
    static constexpr int NT = 128, MINB = 1;
    template <class... B>
    static __device__ __forceinline__ void run(const VB& vb, const B&... b) {
        gz_kernel_body<RC>(vb, b...);
    }
};
template <int RC>
__global__ void __launch_bounds__(128) gz_kernel(Params p, const float* __restrict__ in, float* __restrict__ out,
                                                 GaussTaps gt) {
    gz_kernel_body<RC>(vb_hw(), p, in, out, gt);
}

// y pass: one thread per (z, x) column and strip of kStripZ outputs.
// Periodic y: the composite kernel.  Walls: inputs outside the array are
// zero; a strip whose intermediate rows [y0 - R, y0 + M - 1 + R] are all
// fluid takes the composite kernel, the others two stages, u = P (t * in)
// on rows y0 - R .. y0 + M - 1 + R, then t * u; outputs on solid rows are zero.
template <int R>
__device__ __forceinline__ void gy_kernel_body(const VB& vb, const Params& p, const float* __restrict__ in,
                                               float* __restrict__ out, const GaussTaps& gt) {
    constexpr int M = kStripZ, RC = 2 * R, NV = M + 2 * RC, NU = M + 2 * R;
    const int nx = p.nx, ny = p.ny;
    const long long nzx = (long long)p.nz * nx;
    const long long t = (long long)vb.y * blockDim.x + threadIdx.x;
    if (t >= nzx) return;
    const int z = (int)(t / nx), x = (int)(t - (long long)z * nx);
    const int y0 = vb.x * M;
    const size_t N = (size_t)p.n;
    const size_t col = (size_t)z * ny * nx + x;
    const float* a = in + (size_t)vb.z * N + col;
    float* o = out + (size_t)vb.z * N + col;
    float v[NV];
    if (y0 - RC >= 0 && y0 + M + RC <= ny) {
        // interior strip: every row inside the array, no wrap
        const float* q = a + (size_t)(y0 - RC) * nx;
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] = __ldg(q + (size_t)k * nx);
    } else if (p.walls) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            const int y = y0 - RC + k;
            v[k] = (y >= 0 && y < ny) ? __ldg(a + (size_t)y * nx) : 0.f;
        }
    } else {
        int yk = (y0 - RC) % ny;
        if (yk < 0) yk += ny;
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            v[k] = __ldg(a + (size_t)yk * nx);
            yk = yk + 1 == ny ? 0 : yk + 1;
        }
    }
    float r[M];
#pragma unroll
    for (int j = 0; j < M; ++j) r[j] = 0.f;
    const bool composite = !p.walls || (y0 - R >= 1 && y0 + M - 1 + R <= ny - 2);
    if (composite) {
#pragma unroll
        for (int k = 0; k < NV; ++k)
#pragma unroll
            for (int j = 0; j < M; ++j)
                if (k - j >= 0 && k - j <= 2 * RC) r[j] = fmaf(gt.c[k - j], v[k], r[j]);
    } else {
        float u[NU];
#pragma unroll
        for (int i = 0; i < NU; ++i) u[i] = 0.f;
#pragma unroll
        for (int k = 0; k < NV; ++k)
#pragma unroll
            for (int i = 0; i < NU; ++i)
                if (k - i >= 0 && k - i <= 2 * R) u[i] = fmaf(gt.t[k - i], v[k], u[i]);
#pragma unroll
        for (int i = 0; i < NU; ++i) {
            const int y = y0 - R + i;
            if (!(y >= 1 && y <= ny - 2)) u[i] = 0.f;
        }
#pragma unroll
        for (int i = 0; i < NU; ++i)
#pragma unroll
            for (int j = 0; j < M; ++j)
                if (i - j >= 0 && i - j <= 2 * R) r[j] = fmaf(gt.t[i - j], u[i], r[j]);
    }
#pragma unroll
    for (int j = 0; j < M; ++j) {
        const int y = y0 + j;
        if (y < ny) o[(size_t)y * nx] = (p.walls && (y == 0 || y == ny - 1)) ? 0.f : r[j];
    }
}
template <int R>
struct gy_kernel_op {
    static constexpr int NT = 128, MINB = 1;
    template <class... B>
    static __device__ __forceinline__ void run(const VB& vb, const B&... b) {
        gy_kernel_body<R>(vb, b...);
    }
};
template <int R>
__global__ void __launch_bounds__(128) gy_kernel(Params p, const float* __restrict__ in, float* __restrict__ out,
                                                 GaussTaps gt) {
    gy_kernel_body<R>(vb_hw(), p, in, out, gt);
}

// ---- bulk-copy staged passes (nx % 4 == 0) ----

constexpr int kTileW = 128;  // columns of a z or y strip tile (one per thread)

// Packed FP32 pairs: one fma.rn.f32x2 does the same rounded FMA on two
// columns (bitwise the scalar fmaf of each), halving the FMA issue of the
// strip passes, whose column sums are otherwise bound by instruction issue.
__device__ __forceinline__ float2 ffma2(float c, float2 v, float2 acc) { return __ffma2_rn(make_float2(c, c), v, acc); }

// z pass: a block of 64 threads stages planes z0 - RC .. z0 + M + RC - 1 of a
// 128-column piece of the (x, y) plane, one bulk copy per plane, then each
// thread sums its two adjacent columns (8-byte shared loads and global
// stores, packed FMAs).
template <int RC>
__device__ __forceinline__ void gz_tma_kernel_body(const VB& vb, const Params& p, const float* __restrict__ in,
                                                   float* __restrict__ out, const GaussTaps& gt, DevState* st) {
    constexpr int M = kStripZ, NV = M + 2 * RC;
    __shared__ __align__(128) float tile[NV][kTileW];
    __shared__ __align__(8) uint64_t bar;
    const int nz = p.nz;
    const long long plane = (long long)p.nx * p.ny;
    const long long c0 = (long long)vb.y * kTileW;
    const int width = (int)min((long long)kTileW, plane - c0);
    const int z0 = vb.x * M;
    const size_t N = (size_t)p.n;
    const float* a = in + (size_t)vb.z * N + c0;
    // the barrier is set up by a block's first item; item i waits on phase i
    // (a persistent block of a batched launch runs many items)
    if (vb.it == 0 && threadIdx.x == 0) mbar_init(&bar, 1);
    const uint32_t ph = (uint32_t)vb.it & 1u;
    __syncthreads();
    if (threadIdx.x < 32) {
        // warp 0 issues the copies, one plane per lane (no serial chain)
        const uint32_t bytes = (uint32_t)width * 4u;
        if (threadIdx.x == 0) mbar_arrive_expect(&bar, bytes * NV);
        __syncwarp();
        for (int k = threadIdx.x; k < NV; k += 32) {
            int zk = z0 - RC + k;
            if (nz >= NV) {
                zk = zk < 0 ? zk + nz : (zk >= nz ? zk - nz : zk);
            } else {
                zk %= nz;
                if (zk < 0) zk += nz;
            }
            bulk_load(&tile[k][0], a + (size_t)zk * plane, bytes, &bar);
        }
        __syncwarp();  // every copy issued before any lane of the warp waits
    }
    if (!mbar_wait(&bar, ph)) {
        mbar_give_up(&bar, ph, st);
        return;
    }
    const int t2 = 2 * threadIdx.x;  // columns t2, t2 + 1 (width is a multiple of 4)
    if (t2 >= width) return;
    float2 r[M];
#pragma unroll
    for (int j = 0; j < M; ++j) r[j] = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        const float2 v = *reinterpret_cast<const float2*>(&tile[k][t2]);
#pragma unroll
        for (int j = 0; j < M; ++j)
            if (k - j >= 0 && k - j <= 2 * RC) r[j] = ffma2(gt.c[k - j], v, r[j]);
    }
    float* o = out + (size_t)vb.z * N + c0 + t2 + (size_t)z0 * plane;
    if (z0 + M <= nz) {
#pragma unroll
        for (int j = 0; j < M; ++j) *reinterpret_cast<float2*>(o + (size_t)j * plane) = r[j];
    } else {
#pragma unroll
        for (int j = 0; j < M; ++j)
            if (z0 + j < nz) *reinterpret_cast<float2*>(o + (size_t)j * plane) = r[j];
    }
}
template <int RC>
struct gz_tma_kernel_op {
    static constexpr int NT = 64, MINB = 1;
    template <class... B>
    static __device__ __forceinline__ void run(const VB& vb, const B&... b) {
        gz_tma_kernel_body<RC>(vb, b...);
    }
};
template <int RC>
__global__ void __launch_bounds__(64) gz_tma_kernel(Params p, const float* __restrict__ in, float* __restrict__ out,
                                                    GaussTaps gt, DevState* st) {
    gz_tma_kernel_body<RC>(vb_hw(), p, in, out, gt, st);
}

// y pass: a block of 64 threads stages rows y0 - 2R .. y0 + M + 2R - 1 of a
// 128-column piece of an x row at one z (rows outside the array: zero with
// walls, wrapped without), then each thread runs its two adjacent columns as
// gy_kernel does (composite, or two stages next to the walls).
template <int R>
__device__ __forceinline__ void gy_tma_kernel_body(const VB& vb, const Params& p, const float* __restrict__ in,
                                                   float* __restrict__ out, const GaussTaps& gt, DevState* st,
                                                   int cpr) {
    constexpr int M = kStripZ, RC = 2 * R, NV = M + 2 * RC, NU = M + 2 * R;
    __shared__ __align__(128) float tile[NV][kTileW];
    __shared__ __align__(8) uint64_t bar;
    const int nx = p.nx, ny = p.ny;
    const int z = vb.y / cpr, x0 = (vb.y - z * cpr) * kTileW;
    const int width = min(kTileW, nx - x0);
    const int y0 = vb.x * M;
    const size_t N = (size_t)p.n;
    const float* a = in + (size_t)vb.z * N + (size_t)z * ny * nx + x0;
    if (vb.it == 0 && threadIdx.x == 0) mbar_init(&bar, 1);  // phase i for the block's item i
    const uint32_t ph = (uint32_t)vb.it & 1u;
    // with walls, rows outside the array are zero (generic stores to rows no
    // copy touches); only the strips next to the walls have such rows
    const int klo = p.walls ? max(0, RC - y0) : 0;            // first row inside the array
    const int khi = p.walls ? min(NV, ny - y0 + RC) : NV;     // one past the last
    if (klo > 0 || khi < NV)
        for (int k = 0; k < NV; ++k)
            if (k < klo || k >= khi)
                for (int c = threadIdx.x; c < width; c += blockDim.x) tile[k][c] = 0.f;
    __syncthreads();
    if (threadIdx.x < 32) {
        // warp 0 issues the copies, one row per lane (no serial chain)
        const uint32_t bytes = (uint32_t)width * 4u;
        if (threadIdx.x == 0) mbar_arrive_expect(&bar, bytes * (uint32_t)(khi - klo));
        __syncwarp();
        for (int k = klo + threadIdx.x; k < khi; k += 32) {
            int y = y0 - RC + k;
            if (!p.walls) {
                if (ny >= NV) {
                    y = y < 0 ? y + ny : (y >= ny ? y - ny : y);
                } else {
                    y %= ny;
                    if (y < 0) y += ny;
                }
            }
            bulk_load(&tile[k][0], a + (size_t)y * nx, bytes, &bar);
        }
        __syncwarp();  // every copy issued before any lane of the warp waits
    }
    if (!mbar_wait(&bar, ph)) {
        mbar_give_up(&bar, ph, st);
        return;
    }
    const int t2 = 2 * threadIdx.x;  // columns t2, t2 + 1 (width is a multiple of 4)
    if (t2 >= width) return;
    float2 r[M];
#pragma unroll
    for (int j = 0; j < M; ++j) r[j] = make_float2(0.f, 0.f);
    const bool composite = !p.walls || (y0 - R >= 1 && y0 + M - 1 + R <= ny - 2);
    if (composite) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            const float2 v = *reinterpret_cast<const float2*>(&tile[k][t2]);
#pragma unroll
            for (int j = 0; j < M; ++j)
                if (k - j >= 0 && k - j <= 2 * RC) r[j] = ffma2(gt.c[k - j], v, r[j]);
        }
    } else {
        float2 u[NU];
#pragma unroll
        for (int i = 0; i < NU; ++i) u[i] = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            const float2 v = *reinterpret_cast<const float2*>(&tile[k][t2]);
#pragma unroll
            for (int i = 0; i < NU; ++i)
                if (k - i >= 0 && k - i <= 2 * R) u[i] = ffma2(gt.t[k - i], v, u[i]);
        }
#pragma unroll
        for (int i = 0; i < NU; ++i) {
            const int y = y0 - R + i;
            if (!(y >= 1 && y <= ny - 2)) u[i] = make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int i = 0; i < NU; ++i)
#pragma unroll
            for (int j = 0; j < M; ++j)
                if (i - j >= 0 && i - j <= 2 * R) r[j] = ffma2(gt.t[i - j], u[i], r[j]);
    }
    float* o = out + (size_t)vb.z * N + (size_t)z * ny * nx + x0 + t2 + (size_t)y0 * nx;
    if (y0 + M <= ny - 1 && y0 >= 1) {
#pragma unroll
        for (int j = 0; j < M; ++j) *reinterpret_cast<float2*>(o + (size_t)j * nx) = r[j];
    } else {
#pragma unroll
        for (int j = 0; j < M; ++j) {
            const int y = y0 + j;
            if (y < ny)
                *reinterpret_cast<float2*>(o + (size_t)j * nx) =
                    (p.walls && (y == 0 || y == ny - 1)) ? make_float2(0.f, 0.f) : r[j];
        }
    }
}
template <int R>
struct gy_tma_kernel_op {
    static constexpr int NT = 64, MINB = 1;
    template <class... B>
    static __device__ __forceinline__ void run(const VB& vb, const B&... b) {
        gy_tma_kernel_body<R>(vb, b...);
    }
};
template <int R>
__global__ void __launch_bounds__(64) gy_tma_kernel(Params p, const float* __restrict__ in, float* __restrict__ out,
                                                    GaussTaps gt, DevState* st, int cpr) {
    gy_tma_kernel_body<R>(vb_hw(), p, in, out, gt, st, cpr);
}

// x pass: warp w of the block stages the whole row blockIdx.x * 4 + w plus
// its periodic halo (three bulk copies: the row's last RCP values, the row,
// its first RCP values), so every input is read from DRAM once; lane l then
// produces outputs x = 8 (l + 32 k) .. + 7 as gx_kernel does.  Rows up to
// kGxRowMax long (dynamic shared memory, 4 rows per block).
constexpr int kGxRowMax = 2992;  // 4 rows of (2992 + 2 x 12) floats: 48 KiB

template <int RC>
__device__ __forceinline__ void gx_tma_kernel_body(const VB& vb, const Params& p, const float* __restrict__ in,
                                                   float* __restrict__ out, const GaussTaps& gt, DevState* st,
                                                   long long nrows) {
    constexpr int RCP = rup4(RC);
    constexpr int NW = 8 + 2 * RC;
    extern __shared__ __align__(128) float gx_sm[];
    __shared__ __align__(8) uint64_t bars[4];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long row = (long long)vb.x * 4 + warp;
    const int nx = p.nx;
    // row length rounded up to 8 so that the last lane group's window (up to
    // 8 outputs past a row end that is only 4-aligned) stays inside the row's
    // slot; a multiple of 4, so every warp's slot starts 16-byte aligned
    const int sw = ((nx + 7) & ~7) + 2 * RCP;
    float* s = gx_sm + warp * sw;
    uint64_t* bar = &bars[warp];
    const bool live = row < nrows;
    // the barriers are set up by a block's first item; item i waits on phase
    // i, and a warp without a row completes its phase by a plain arrival
    if (vb.it == 0) {
        if (threadIdx.x < 4) mbar_init(&bars[threadIdx.x], 1);
        __syncthreads();
    }
    const uint32_t ph = (uint32_t)vb.it & 1u;
    if (!live) {  // whole warp
        if (lane == 0) mbar_arrive(bar);
        return;
    }
    const float* src = in + row * nx;
    if (lane == 0) {
        mbar_arrive_expect(bar, (uint32_t)(nx + 2 * RCP) * 4u);
        bulk_load(s, src + nx - RCP, RCP * 4u, bar);
        bulk_load(s + RCP, src, (uint32_t)nx * 4u, bar);
        bulk_load(s + RCP + nx, src, RCP * 4u, bar);
    }
    __syncwarp();  // the copies issued before any lane waits
    if (!mbar_wait(bar, ph)) {
        atomicOr(&st->status, kStatusTimeout);
        mbar_wait(bar, ph);
        return;
    }
    constexpr int VW = RC % 4 == 0 ? 4 : 2;
    for (int xl = lane * 8; xl < nx; xl += 256) {
        // window s[xl + RCP - RC + m], m = 0 .. NW - 1 (16-byte aligned when RC % 4 == 0)
        const float* w0 = s + xl + (RCP - RC);
        float o[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) o[j] = 0.f;
#pragma unroll
        for (int m0 = 0; m0 < NW; m0 += VW) {
            float w[VW];
            if constexpr (VW == 4) {
                const float4 q = *reinterpret_cast<const float4*>(w0 + m0);
                w[0] = q.x; w[1] = q.y; w[2] = q.z; w[3] = q.w;
            } else {
                const float2 q = *reinterpret_cast<const float2*>(w0 + m0);
                w[0] = q.x; w[1] = q.y;
            }
#pragma unroll
            for (int e = 0; e < VW; ++e) {
                const int m = m0 + e;
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if (m - j >= 0 && m - j <= 2 * RC) o[j] = fmaf(gt.c[m - j], w[e], o[j]);
            }
        }
        float* dst = out + row * nx + xl;
        if (xl + 8 <= nx) {
            reinterpret_cast<float4*>(dst)[0] = make_float4(o[0], o[1], o[2], o[3]);
            reinterpret_cast<float4*>(dst)[1] = make_float4(o[4], o[5], o[6], o[7]);
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (xl + j < nx) dst[j] = o[j];
        }
    }
}
template <int RC>
struct gx_tma_kernel_op {
    static constexpr int NT = 128, MINB = 1;
    template <class... B>
    static __device__ __forceinline__ void run(const VB& vb, const B&... b) {
        gx_tma_kernel_body<RC>(vb, b...);
    }
};
template <int RC>
__global__ void __launch_bounds__(128) gx_tma_kernel(Params p, const float* __restrict__ in, float* __restrict__ out,
                                                     GaussTaps gt, DevState* st, long long nrows) {
    gx_tma_kernel_body<RC>(vb_hw(), p, in, out, gt, st, nrows);
}

}  // namespace

bool launch_gauss_rr_supported(int radius) { return radius == 1 || radius == 2 || radius == 4 || radius == 6; }

template <int R>
static void gauss_pass(const Params& p, int axis, const float* in, float* out, int ncomp, const GaussTaps& gt,
                       DevState* st, cudaStream_t s) {
    constexpr int RC = 2 * R;
    const bool bulk = p.nx % 4 == 0;  // rows and planes in whole 16-byte groups
    if (axis == 0) {
        const int cpr = (p.nx + kGxChunk - 1) / kGxChunk;
        const long long nrows = (long long)ncomp * p.nz * p.ny;
        if (bulk && p.nx >= rup4(RC) && p.nx <= kGxRowMax) {
            const size_t smem = (size_t)4 * (((p.nx + 7) & ~7) + 2 * rup4(RC)) * sizeof(float);
            go<gx_tma_kernel_op<RC>>(gx_tma_kernel<RC>, (unsigned)((nrows + 3) / 4), 128, smem, s, p, in, out, gt, st,
                                     nrows);
            return;
        }
        const long long nchunks = nrows * cpr;
        go<gx_kernel_op<RC>>(gx_kernel<RC>, (unsigned)((nchunks + 3) / 4), 128, 0, s, p, in, out, gt, cpr, nchunks);
    } else if (axis == 2) {
        const long long plane = (long long)p.nx * p.ny;
        if (bulk) {
            const dim3 g((p.nz + kStripZ - 1) / kStripZ, (unsigned)((plane + kTileW - 1) / kTileW), ncomp);
            go<gz_tma_kernel_op<RC>>(gz_tma_kernel<RC>, g, 64, 0, s, p, in, out, gt, st);
            return;
        }
        const dim3 g((p.nz + kStripZ - 1) / kStripZ, (unsigned)((plane + 127) / 128), ncomp);
        go<gz_kernel_op<RC>>(gz_kernel<RC>, g, 128, 0, s, p, in, out, gt);
    } else {
        if (bulk) {
            const int cpr = (p.nx + kTileW - 1) / kTileW;
            const dim3 g((p.ny + kStripZ - 1) / kStripZ, (unsigned)(p.nz * cpr), ncomp);
            go<gy_tma_kernel_op<R>>(gy_tma_kernel<R>, g, 64, 0, s, p, in, out, gt, st, cpr);
            return;
        }
        const long long nzx = (long long)p.nz * p.nx;
        const dim3 g((p.ny + kStripZ - 1) / kStripZ, (unsigned)((nzx + 127) / 128), ncomp);
        go<gy_kernel_op<R>>(gy_kernel<R>, g, 128, 0, s, p, in, out, gt);
    }
}

cudaError_t launch_gauss_pass(const Params& p, int axis, const float* in, float* out, int ncomp, const GaussTaps& gt,
                              DevState* st, cudaStream_t s) {
    switch (gt.radius) {
        case 1: gauss_pass<1>(p, axis, in, out, ncomp, gt, st, s); break;
        case 2: gauss_pass<2>(p, axis, in, out, ncomp, gt, st, s); break;
        case 4: gauss_pass<4>(p, axis, in, out, ncomp, gt, st, s); break;
        case 6: gauss_pass<6>(p, axis, in, out, ncomp, gt, st, s); break;
        default: return cudaErrorNotSupported;
    }
    return cudaGetLastError();
}

}  // namespace lbm
