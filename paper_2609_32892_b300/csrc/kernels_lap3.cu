// One 3-D L_3 application (Sec. 4.1, Eq. laplace) in a single pass over the
// field, nx % 4 == 0.  L_s is L_1 dilated by the Kronecker product with the
// s^3 block of ones, so L_3 = c C_3 * B_3: B_3 the 3 x 3 x 3 box and C_3 the
// 13-point cross of l = (1, -4, 6, -4, 1) at stride 3 along every axis
// (centre 3 x 6 = 18).  The output is zero on solid rows (P K P); the input is
// zero beyond the array (its solid rows are zero too, so the box there is).
//
// A block owns a TX x TY tile of (x, y) and marches along a segment of z:
//
//   raw ring   input planes with a 7-node halo in y and 8 in x (periodic in
//              x; zero beyond a wall, periodic in y without walls), staged by
//              16-byte asynchronous copies NS planes ahead
//   box        per plane, the in-plane 3 x 3 box P_k over the tile plus a
//              6-node halo (column sums from shared memory, the x neighbours
//              by warp shuffles); B = P_{k-1} + P_k + P_{k+1} summed in
//              registers and written to one shared plane buffer
//   cross      the in-plane arms of B (x, y +- 3, +- 6) from that buffer; the
//              z arms are scattered into a ring of 13 pending output quads per
//              thread held in registers (the loop is unrolled by 13 so that
//              every ring index is a constant)
//
// DRAM sees each input node once (plus the z halo of a segment) and each
// output node once: 8 B per node and component.
#include "lbm_common.cuh"

namespace lbm {

namespace {

namespace l3f {
constexpr int TX = 48, TY = 16;          // output tile: 12 quads x 16 rows
constexpr int NT = (TX / 4) * TY;        // 192 threads, one output quad each
constexpr int RQ = 16;                   // quads per staged row: x0 - 8 .. x0 + 55
constexpr int RW = 4 * RQ;               // 64 floats
constexpr int RRH = TY + 14;             // 30 raw rows: y0 - 7 .. y0 + 22
constexpr int BRH = TY + 12;             // 28 box rows: y0 - 6 .. y0 + 21
constexpr int NRC = RRH * RQ;            // 480 raw chunks per plane
constexpr int NBQ = BRH * RQ;            // 448 box quads per plane
constexpr int NS = 4;                    // raw ring slots
constexpr int BS = 80;                   // box row stride (floats): rows 64 B apart in the banks
constexpr int RING = 13;                 // pending outputs z - 6 .. z + 6
constexpr int MR = (NRC + NT - 1) / NT;  // raw chunks per thread (3)
constexpr int MB = (NBQ + NT - 1) / NT;  // box quads per thread (3)
static_assert(NBQ % 32 == 0, "box quads fill whole warps (the shuffles)");
static_assert(NT % 32 == 0 && RQ == 16, "a warp covers two whole box rows");
}  // namespace l3f

__device__ __forceinline__ void cpa16(float* smem, const float* gmem, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"((unsigned)__cvta_generic_to_shared(smem)),
                 "l"(gmem), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cpa_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
__device__ __forceinline__ int wrap(int v, int n) {
    v %= n;
    return v < 0 ? v + n : v;
}
__device__ __forceinline__ float4 add4(float4 a, float4 b) {
    return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}
__device__ __forceinline__ float4 axpy4(float s, float4 a, float4 b) {
    return make_float4(fmaf(s, a.x, b.x), fmaf(s, a.y, b.y), fmaf(s, a.z, b.z), fmaf(s, a.w, b.w));
}

__global__ void __launch_bounds__(l3f::NT, 2) lap3_fused_kernel(Params p, const float* __restrict__ in,
                                                                 float* __restrict__ out, float scale, int ncomp,
                                                                 int seg) {
    using namespace l3f;
    __shared__ __align__(16) float raw[NS][RRH * RW];
    __shared__ __align__(16) float box[BRH * BS];
    const int t = threadIdx.x;
    const int c = blockIdx.z % ncomp, zs = blockIdx.z / ncomp;
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const int z0 = zs * seg, z1 = min(nz, z0 + seg);
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const size_t plane_n = (size_t)ny * nx;
    const float* a = in + (size_t)c * p.n;

    // this thread's raw chunks: in-plane offset, or -1 beyond a wall (zero fill)
    int roff[MR];
#pragma unroll
    for (int m = 0; m < MR; ++m) {
        const int i = t + NT * m;
        roff[m] = -1;
        if (i < NRC) {
            int gy = y0 - 7 + i / RQ;
            const int gx = wrap(x0 - 8 + 4 * (i % RQ), nx);
            bool ok = true;
            if (p.walls) ok = gy >= 0 && gy < ny;
            else gy = wrap(gy, ny);
            if (ok) roff[m] = gy * nx + gx;
        }
    }
    const int K = (z1 - z0) + 14;  // raw planes z0 - 7 .. z1 + 6
    auto issue = [&](int k) {
        const float* pl = a + (size_t)wrap(z0 - 7 + k, nz) * plane_n;
        float* dst = raw[k % NS];
#pragma unroll
        for (int m = 0; m < MR; ++m) {
            const int i = t + NT * m;
            if (i < NRC) cpa16(dst + 4 * i, roff[m] >= 0 ? pl + roff[m] : pl, roff[m] >= 0 ? 16 : 0);
        }
    };
#pragma unroll
    for (int k = 0; k < NS; ++k) {
        if (k < K) issue(k);
        cpa_commit();  // one group per plane slot, empty or not
    }

    // the output quad
    const int qx = t % (TX / 4), ry = t / (TX / 4);
    const int x = x0 + 4 * qx, y = y0 + ry;
    const bool live = x < nx && y < ny;
    const bool solid = p.walls && (y == 0 || y == ny - 1);
    float* oq = out + (size_t)c * p.n + (size_t)y * nx + x;
    const int bq = (ry + 6) * BS + 8 + 4 * qx;  // the output quad in the box plane

    float4 pm1[MB], pm2[MB];
    float4 acc[RING];
#pragma unroll
    for (int m = 0; m < MB; ++m) pm1[m] = pm2[m] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int r = 0; r < RING; ++r) acc[r] = make_float4(0.f, 0.f, 0.f, 0.f);

    for (int k0 = 0; k0 < K; k0 += RING) {
#pragma unroll
        for (int u = 0; u < RING; ++u) {
            const int k = k0 + u;
            if (k >= K) break;  // uniform over the block
            cpa_wait<NS - 1>();
            __syncthreads();  // plane k landed; every thread has left the box buffer
            // box: P_k at this thread's box quads, B_{k-1} = P_{k-2} + P_{k-1} + P_k
            const float* rw = raw[k % NS];
#pragma unroll
            for (int m = 0; m < MB; ++m) {
                const int i = t + NT * m;
                if (i < NBQ) {  // whole warps (NBQ % 32 == 0)
                    const int br = i / RQ, cq = i % RQ;
                    const float* r0 = rw + br * RW + 4 * cq;  // raw rows br .. br + 2 <-> box row br
                    const float4 u0 = *reinterpret_cast<const float4*>(r0);
                    const float4 u1 = *reinterpret_cast<const float4*>(r0 + RW);
                    const float4 u2 = *reinterpret_cast<const float4*>(r0 + 2 * RW);
                    const float4 cs = add4(add4(u0, u1), u2);
                    // neighbours x - 1 and x + 4 from the adjacent lanes (the same
                    // box row; at the row ends the value is one the cross never reads)
                    float lf = __shfl_up_sync(0xffffffffu, cs.w, 1);
                    float rt = __shfl_down_sync(0xffffffffu, cs.x, 1);
                    if (cq == 0) lf = 0.f;
                    if (cq == RQ - 1) rt = 0.f;
                    const float4 pk =
                        make_float4(lf + cs.x + cs.y, cs.x + cs.y + cs.z, cs.y + cs.z + cs.w, cs.z + cs.w + rt);
                    const float4 b = add4(add4(pm2[m], pm1[m]), pk);
                    pm2[m] = pm1[m];
                    pm1[m] = pk;
                    if (k >= 2) *reinterpret_cast<float4*>(box + br * BS + 4 * cq) = b;
                }
            }
            __syncthreads();  // the box plane is complete; raw slot k % NS is free
            if (k + NS < K) issue(k + NS);
            cpa_commit();
            if (k >= 2) {
                // box plane z_b = z0 - 8 + k: its in-plane arms at the output quad
                float v[20];  // box columns 4 qx .. 4 qx + 19 (from x0 - 8); the quad is v[8 .. 11]
#pragma unroll
                for (int m = 0; m < 5; ++m) {
                    const float4 w = *reinterpret_cast<const float4*>(box + bq - 8 + 4 * m);
                    v[4 * m] = w.x; v[4 * m + 1] = w.y; v[4 * m + 2] = w.z; v[4 * m + 3] = w.w;
                }
                const float4 ym6 = *reinterpret_cast<const float4*>(box + bq - 6 * BS);
                const float4 ym3 = *reinterpret_cast<const float4*>(box + bq - 3 * BS);
                const float4 yp3 = *reinterpret_cast<const float4*>(box + bq + 3 * BS);
                const float4 yp6 = *reinterpret_cast<const float4*>(box + bq + 6 * BS);
                const float4 bc = make_float4(v[8], v[9], v[10], v[11]);
                const float4 a3 =
                    add4(make_float4(v[5] + v[11], v[6] + v[12], v[7] + v[13], v[8] + v[14]), add4(ym3, yp3));
                const float4 a6 =
                    add4(make_float4(v[2] + v[14], v[3] + v[15], v[4] + v[16], v[5] + v[17]), add4(ym6, yp6));
                const float4 inpl = axpy4(18.f, bc, axpy4(-4.f, a3, a6));
                // output z_b + d sits in ring slot (k - 8 + d) mod 13; k0 is a
                // multiple of 13, so every slot below is a constant
                constexpr int o = 2 * RING - 8;
                const int sm6 = (u + o - 6) % RING, sm3 = (u + o - 3) % RING, sc = (u + o) % RING;
                const int sp3 = (u + o + 3) % RING, sp6 = (u + o + 6) % RING;
                const float4 done = add4(acc[sm6], bc);  // output z_b - 6 takes its z + 6 arm
                acc[sm3] = axpy4(-4.f, bc, acc[sm3]);
                acc[sc] = add4(acc[sc], inpl);
                acc[sp3] = axpy4(-4.f, bc, acc[sp3]);
                acc[sp6] = bc;  // output z_b + 6 starts with its z - 6 arm
                if (k >= 14 && live) {
                    const int zo = z0 + k - 14;
                    const float4 r = solid ? make_float4(0.f, 0.f, 0.f, 0.f)
                                           : make_float4(scale * done.x, scale * done.y, scale * done.z,
                                                         scale * done.w);
                    *reinterpret_cast<float4*>(oq + (size_t)zo * plane_n) = r;
                }
            }
        }
    }
    cpa_wait<0>();  // no copy is left in flight when the block exits
}

int seg_for(const Params& p, int blocks_xy, int ncomp, int per_sm) {
    // z segments for about `per_sm` blocks per SM; each segment re-reads 14
    // halo planes, so a segment is kept at least that long
    if (p.tune.one_seg) return p.nz;
    const long long want = 148LL * per_sm;
    long long nseg = (want + (long long)blocks_xy * ncomp - 1) / ((long long)blocks_xy * ncomp);
    if (nseg < 1) nseg = 1;
    int seg = (int)((p.nz + nseg - 1) / nseg);
    if (seg < 14) seg = 14;
    if (seg > p.nz) seg = p.nz;
    return seg;
}

}  // namespace

cudaError_t launch_lap3_fused(const Params& p, const float* in, float* out, int ncomp, float scale, int per_sm,
                              cudaStream_t s) {
    using namespace l3f;
    const int bx = (p.nx + TX - 1) / TX, by = (p.ny + TY - 1) / TY;
    const int seg = seg_for(p, bx * by, ncomp, per_sm > 0 ? per_sm : 4);
    const int nseg = (p.nz + seg - 1) / seg;
    lap3_fused_kernel<<<dim3(bx, by, ncomp * nseg), NT, 0, s>>>(p, in, out, scale, ncomp, seg);
    return cudaGetLastError();
}

}  // namespace lbm
