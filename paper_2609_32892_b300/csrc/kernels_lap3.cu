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
//              16-byte asynchronous copies NS - 1 planes ahead
//   box        per plane, the in-plane 3 x 3 box P_k over the tile plus a
//              6-node halo: a half-warp holds a row of 16 quads and slides
//              down 4 rows (column sums of 3 staged rows), the x neighbours
//              come by warp shuffles; B = P_{k-1} + P_k + P_{k+1} is summed
//              in registers and written to a box plane buffer (two buffers,
//              so that one barrier per plane separates the stages)
//   cross      the in-plane arms of B (x, y +- 3, +- 6) from the box plane of
//              the previous iteration; the z arms are scattered into a ring of
//              13 pending output quads per thread held in registers (the loop
//              is unrolled by 13 so that every ring index is a constant)
//
// DRAM sees each input node once (plus the z halo of a segment) and each
// output node once: 8 B per node and component.
#include <mutex>

#include "batch.cuh"
#include "lbm_common.cuh"

namespace lbm {

namespace {

// Tile TX = 48 x TY outputs (12 x TY quads, one per thread); staged rows of
// 16 quads (x0 - 8 .. x0 + 55); NS raw planes in the ring.
template <int TY, int NS>
struct L3Shape {
    static constexpr int TX = 48, NT = (TX / 4) * TY, RQ = 16, RW = 4 * RQ;
    static constexpr int RRH = TY + 14;  // raw rows y0 - 7 .. y0 + TY + 6
    static constexpr int BRH = TY + 12;  // box rows y0 - 6 .. y0 + TY + 5
    static constexpr int NRC = RRH * RQ;
    static constexpr int BS = 80;  // box row stride (floats): consecutive rows 64 B apart in the banks
    static constexpr int MR = (NRC + NT - 1) / NT;
    static constexpr int NHW = BRH / 4;  // half-warps of the box stage, 4 box rows each
    static constexpr int RAW = RRH * RW, BOX = BRH * BS;
    static constexpr size_t smem = (size_t)(NS * RAW + 2 * BOX) * sizeof(float);
    static_assert(BRH % 4 == 0 && NHW <= NT / 16 && NT % 32 == 0, "the box stage: whole half-warps");
    static_assert(NS >= 2, "at least one plane in flight");
};
constexpr int kRing = 13;  // pending outputs z - 6 .. z + 6

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

// a quad of x-consecutive values as two packed pairs (f32x2 arithmetic)
struct Quad {
    float2 lo, hi;
};
__device__ __forceinline__ Quad ldq(const float* s) {
    const float4 w = *reinterpret_cast<const float4*>(s);
    return {make_float2(w.x, w.y), make_float2(w.z, w.w)};
}
__device__ __forceinline__ void stq(float* s, Quad q) {
    *reinterpret_cast<float4*>(s) = make_float4(q.lo.x, q.lo.y, q.hi.x, q.hi.y);
}
__device__ __forceinline__ Quad qadd(Quad a, Quad b) { return {__fadd2_rn(a.lo, b.lo), __fadd2_rn(a.hi, b.hi)}; }
__device__ __forceinline__ Quad qfma(float s, Quad a, Quad b) {
    const float2 ss = make_float2(s, s);
    return {__ffma2_rn(ss, a.lo, b.lo), __ffma2_rn(ss, a.hi, b.hi)};
}
__device__ __forceinline__ Quad qzero() { return {make_float2(0.f, 0.f), make_float2(0.f, 0.f)}; }

template <int TY, int NS>
__device__ __forceinline__ void lap3_fused_kernel_body(const VB& vb, const Params& p, const float* __restrict__ in,
                                                       float* __restrict__ out, float scale, int ncomp, int seg) {
    using S = L3Shape<TY, NS>;
    constexpr int NT = S::NT, RQ = S::RQ, RW = S::RW, BS = S::BS;
    extern __shared__ __align__(16) float l3_smem[];
    float* raw = l3_smem;                // [NS][RAW]
    float* box = l3_smem + NS * S::RAW;  // [2][BOX]
    const int t = threadIdx.x;
    const int c = vb.z % ncomp, zs = vb.z / ncomp;
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const int z0 = zs * seg, z1 = min(nz, z0 + seg);
    const int x0 = vb.x * S::TX, y0 = vb.y * TY;
    const size_t plane_n = (size_t)ny * nx;
    const float* a = in + (size_t)c * p.n;

    // this thread's raw chunks: in-plane offset, or -1 beyond a wall (zero fill)
    int roff[S::MR];
#pragma unroll
    for (int m = 0; m < S::MR; ++m) {
        const int i = t + NT * m;
        roff[m] = -1;
        if (i < S::NRC) {
            int gy = y0 - 7 + i / RQ;
            const int gx = wrap(x0 - 8 + 4 * (i % RQ), nx);
            bool ok = true;
            if (p.walls) ok = gy >= 0 && gy < ny;
            else gy = wrap(gy, ny);
            if (ok) roff[m] = gy * nx + gx;
        }
    }
    const int K = (z1 - z0) + 14;  // raw planes z0 - 7 .. z1 + 6
    // planes are issued in order: a running plane index and ring slot
    int zq = wrap(z0 - 7, nz), slot_w = 0;
    auto issue = [&]() {
        const float* pl = a + (size_t)zq * plane_n;
        float* dst = raw + slot_w * S::RAW;
        zq = zq + 1 == nz ? 0 : zq + 1;
        slot_w = slot_w + 1 == NS ? 0 : slot_w + 1;
#pragma unroll
        for (int m = 0; m < S::MR; ++m) {
            const int i = t + NT * m;
            if (i < S::NRC) cpa16(dst + 4 * i, roff[m] >= 0 ? pl + roff[m] : pl, roff[m] >= 0 ? 16 : 0);
        }
    };
#pragma unroll
    for (int k = 0; k < NS - 1; ++k) {
        if (k < K) issue();
        cpa_commit();  // one group per plane, empty or not
    }

    // the output quad
    const int qx = t % (S::TX / 4), ry = t / (S::TX / 4);
    const int x = x0 + 4 * qx, y = y0 + ry;
    const bool live = x < nx && y < ny;
    const float sc_out = p.walls && (y == 0 || y == ny - 1) ? 0.f : scale;  // zero on solid rows
    float* op = out + (size_t)c * p.n + (size_t)y * nx + x + (size_t)z0 * plane_n;
    const int bq = (ry + 6) * BS + 8 + 4 * qx;  // the output quad in a box plane

    Quad pm1[4], pm2[4];  // P_{k-1}, P_{k-2} of this thread's box quads
    Quad acc[kRing];
#pragma unroll
    for (int j = 0; j < 4; ++j) pm1[j] = pm2[j] = qzero();
#pragma unroll
    for (int r = 0; r < kRing; ++r) acc[r] = qzero();

    int slot_r = 0;  // ring slot of raw plane k
    // iteration k: the box stage of raw plane k (B_{k-1} into box buffer k & 1)
    // and the cross stage of the box plane of iteration k - 1 (B_{k-2}, at
    // z_b = z0 - 9 + k), one barrier between consecutive iterations
    for (int k0 = 0; k0 <= K; k0 += kRing) {
#pragma unroll
        for (int u = 0; u < kRing; ++u) {
            const int k = k0 + u;
            if (k > K) break;  // uniform over the block
            cpa_wait<NS - 2>();
            // plane k landed; box buffer (k - 1) & 1 is complete; nobody reads
            // box buffer k & 1 or raw slot (k - 1) % NS any more
            __syncthreads();
            if (k + NS - 1 < K) issue();
            cpa_commit();
            if (k < K && t < 32 * ((S::NHW + 1) / 2)) {  // whole warps (the shuffles)
                // half-warp h: box rows 4 h .. 4 h + 3 of its quad column, from
                // raw rows 4 h .. 4 h + 5 (a sliding window in y); a half-warp
                // beyond the box rows only takes part in the shuffles
                const int h = t >> 4, cq = t & 15;
                const bool on = h < S::NHW;
                const float* r0 = raw + slot_r * S::RAW + 4 * h * RW + 4 * cq;
                float* bw = box + (k & 1) * S::BOX + 4 * h * BS + 4 * cq;
                Quad r[6];
#pragma unroll
                for (int j = 0; j < 6; ++j) r[j] = on ? ldq(r0 + j * RW) : qzero();
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const Quad cs = qadd(qadd(r[j], r[j + 1]), r[j + 2]);
                    // x - 1 and x + 4 from the adjacent lanes (the same box row;
                    // at the row ends a value the cross never reads)
                    float lf = __shfl_up_sync(0xffffffffu, cs.hi.y, 1);
                    float rt = __shfl_down_sync(0xffffffffu, cs.lo.x, 1);
                    if (cq == 0) lf = 0.f;
                    if (cq == RQ - 1) rt = 0.f;
                    const float s01 = cs.lo.x + cs.lo.y, s23 = cs.hi.x + cs.hi.y;
                    const Quad pk = {make_float2(lf + s01, s01 + cs.hi.x), make_float2(cs.lo.y + s23, s23 + rt)};
                    const Quad b = qadd(qadd(pm2[j], pm1[j]), pk);
                    pm2[j] = pm1[j];
                    pm1[j] = pk;
                    if (k >= 2 && on) stq(bw + j * BS, b);
                }
            }
            slot_r = slot_r + 1 == NS ? 0 : slot_r + 1;
            if (k >= 3) {
                const float* bb = box + ((k - 1) & 1) * S::BOX + bq;
                const float2 w0 = *reinterpret_cast<const float2*>(bb - 6);  // x - 6, x - 5
                const float4 w1 = *reinterpret_cast<const float4*>(bb - 4);
                const Quad bc = ldq(bb);
                const float4 w3 = *reinterpret_cast<const float4*>(bb + 4);
                const float2 w4 = *reinterpret_cast<const float2*>(bb + 8);  // x + 8, x + 9
                const Quad y3 = qadd(ldq(bb - 3 * BS), ldq(bb + 3 * BS));
                const Quad y6 = qadd(ldq(bb - 6 * BS), ldq(bb + 6 * BS));
                // x arms: x +- 3 and x +- 6 of the four nodes
                const Quad x3 = {make_float2(w1.y + bc.hi.y, w1.z + w3.x), make_float2(w1.w + w3.y, bc.lo.x + w3.z)};
                const Quad x6 = {make_float2(w0.x + w3.z, w0.y + w3.w), make_float2(w1.x + w4.x, w1.y + w4.y)};
                const Quad a3 = qadd(x3, y3), a6 = qadd(x6, y6);
                const Quad inpl = qfma(18.f, bc, qfma(-4.f, a3, a6));
                // output z_b + d sits in ring slot (k - 9 + d) mod 13; k0 is a
                // multiple of 13, so every slot below is a constant
                constexpr int o = 2 * kRing - 9;
                const int sm6 = (u + o - 6) % kRing, sm3 = (u + o - 3) % kRing, sc = (u + o) % kRing;
                const int sp3 = (u + o + 3) % kRing, sp6 = (u + o + 6) % kRing;
                const Quad done = qadd(acc[sm6], bc);  // output z_b - 6 takes its z + 6 arm
                acc[sm3] = qfma(-4.f, bc, acc[sm3]);
                acc[sc] = qadd(acc[sc], inpl);
                acc[sp3] = qfma(-4.f, bc, acc[sp3]);
                acc[sp6] = bc;  // output z_b + 6 starts with its z - 6 arm
                if (k >= 15) {
                    if (live) {
                        const float2 s2 = make_float2(sc_out, sc_out);
                        stq(op, {__fmul2_rn(s2, done.lo), __fmul2_rn(s2, done.hi)});
                    }
                    op += plane_n;
                }
            }
        }
    }
    cpa_wait<0>();  // no copy is left in flight when the block exits
}
template <int TY, int NS>
struct lap3_fused_kernel_op {
    static constexpr int NT = L3Shape<TY, NS>::NT, MINB = 2;
    template <class... B>
    static __device__ __forceinline__ void run(const VB& vb, const B&... b) {
        lap3_fused_kernel_body<TY, NS>(vb, b...);
    }
};
template <int TY, int NS>
__global__ void __launch_bounds__(L3Shape<TY, NS>::NT, 2) lap3_fused_kernel(Params p, const float* __restrict__ in,
                                                                          float* __restrict__ out, float scale,
                                                                          int ncomp, int seg) {
    lap3_fused_kernel_body<TY, NS>(vb_hw(), p, in, out, scale, ncomp, seg);
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

template <int TY, int NS>
cudaError_t run_lap3(const Params& p, const float* in, float* out, int ncomp, float scale, int per_sm,
                     cudaStream_t s) {
    using S = L3Shape<TY, NS>;
    // the opt-in above 48 KiB of dynamic shared memory (a host-side function
    // attribute, set before the first launch, outside any graph capture)
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [&] {
        attr = cudaFuncSetAttribute(lap3_fused_kernel<TY, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)S::smem);
    });
    if (attr != cudaSuccess) return attr;
    const int bx = (p.nx + S::TX - 1) / S::TX, by = (p.ny + TY - 1) / TY;
    const int seg = seg_for(p, bx * by, ncomp, per_sm > 0 ? per_sm : 2);
    const int nseg = (p.nz + seg - 1) / seg;
    return go<lap3_fused_kernel_op<TY, NS>>(lap3_fused_kernel<TY, NS>, dim3(bx, by, ncomp * nseg), S::NT, S::smem, s,
                                            p, in, out, scale, ncomp, seg);
}

}  // namespace

cudaError_t launch_lap3_fused(const Params& p, const float* in, float* out, int ncomp, float scale, int per_sm,
                              cudaStream_t s) {
    // 16 output rows per tile (32 was slower: one 384-thread block per SM at
    // 168 registers); five raw plane slots, four in flight
    return run_lap3<16, 5>(p, in, out, ncomp, scale, per_sm, s);
}

}  // namespace lbm
