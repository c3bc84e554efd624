// Batched execution of one kernel over many ensemble members in one launch.
//
// A kernel that supports it is written as a device body taking a virtual
// block (VB: its block index and grid) plus its hardware kernel, which calls
// the body with blockIdx / gridDim.  Its launch goes through go(): normally a
// plain launch; while a Recorder is installed on the calling thread, the
// launch is recorded instead (the body's operation, the grid, the block, the
// dynamic shared memory and the argument values), which is how a member's step
// becomes a program of launches.
//
// batch_kernel runs one recorded launch position for every member of a batch:
// a persistent grid (the SMs times the resident blocks) whose blocks draw work
// items from a global atomic queue; item t is virtual block t - start[m] of
// member m (start[] the prefix sums of the members' grids, searched by
// bisection), run on member m's recorded arguments.  Bodies see exactly the
// block index and grid of their own launch, so a member's results do not
// depend on the batch it runs in.  The last block to leave resets the queue,
// so consecutive launches on one stream reuse it.
#pragma once

#include <stdint.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "lbm_common.cuh"

namespace lbm {

// a kernel body's block index and grid, and how many items the executing
// block ran before this one (0 in a plain launch; a body that keeps state in
// shared memory across items, such as mbarrier phases, reads it)
struct VB {
    int x, y, z, gx, gy, gz, it;
};
__device__ __forceinline__ VB vb_hw() {
    VB v;
    v.x = blockIdx.x; v.y = blockIdx.y; v.z = blockIdx.z;
    v.gx = gridDim.x; v.gy = gridDim.y; v.gz = gridDim.z;
    v.it = 0;
    return v;
}

// argument values of a recorded launch, in kernel-parameter order
template <class... A>
struct Pack;
template <>
struct Pack<> {
    template <class Op, class... B>
    __device__ __forceinline__ void call(const VB& vb, const B&... b) const {
        Op::run(vb, b...);
    }
};
template <class H, class... R>
struct Pack<H, R...> {
    H h;
    Pack<R...> r;
    template <class Op, class... B>
    __device__ __forceinline__ void call(const VB& vb, const B&... b) const {
        r.template call<Op>(vb, b..., h);
    }
};
inline Pack<> make_pack() { return Pack<>{}; }
template <class H, class... R>
inline Pack<H, R...> make_pack(const H& h, const R&... r) {
    return Pack<H, R...>{h, make_pack(r...)};
}

template <class P>
struct BatchArgs {
    int gx, gy, gz, pad;  // the member's grid
    P pack;
};

// one member of a batched launch: its recorded arguments (device memory) and
// the first work item of its blocks
struct BEntry {
    const void* args;
    long long start;
};

template <class Op, class P>
__global__ void __launch_bounds__(Op::NT, Op::MINB) batch_kernel(const BEntry* __restrict__ tab, int nm,
                                                                  long long total, unsigned long long* ctr) {
    __shared__ long long s_t;
    if (threadIdx.x == 0) s_t = (long long)atomicAdd(&ctr[0], 1ull);
    __syncthreads();
    for (int it = 0;; ++it) {
        const long long t = s_t;
        if (t >= total) break;  // uniform over the block
        // the next ticket is drawn now: its latency hides behind this item
        long long next = 0;
        if (threadIdx.x == 0) next = (long long)atomicAdd(&ctr[0], 1ull);
        // member of item t: bisection over the prefix sums (every thread)
        int lo = 0, hi = nm - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (tab[mid].start <= t) lo = mid;
            else hi = mid - 1;
        }
        const BEntry e = tab[lo];
        const BatchArgs<P>& a = *static_cast<const BatchArgs<P>*>(e.args);
        const int local = (int)(t - e.start);
        VB vb;
        vb.gx = a.gx; vb.gy = a.gy; vb.gz = a.gz;
        vb.x = local % a.gx;
        const int r = local / a.gx;
        vb.y = r % a.gy;
        vb.z = r / a.gy;
        vb.it = it;
        a.pack.template call<Op>(vb);
        // every thread (each warp reconverged) is done with the item's shared
        // memory and with s_t; each orders its generic shared-memory accesses
        // before the next item's asynchronous copies
        __syncthreads();
        if (threadIdx.x == 0) s_t = next;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
    }
    // the last block to draw its closing ticket resets the queue
    if (threadIdx.x == 0 && atomicAdd(&ctr[1], 1ull) == (unsigned long long)gridDim.x - 1) {
        ctr[0] = 0;
        ctr[1] = 0;
    }
}

// host side of one batched operation: resident blocks per SM, then the launch
using BatchPrepFn = int (*)(size_t smem);
using BatchLaunchFn = cudaError_t (*)(const BEntry* tab, int nm, long long total, unsigned long long* ctr, int grid,
                                      size_t smem, cudaStream_t s);

template <class Op, class P>
int batch_prep(size_t smem) {
    if (smem > 48 * 1024)
        if (cudaFuncSetAttribute(batch_kernel<Op, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_kernel<Op, P>, Op::NT, smem) != cudaSuccess) return 0;
    return nb;
}
template <class Op, class P>
cudaError_t batch_launch(const BEntry* tab, int nm, long long total, unsigned long long* ctr, int grid, size_t smem,
                         cudaStream_t s) {
    batch_kernel<Op, P><<<grid, Op::NT, smem, s>>>(tab, nm, total, ctr);
    return cudaGetLastError();
}

// one recorded launch of a member's step
struct RecOp {
    BatchLaunchFn launch = nullptr;  // also the identity of the operation
    BatchPrepFn prep = nullptr;      // resident blocks per SM for a dynamic shared-memory size
    int blocks_per_sm = 0;
    size_t smem = 0;
    long long blocks = 0;            // the member's grid, flattened
    std::vector<unsigned char> args; // BatchArgs<P>, copied to device memory by the batch
};
struct Recorder {
    std::vector<RecOp> ops;
    bool ok = true;          // false once a launch could not be recorded
    const char* why = nullptr;
};
extern thread_local Recorder* g_rec;

inline void rec_refuse(const char* why) {
    if (g_rec && g_rec->ok) {
        g_rec->ok = false;
        g_rec->why = why;
    }
}

template <class Op, class... KA>
cudaError_t rec_launch(dim3 g, dim3 b, size_t smem, const KA&... a) {
    using P = Pack<KA...>;
    if ((int)b.x != Op::NT || b.y != 1 || b.z != 1) {
        rec_refuse("block shape differs from the operation's");
        return cudaSuccess;
    }
    RecOp r;
    r.launch = &batch_launch<Op, P>;
    r.prep = &batch_prep<Op, P>;
    r.smem = smem;
    r.blocks_per_sm = batch_prep<Op, P>(smem);
    if (r.blocks_per_sm < 1) {
        rec_refuse("batched kernel does not fit on an SM");
        return cudaSuccess;
    }
    r.blocks = (long long)g.x * g.y * g.z;
    BatchArgs<P> ba;
    memset(&ba, 0, sizeof ba);
    ba.gx = (int)g.x; ba.gy = (int)g.y; ba.gz = (int)g.z;
    ba.pack = make_pack(a...);
    r.args.resize(sizeof ba);
    memcpy(r.args.data(), &ba, sizeof ba);
    g_rec->ops.push_back(std::move(r));
    return cudaSuccess;
}

// lbm_api.cu: a context's step programs (after its pre-step checks and
// tuning), its population parity, and the host-side advance after n steps run
// by a batch
int record_step_programs(lbm_ctx* c, Recorder prog[2]);
int step_parity(const lbm_ctx* c);
void steps_taken(lbm_ctx* c, int64_t n);

// Launch `kernel` (the hardware kernel of operation Op), or record it.
template <class Op, class... KA, class... A>
cudaError_t go(void (*kernel)(KA...), dim3 g, dim3 b, size_t smem, cudaStream_t s, const A&... a) {
    if (g_rec) return rec_launch<Op, KA...>(g, b, smem, static_cast<KA>(a)...);
    kernel<<<g, b, smem, s>>>(a...);
    return cudaGetLastError();
}

}  // namespace lbm
