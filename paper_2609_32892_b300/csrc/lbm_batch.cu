// Ensemble batches on one GPU (include/lbm.h, lbm_batch_*): admission by
// pool budget, non-blocking completion polling, and two ways to advance the
// members:
//
//   persistent (default)  a member's step is recorded once as a program of
//                         launches (batch.cuh); members whose programs run
//                         the same operations form a class, and each launch
//                         position of a class runs as ONE batched kernel over
//                         every active member of the class: a persistent grid
//                         drawing (member, block) items from a global queue,
//                         over a member table in device memory (recorded
//                         arguments, prefix sums of the members' grids); a
//                         round of steps of a class is captured in one CUDA
//                         graph on the class's stream
//   per member            each member replays its own two-step CUDA graph on
//                         its own stream (also the fallback for a member whose
//                         step has a launch that cannot be batched: a library
//                         call such as cuFFT)
//
// A member's results are bit-identical either way (the batched kernel runs the
// same body on the same block index and grid as the plain launch).
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include "batch.cuh"
#include "lbm_common.cuh"

namespace lbm {
thread_local Recorder* g_rec = nullptr;
}  // namespace lbm

namespace {

struct Block {
    size_t off, size;
};

constexpr int kRounds = 4;  // lbm_batch_run calls whose end each member remembers

struct Member {
    bool used = false;
    int prog = 0;   // 0: step programs not recorded yet, 1: batched, -1: steps on its own
    int64_t nodes = 0;
    int cls = -1;   // its class (batched)
    std::vector<lbm::RecOp> ops[2];      // step programs from population buffer 0 and 1 (arguments uploaded)
    std::vector<const void*> dargs[2];   // device address of each launch's arguments
    unsigned char* dblob = nullptr;      // device copy of the argument blocks
    cudaEvent_t ev_in = nullptr;         // the member's own stream's work, before a batched round
    lbm_ctx* ctx = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    cudaEvent_t rev[kRounds] = {};      // end of this member's work of run call r (slot r % kRounds)
    int64_t rround[kRounds] = {-1, -1, -1, -1};
    size_t off = 0, size = 0;
    int64_t horizon = 0, queued = 0;
    uint64_t tag = 0;
    bool done_recorded = false, reported = false;
};

int berr(int code, const char* fmt, ...) {
    char buf[256];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    lbm::set_global_error(buf);
    return code;
}

}  // namespace

// a class of batched members: the same operations at every launch position
struct TableSlot {
    lbm::BEntry* dev = nullptr;   // member tables of one round (device)
    lbm::BEntry* host = nullptr;  // staging (pinned)
    size_t cap = 0;
    cudaEvent_t used = nullptr;   // after the round's last launch
};
struct Class {
    std::vector<lbm::BatchLaunchFn> sig;
    int lane = 0;                       // classes of one signature split members over lanes
    cudaStream_t s = nullptr;
    unsigned long long* ctr = nullptr;  // [positions][2] work queues (device, self-resetting)
    TableSlot slot[kRounds];
    cudaGraphExec_t gexec = nullptr;    // the last round's graph
};

struct lbm_batch {
    char* pool;
    size_t pool_bytes;
    std::vector<Block> free_list;  // sorted by offset, coalesced
    std::vector<Member> m;
    std::vector<Class> cls;
    cudaEvent_t epoch;
    int64_t round = 0;  // lbm_batch_run calls so far
    int persistent = 1; // 0: per-member graphs; n > 0: persistent, n lanes per signature
    int64_t max_nodes = 16384;  // persistent for members up to this many nodes
    int n_sm = 0;
};

static void destroy_member_events(Member& mm) {
    if (mm.ev_in) cudaEventDestroy(mm.ev_in);
    if (mm.done) cudaEventDestroy(mm.done);
    for (int k = 0; k < kRounds; ++k)
        if (mm.rev[k]) cudaEventDestroy(mm.rev[k]);
}

static size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

static bool pool_alloc(lbm_batch* b, size_t size, size_t* off) {
    size = align256(size);
    for (size_t i = 0; i < b->free_list.size(); ++i) {
        Block& f = b->free_list[i];
        if (f.size >= size) {
            *off = f.off;
            f.off += size;
            f.size -= size;
            if (f.size == 0) b->free_list.erase(b->free_list.begin() + i);
            return true;
        }
    }
    return false;
}

static void pool_free(lbm_batch* b, size_t off, size_t size) {
    size = align256(size);
    size_t i = 0;
    while (i < b->free_list.size() && b->free_list[i].off < off) ++i;
    b->free_list.insert(b->free_list.begin() + i, Block{off, size});
    // coalesce with neighbours
    if (i + 1 < b->free_list.size() && b->free_list[i].off + b->free_list[i].size == b->free_list[i + 1].off) {
        b->free_list[i].size += b->free_list[i + 1].size;
        b->free_list.erase(b->free_list.begin() + i + 1);
    }
    if (i > 0 && b->free_list[i - 1].off + b->free_list[i - 1].size == b->free_list[i].off) {
        b->free_list[i - 1].size += b->free_list[i].size;
        b->free_list.erase(b->free_list.begin() + i);
    }
}

extern "C" {

int lbm_batch_create(int32_t n_slots, void* dev_pool, size_t pool_bytes, lbm_batch** out) {
    if (!out || !dev_pool || n_slots < 1) return berr(LBM_ERR_ARG, "lbm_batch_create: bad argument");
    if (((uintptr_t)dev_pool & 255) != 0) return berr(LBM_ERR_ARG, "lbm_batch_create: pool must be 256-byte aligned");
    lbm_batch* b = new lbm_batch();
    b->pool = (char*)dev_pool;
    b->pool_bytes = pool_bytes;
    b->free_list.push_back(Block{0, pool_bytes & ~(size_t)255});
    b->m.resize(n_slots);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->n_sm, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaEventCreate(&b->epoch);
    if (e == cudaSuccess) e = cudaEventRecord(b->epoch, 0);
    if (e != cudaSuccess) {
        delete b;
        return berr(LBM_ERR_CUDA, "lbm_batch_create: %s", cudaGetErrorString(e));
    }
    *out = b;
    return LBM_OK;
}

int lbm_batch_release(lbm_batch* b, int32_t slot) {
    if (!b || slot < 0 || slot >= (int32_t)b->m.size() || !b->m[slot].used)
        return berr(LBM_ERR_ARG, "lbm_batch_release: bad slot");
    Member& mm = b->m[slot];
    if (mm.stream) cudaStreamSynchronize(mm.stream);  // its batched rounds too (the stream waited on them)
    if (mm.dblob) cudaFreeAsync(mm.dblob, mm.stream);
    lbm_destroy(mm.ctx);
    destroy_member_events(mm);
    if (mm.stream) cudaStreamDestroy(mm.stream);
    pool_free(b, mm.off, mm.size);
    mm = Member();
    return LBM_OK;
}

int lbm_batch_destroy(lbm_batch* b) {
    if (!b) return LBM_OK;
    for (int32_t i = 0; i < (int32_t)b->m.size(); ++i)
        if (b->m[i].used) lbm_batch_release(b, i);
    for (Class& c : b->cls) {
        cudaStreamSynchronize(c.s);
        if (c.gexec) cudaGraphExecDestroy(c.gexec);
        for (TableSlot& t : c.slot) {
            if (t.dev) cudaFreeAsync(t.dev, c.s);
            if (t.host) cudaFreeHost(t.host);
            if (t.used) cudaEventDestroy(t.used);
        }
        if (c.ctr) cudaFreeAsync(c.ctr, c.s);
        cudaStreamSynchronize(c.s);
        cudaStreamDestroy(c.s);
    }
    cudaEventDestroy(b->epoch);
    delete b;
    return LBM_OK;
}

int lbm_batch_admit(lbm_batch* b, const lbm_config* cfg, const double* u0, int64_t horizon, uint64_t tag,
                    int32_t* slot) {
    if (!b || !cfg || !u0 || !slot || horizon < 0) return berr(LBM_ERR_ARG, "lbm_batch_admit: bad argument");
    size_t need = 0;
    int rc = lbm_required_bytes(cfg, &need);
    if (rc) return rc;
    int32_t s = -1;
    for (int32_t i = 0; i < (int32_t)b->m.size(); ++i)
        if (!b->m[i].used) {
            s = i;
            break;
        }
    if (s < 0) return berr(LBM_ERR_BUDGET, "lbm_batch_admit: no free slot");
    size_t off = 0;
    if (!pool_alloc(b, need, &off)) return berr(LBM_ERR_BUDGET, "lbm_batch_admit: %zu bytes do not fit in the pool", need);
    Member& mm = b->m[s];
    cudaError_t e = cudaStreamCreateWithFlags(&mm.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&mm.done, cudaEventDefault);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&mm.ev_in, cudaEventDisableTiming);
    for (int k = 0; k < kRounds && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&mm.rev[k], cudaEventDisableTiming);
    if (e != cudaSuccess) {
        destroy_member_events(mm);
        if (mm.stream) cudaStreamDestroy(mm.stream);
        pool_free(b, off, need);
        mm = Member();
        return berr(LBM_ERR_CUDA, "lbm_batch_admit: %s", cudaGetErrorString(e));
    }
    rc = lbm_create(cfg, b->pool + off, need, mm.stream, &mm.ctx);
    // members overlap one another: a per-member branch only adds queue
    // traffic, and launch shapes should minimise total work, not one
    // member's step time
    if (rc == LBM_OK) rc = lbm_set_branching(mm.ctx, 0);
    if (rc == LBM_OK) rc = lbm_set_launch_goal(mm.ctx, LBM_GOAL_THROUGHPUT);
    if (rc == LBM_OK) rc = lbm_init_macros(mm.ctx, nullptr, u0);
    if (rc != LBM_OK) {
        if (mm.ctx) lbm_destroy(mm.ctx);
        destroy_member_events(mm);
        cudaStreamDestroy(mm.stream);
        pool_free(b, off, need);
        mm = Member();
        return rc;
    }
    mm.used = true;
    mm.nodes = (int64_t)cfg->nx * cfg->ny * cfg->nz;
    mm.off = off;
    mm.size = need;
    mm.horizon = horizon;
    mm.queued = 0;
    mm.tag = tag;
    *slot = s;
    return LBM_OK;
}

int lbm_batch_member(lbm_batch* b, int32_t slot, lbm_ctx** ctx) {
    if (!b || !ctx || slot < 0 || slot >= (int32_t)b->m.size() || !b->m[slot].used)
        return berr(LBM_ERR_ARG, "lbm_batch_member: bad slot");
    *ctx = b->m[slot].ctx;
    return LBM_OK;
}

// Record a member's step programs and upload their arguments; classify it.
static int prepare_member(lbm_batch* b, Member& mm) {
    lbm::Recorder prog[2];
    int rc = lbm::record_step_programs(mm.ctx, prog);
    if (rc) return rc;
    bool ok = prog[0].ok && prog[1].ok && prog[0].ops.size() == prog[1].ops.size() && !prog[0].ops.empty();
    for (size_t i = 0; ok && i < prog[0].ops.size(); ++i) ok = prog[0].ops[i].launch == prog[1].ops[i].launch;
    if (!ok) {
        mm.prog = -1;
        return LBM_OK;
    }
    // argument blocks of both programs in one device blob (16-byte aligned)
    std::vector<unsigned char> blob;
    std::vector<size_t> off[2];
    for (int par = 0; par < 2; ++par)
        for (const lbm::RecOp& r : prog[par].ops) {
            off[par].push_back(blob.size());
            blob.insert(blob.end(), r.args.begin(), r.args.end());
            blob.resize((blob.size() + 15) & ~(size_t)15);
        }
    // stream-ordered: no device-wide synchronisation while other rounds run
    // (the class stream waits on the member's stream before its first round)
    cudaError_t e = cudaMallocAsync((void**)&mm.dblob, blob.size(), mm.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(mm.dblob, blob.data(), blob.size(), cudaMemcpyHostToDevice, mm.stream);
    if (e != cudaSuccess) return berr(LBM_ERR_CUDA, "lbm_batch_run: member arguments: %s", cudaGetErrorString(e));
    for (int par = 0; par < 2; ++par) {
        mm.dargs[par].clear();
        for (size_t i = 0; i < prog[par].ops.size(); ++i) {
            mm.dargs[par].push_back(mm.dblob + off[par][i]);
            prog[par].ops[i].args.clear();
            prog[par].ops[i].args.shrink_to_fit();
        }
        mm.ops[par] = std::move(prog[par].ops);
    }
    // its class: the same operation at every position
    std::vector<lbm::BatchLaunchFn> sig;
    for (const lbm::RecOp& r : mm.ops[0]) sig.push_back(r.launch);
    // the lane of this signature with the fewest active members: lanes run
    // on their own streams, so one lane's small launches (totals, solve)
    // overlap another lane's field kernels
    std::vector<int> count(b->persistent, 0);
    for (const Member& o : b->m)
        if (o.used && o.prog == 1 && b->cls[o.cls].sig == sig) ++count[b->cls[o.cls].lane];
    int lane = 0;
    for (int l = 1; l < b->persistent; ++l)
        if (count[l] < count[lane]) lane = l;
    int ci = -1;
    for (size_t k = 0; k < b->cls.size(); ++k)
        if (b->cls[k].sig == sig && b->cls[k].lane == lane) ci = (int)k;
    if (ci < 0) {
        Class c;
        c.sig = sig;
        c.lane = lane;
        e = cudaStreamCreateWithFlags(&c.s, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaMalloc(&c.ctr, sizeof(unsigned long long) * 2 * sig.size());
        if (e == cudaSuccess) e = cudaMemset(c.ctr, 0, sizeof(unsigned long long) * 2 * sig.size());
        for (int k = 0; k < kRounds && e == cudaSuccess; ++k)
            e = cudaEventCreateWithFlags(&c.slot[k].used, cudaEventDisableTiming);
        if (e != cudaSuccess) return berr(LBM_ERR_CUDA, "lbm_batch_run: new class: %s", cudaGetErrorString(e));
        b->cls.push_back(c);
        ci = (int)b->cls.size() - 1;
    }
    mm.cls = ci;
    mm.prog = 1;
    return LBM_OK;
}

// Queue one round of a class: steps 0 .. S-1, member m active while j < n_m;
// launch position i of step j is one batched kernel over the active members.
static int run_class(lbm_batch* b, int ci, int64_t steps, int k) {
    Class& c = b->cls[ci];
    std::vector<int> mem;
    std::vector<int64_t> nm;
    for (int i = 0; i < (int)b->m.size(); ++i) {
        Member& mm = b->m[i];
        if (!mm.used || mm.prog != 1 || mm.cls != ci || mm.queued >= mm.horizon) continue;
        mem.push_back(i);
        nm.push_back(steps < mm.horizon - mm.queued ? steps : mm.horizon - mm.queued);
    }
    if (mem.empty()) return LBM_OK;
    int64_t S = 0;
    for (int64_t v : nm) S = v > S ? v : S;
    const size_t P = c.sig.size();
    // member tables: for every step and position, the active members' argument
    // blocks and the prefix sums of their grids
    size_t need = 0;
    for (int64_t j = 0; j < S; ++j)
        for (size_t q = 0; q < mem.size(); ++q) need += nm[q] > j ? P : 0;
    TableSlot& ts = c.slot[k];
    cudaError_t e = cudaEventSynchronize(ts.used);  // its previous round has run
    if (e == cudaSuccess && ts.cap < need) {
        if (ts.dev) cudaFreeAsync(ts.dev, c.s);
        if (ts.host) cudaFreeHost(ts.host);
        ts.dev = nullptr;
        ts.host = nullptr;
        ts.cap = need + need / 2 + 64;
        e = cudaMallocAsync((void**)&ts.dev, sizeof(lbm::BEntry) * ts.cap, c.s);
        if (e == cudaSuccess) e = cudaMallocHost((void**)&ts.host, sizeof(lbm::BEntry) * ts.cap);
    }
    if (e != cudaSuccess) return berr(LBM_ERR_CUDA, "lbm_batch_run: tables: %s", cudaGetErrorString(e));
    struct L {
        size_t off;
        int n;
        long long total;
        size_t smem;
    };
    std::vector<L> launches;
    launches.reserve((size_t)S * P);
    size_t at = 0;
    for (int64_t j = 0; j < S; ++j)
        for (size_t i = 0; i < P; ++i) {
            L l{at, 0, 0, 0};
            for (size_t q = 0; q < mem.size(); ++q) {
                if (nm[q] <= j) continue;
                Member& mm = b->m[mem[q]];
                const int par = (lbm::step_parity(mm.ctx) + (int)(j & 1)) & 1;
                const lbm::RecOp& r = mm.ops[par][i];
                ts.host[at].args = mm.dargs[par][i];
                ts.host[at].start = l.total;
                ++at;
                ++l.n;
                l.total += r.blocks;
                if (r.smem > l.smem) l.smem = r.smem;
            }
            launches.push_back(l);
        }
    // the members' own streams (initial fields, coefficients) come first
    for (int i : mem) {
        Member& mm = b->m[i];
        e = cudaEventRecord(mm.ev_in, mm.stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(c.s, mm.ev_in, 0);
        if (e != cudaSuccess) return berr(LBM_ERR_CUDA, "lbm_batch_run: %s", cudaGetErrorString(e));
    }
    // the round as one graph: table upload, S x P batched kernels, the
    // members' completion events
    e = cudaStreamBeginCapture(c.s, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ts.dev, ts.host, sizeof(lbm::BEntry) * at, cudaMemcpyHostToDevice, c.s);
    for (int64_t j = 0; j < S && e == cudaSuccess; ++j) {
        for (size_t i = 0; i < P && e == cudaSuccess; ++i) {
            const L& l = launches[(size_t)j * P + i];
            if (l.n == 0 || l.total == 0) continue;
            const lbm::RecOp& r0 = b->m[mem[0]].ops[0][i];
            int bpsm = r0.smem == l.smem ? r0.blocks_per_sm : r0.prep(l.smem);
            if (bpsm < 1) bpsm = 1;
            const long long cap = (long long)bpsm * b->n_sm;
            const int grid = (int)(l.total < cap ? l.total : cap);
            e = c.sig[i](ts.dev + l.off, l.n, l.total, c.ctr + 2 * i, grid, l.smem, c.s);
        }
        for (size_t q = 0; q < mem.size() && e == cudaSuccess; ++q) {
            Member& mm = b->m[mem[q]];
            if (nm[q] == j + 1 && mm.queued + nm[q] >= mm.horizon && !mm.done_recorded)
                e = cudaEventRecordWithFlags(mm.done, c.s, cudaEventRecordExternal);
        }
    }
    for (int i : mem)
        if (e == cudaSuccess) e = cudaEventRecordWithFlags(b->m[i].rev[k], c.s, cudaEventRecordExternal);
    if (e == cudaSuccess) e = cudaEventRecordWithFlags(ts.used, c.s, cudaEventRecordExternal);
    cudaGraph_t g = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(c.s, &g);
    if (e == cudaSuccess) e = ee;
    if (e == cudaSuccess) {
        // reuse the last round's executable graph when the shape allows
        cudaGraphExecUpdateResultInfo info;
        if (!c.gexec || cudaGraphExecUpdate(c.gexec, g, &info) != cudaSuccess) {
            cudaGetLastError();
            if (c.gexec) cudaGraphExecDestroy(c.gexec);
            c.gexec = nullptr;
            e = cudaGraphInstantiate(&c.gexec, g, 0);
        }
    }
    if (g) cudaGraphDestroy(g);
    if (e == cudaSuccess) e = cudaGraphLaunch(c.gexec, c.s);
    if (e != cudaSuccess) return berr(LBM_ERR_CUDA, "lbm_batch_run: batched round: %s", cudaGetErrorString(e));
    for (size_t q = 0; q < mem.size(); ++q) {
        Member& mm = b->m[mem[q]];
        // later work on the member's own stream (reads, release) follows the round
        e = cudaStreamWaitEvent(mm.stream, mm.rev[k], 0);
        if (e != cudaSuccess) return berr(LBM_ERR_CUDA, "lbm_batch_run: %s", cudaGetErrorString(e));
        mm.rround[k] = b->round;
        mm.queued += nm[q];
        lbm::steps_taken(mm.ctx, nm[q]);
        if (mm.queued >= mm.horizon) mm.done_recorded = true;
    }
    return LBM_OK;
}

int lbm_batch_set_persistent(lbm_batch* b, int lanes, int64_t max_nodes) {
    if (!b || lanes < 0 || lanes > 64 || max_nodes < 0)
        return berr(LBM_ERR_ARG, "lbm_batch_set_persistent: lanes must be 0..64, max_nodes >= 0");
    for (const Member& mm : b->m)
        if (mm.used && mm.prog != 0)
            return berr(LBM_ERR_STATE, "lbm_batch_set_persistent must precede the first lbm_batch_run of its members");
    b->persistent = lanes;
    b->max_nodes = max_nodes;
    return LBM_OK;
}

int lbm_batch_run(lbm_batch* b, int64_t steps) {
    if (!b || steps < 0) return berr(LBM_ERR_ARG, "lbm_batch_run: bad argument");
    const int k = (int)(b->round % kRounds);
    for (Member& mm : b->m) {
        if (!mm.used || mm.prog != 0) continue;
        if (b->persistent && mm.nodes <= b->max_nodes) {
            const int rc = prepare_member(b, mm);
            if (rc) return rc;
        } else {
            mm.prog = -1;
        }
    }
    for (int ci = 0; ci < (int)b->cls.size(); ++ci) {
        const int rc = run_class(b, ci, steps, k);
        if (rc) return rc;
    }
    for (Member& mm : b->m) {
        if (!mm.used || mm.prog != -1 || mm.queued >= mm.horizon) continue;
        const int64_t n = steps < mm.horizon - mm.queued ? steps : mm.horizon - mm.queued;
        const int rc = lbm_step(mm.ctx, n);
        if (rc) return rc;
        mm.queued += n;
        const cudaError_t er = cudaEventRecord(mm.rev[k], mm.stream);
        if (er != cudaSuccess) return berr(LBM_ERR_CUDA, "lbm_batch_run: %s", cudaGetErrorString(er));
        mm.rround[k] = b->round;
        if (mm.queued >= mm.horizon && !mm.done_recorded) {
            const cudaError_t e = cudaEventRecord(mm.done, mm.stream);
            if (e != cudaSuccess) return berr(LBM_ERR_CUDA, "lbm_batch_run: %s", cudaGetErrorString(e));
            mm.done_recorded = true;
        }
    }
    ++b->round;
    return LBM_OK;
}

int lbm_batch_wait(lbm_batch* b, int32_t rounds) {
    if (!b || rounds < 0 || rounds >= kRounds) return berr(LBM_ERR_ARG, "lbm_batch_wait: rounds must be 0..%d", kRounds - 1);
    const int64_t target = b->round - 1 - rounds;  // the latest call that must have finished
    if (target < 0) return LBM_OK;
    const int k = (int)(target % kRounds);
    for (Member& mm : b->m) {
        if (!mm.used || mm.rround[k] != target) continue;  // not active in that call
        const cudaError_t e = cudaEventSynchronize(mm.rev[k]);
        if (e != cudaSuccess) return berr(LBM_ERR_CUDA, "lbm_batch_wait: %s", cudaGetErrorString(e));
    }
    return LBM_OK;
}

int lbm_batch_poll(lbm_batch* b, lbm_completion* out, int32_t cap, int32_t* n) {
    if (!b || !n || (cap > 0 && !out)) return berr(LBM_ERR_ARG, "lbm_batch_poll: bad argument");
    *n = 0;
    for (int32_t i = 0; i < (int32_t)b->m.size() && *n < cap; ++i) {
        Member& mm = b->m[i];
        if (!mm.used || mm.reported) continue;
        if (mm.horizon == 0) {
            mm.done_recorded = true;
            cudaEventRecord(mm.done, mm.stream);
        }
        if (!mm.done_recorded) continue;
        const cudaError_t q = cudaEventQuery(mm.done);
        if (q == cudaErrorNotReady) continue;
        if (q != cudaSuccess) return berr(LBM_ERR_CUDA, "lbm_batch_poll: %s", cudaGetErrorString(q));
        lbm_completion& c = out[(*n)++];
        c.slot = i;
        c.tag = mm.tag;
        c.steps = mm.queued;
        c.status = lbm_sync(mm.ctx);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, b->epoch, mm.done);
        c.t_done_ms = ms;
        mm.reported = true;
    }
    return LBM_OK;
}

int lbm_batch_stats(lbm_batch* b, size_t* free_bytes, size_t* largest, int32_t* active) {
    if (!b) return berr(LBM_ERR_ARG, "lbm_batch_stats: NULL batch");
    size_t tot = 0, big = 0;
    for (const Block& f : b->free_list) {
        tot += f.size;
        if (f.size > big) big = f.size;
    }
    int32_t act = 0;
    for (const Member& mm : b->m) act += mm.used ? 1 : 0;
    if (free_bytes) *free_bytes = tot;
    if (largest) *largest = big;
    if (active) *active = act;
    return LBM_OK;
}

}  // extern "C"
