// Ensemble batches on one GPU (include/lbm.h, lbm_batch_*): admission by
// pool budget, per-member streams and graphs, non-blocking completion polling.
// Built only on the public C ABI of the single-member library.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include "lbm_common.cuh"

namespace {

struct Block {
    size_t off, size;
};

constexpr int kRounds = 4;  // lbm_batch_run calls whose end each member remembers

struct Member {
    bool used = false;
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

struct lbm_batch {
    char* pool;
    size_t pool_bytes;
    std::vector<Block> free_list;  // sorted by offset, coalesced
    std::vector<Member> m;
    cudaEvent_t epoch;
    int64_t round = 0;  // lbm_batch_run calls so far
};

static void destroy_member_events(Member& mm) {
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
    if (mm.stream) cudaStreamSynchronize(mm.stream);
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

int lbm_batch_run(lbm_batch* b, int64_t steps) {
    if (!b || steps < 0) return berr(LBM_ERR_ARG, "lbm_batch_run: bad argument");
    for (Member& mm : b->m) {
        if (!mm.used || mm.queued >= mm.horizon) continue;
        const int64_t n = steps < mm.horizon - mm.queued ? steps : mm.horizon - mm.queued;
        const int rc = lbm_step(mm.ctx, n);
        if (rc) return rc;
        mm.queued += n;
        const int k = (int)(b->round % kRounds);
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
