// eis_api.cu -- host runtime behind the C-ABI of include/eis.h: contexts,
// plans (device-resident pipelines captured into CUDA graphs) and the
// convenience calls.  All device memory of a pipeline is allocated when the
// plan is created; eis_plan_launch only enqueues kernels (or one graph).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <numeric>
#include <vector>

#include "eis.h"
#include "eis_bsgs.cuh"
#include "eis_internal.h"
#include "eis_kernels.h"

using namespace eis;

#define EIS_CK(call)                                            \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) {                                \
            eis_last_cuda_error = e_;                           \
            return EIS_EDEVICE;                                 \
        }                                                       \
    } while (0)

static thread_local cudaError_t eis_last_cuda_error = cudaSuccess;

extern "C" const char *eis_last_cuda_error_string(void) {
    return cudaGetErrorString(eis_last_cuda_error);
}

struct eis_ctx {
    int device = 0;
    int sm_count = 0;
    cudaStream_t stream = nullptr;
    uint64_t budget = 0;
    // Device bytes charged against the budget: the context's tables, every
    // live plan and every live server.  Atomic, because a server's dispatcher
    // thread and plan builds on other threads may reserve at the same time.
    std::atomic<uint64_t> in_use{0};
    uint32_t *d_primes = nullptr;
    uint64_t *d_sqtab = nullptr;  // per odd prime p: (p^2)^(-1) mod 2^64, floor((2^64-1)/p^2)
    uint32_t nprimes = 0;
    std::vector<uint32_t> primes;  // host copy of the odd primes of d_primes
    int *d_single = nullptr;  // [0] result, [1] steps, [2] status
    unsigned char *d_query = nullptr;  // K3 single query: u64 d, i8 out, int status, u64 acc[2], u32 next
    // A lane-search table pool kept from a freed plan for the next one (its
    // bytes stay charged to in_use): freeing and mapping tens of GB per plan
    // cost milliseconds in every eis_classify_range / eis_count_range call.
    std::mutex pool_mu;
    unsigned char *pool_cache = nullptr;
    uint64_t pool_cache_bytes = 0;
    int mode = EIS_MODE_PERSISTENT;
    int ctas_per_sm = 0;
    int threads = 256;
    int64_t step_limit = (int64_t)1 << 26;  // >> any half period below 2^44
    int use_graph = 1;
    int64_t giant_threshold = 0;
    int64_t giant_stride = 0;
    int giant_compose = EIS_COMPOSE_TEXTBOOK;
    int giant_kernel = EIS_GIANT_LANE;
    int mark_every = 16;                    // marked states: about 1 in mark_every
    int64_t bsgs_chunk = (int64_t)1 << 23;  // survivors per record/search round
    int64_t bsgs_walk_cap = 1 << 14;        // steps a giant cycle's walk may take
    int64_t bsgs_window = 64;               // steps a lane walks per search iteration (0: no limit)
    int occ_persistent = 1;
    int occ_record = 1;                     // resident CTAs/SM of k_walk_record
    int occ_bsgs = 1;                       // ... and of k_bsgs
    std::vector<eis_tune_row> tune;         // per-decade lane-search settings (empty: none)
    eis_stats last{};
};

struct PlainBlock {
    uint64_t d_first, cand_first;
    uint32_t ncand;
};

struct eis_plan {
    eis_ctx *ctx = nullptr;
    int mode = EIS_MODE_PERSISTENT;
    size_t n = 0;
    std::vector<Seg> segs;              // layout order (sorted by d0)
    std::vector<uint32_t> user_of;      // layout index -> user index
    std::vector<uint64_t> word_off;     // user index -> first word
    std::vector<Tile> tiles;
    std::vector<PlainBlock> blocks;
    uint64_t total_cand = 0, nwords = 0;
    Seg *d_segs = nullptr;
    Tile *d_tiles = nullptr;
    uint32_t *d_sqfree = nullptr, *d_flags = nullptr;
    uint32_t *d_tile_pop = nullptr, *d_tile_off = nullptr, *d_surv = nullptr;
    uint32_t *d_ctr = nullptr;  // [0] survivors, [1] queue head
    int *d_status = nullptr;
    unsigned long long *d_counts = nullptr;  // [2 s] #E, [2 s + 1] #D
    unsigned long long *d_steps = nullptr;   // [0] baby, [1] giant, [2] deferred
    uint8_t *d_glog = nullptr;
    unsigned long long *d_cls = nullptr;  // [3 s + g] #{d : log eps_d = g} (EIS_PLAN_CLASSES)
    int primes_only = 0;          // EIS_PLAN_PRIMES: classify prime d only
    uint32_t *d_defer = nullptr;  // candidates handed to the giant-step kernel
    uint32_t defer_cap = 0, defer_after = 0;
    int fast = 1;                 // every d of the plan is below kFastDLimit
    int giant_nbaby = 0, giant_log2n = 0;
    uint32_t giant_grid = 0;
    // lane-per-d search (EIS_GIANT_LANE): the survivor queue in rounds of
    // bsgs_chunk positions; each round runs the recording walk, the table
    // index, the search and the fallback walk
    int bsgs = 0;
    uint32_t bsgs_chunk = 0, bsgs_rounds = 0;
    uint32_t bsgs_grid_a = 0, bsgs_grid_b = 0, bsgs_walk_cap = 0, bsgs_window = 0;
    TuneTab tt{};  // the settings each d looks up
    DRecord *d_recs = nullptr;
    unsigned char *d_pool = nullptr;
    uint64_t pool_bytes = 0;  // size of d_pool (possibly a larger cached pool)
    uint32_t *d_fb = nullptr;
    uint32_t *d_bctr = nullptr;  // [0] walk head [1] records [3] search head
                                 // [4] fallbacks [5] fallback walk head
    std::vector<cudaEvent_t> bev;  // per round: start, after the walk, end
    uint64_t bytes = 0;
    uint32_t walk_grid = 0;
    int launches = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    cudaStream_t last_stream = nullptr;
    bool launched = false;
};

// ------------------------------------------------------------------ helpers

// Charge `bytes` to the context's budget; false (nothing charged) if they do
// not fit.
static bool ctx_reserve(eis_ctx *c, uint64_t bytes) {
    uint64_t cur = c->in_use.load();
    do {
        if (bytes > c->budget || cur > c->budget - bytes) return false;
    } while (!c->in_use.compare_exchange_weak(cur, cur + bytes));
    return true;
}

static void ctx_release(eis_ctx *c, uint64_t bytes) {
    uint64_t cur = c->in_use.load();
    while (!c->in_use.compare_exchange_weak(cur, cur - std::min(cur, bytes))) {
    }
}

static int plan_alloc(eis_plan *p, void **ptr, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (!ctx_reserve(p->ctx, bytes)) return EIS_ENOMEM;
    if (cudaMalloc(ptr, bytes) != cudaSuccess) {
        cudaGetLastError();
        ctx_release(p->ctx, bytes);
        return EIS_ENOMEM;
    }
    p->bytes += bytes;
    return EIS_OK;
}

// The cached search pool if it holds at least `bytes` (its charge moves to the
// caller, *got = its size); a smaller one is freed.  nullptr if none fits.
static unsigned char *pool_take(eis_ctx *c, uint64_t bytes, uint64_t *got) {
    std::lock_guard<std::mutex> lk(c->pool_mu);
    *got = 0;
    if (!c->pool_cache) return nullptr;
    unsigned char *q = c->pool_cache;
    const uint64_t qb = c->pool_cache_bytes;
    c->pool_cache = nullptr;
    c->pool_cache_bytes = 0;
    if (qb >= bytes) {
        *got = qb;
        return q;
    }
    cudaFree(q);
    ctx_release(c, qb);
    return nullptr;
}

// Keep a freed plan's pool (still charged) for the next plan; of two pools
// the larger is kept.  The caller has synchronized the device, so no kernel
// still uses it.
static void pool_give(eis_ctx *c, unsigned char *q, uint64_t bytes) {
    std::lock_guard<std::mutex> lk(c->pool_mu);
    if (c->pool_cache && c->pool_cache_bytes >= bytes) {
        cudaFree(q);
        ctx_release(c, bytes);
        return;
    }
    if (c->pool_cache) {
        cudaFree(c->pool_cache);
        ctx_release(c, c->pool_cache_bytes);
    }
    c->pool_cache = q;
    c->pool_cache_bytes = bytes;
}

static uint64_t pool_cached_bytes(eis_ctx *c) {
    std::lock_guard<std::mutex> lk(c->pool_mu);
    return c->pool_cache_bytes;
}

static uint64_t num_candidates(uint64_t lo, uint64_t hi, uint64_t *d0) {
    const uint64_t first = lo + ((13 - lo % 8) % 8);
    *d0 = first;
    return hi > first ? (hi - first + 7) / 8 : 0;
}

static std::vector<uint32_t> odd_primes_below(uint32_t n) {
    std::vector<uint8_t> comp(n, 0);
    std::vector<uint32_t> out;
    for (uint32_t i = 2; i < n; ++i) {
        if (comp[i]) continue;
        if (i > 2) out.push_back(i);
        for (uint64_t j = (uint64_t)i * i; j < n; j += i) comp[j] = 1;
    }
    return out;
}

// Bytes a plan needs per candidate: survivor queue (4) + two bitmaps (1/4),
// plus the optional per-candidate log byte.
static uint64_t max_chunk_cands(const eis_ctx *c, int with_log) {
    const uint64_t used = c->in_use.load();
    const uint64_t free_b = c->budget > used ? c->budget - used : 0;
    uint64_t m = free_b / (5 + (uint64_t)with_log + 1);
    m = std::min<uint64_t>(m, (uint64_t)1 << 31);
    m -= m % kTileCands;
    return m;
}

// Baby-step count N of the giant-step search for discriminants up to d: about
// twice the square root of a typical period (~0.13 sqrt(d) steps), a power of
// two in [256, 4096]; the table holds 4N entries (load <= 1/2).
static void giant_params(uint64_t d, int64_t forced, int &nbaby, int &log2n) {
    int n;
    if (forced > 0) {
        n = 256;
        while (n < forced && n < 4096) n *= 2;
    } else {
        const double ell = 0.13 * std::sqrt((double)d);
        const double want = 2.0 * std::sqrt(std::max(ell, 1.0));
        n = 256;
        while (n < want && n < 4096) n *= 2;
    }
    nbaby = n;
    log2n = 2;
    while ((1 << log2n) < 4 * n) ++log2n;
}

static constexpr int kGiantMaxLog2 = 14;  // 128 KB table per warp at most
static constexpr uint32_t kGiantMaxRounds = 1u << 20;
static constexpr double kTuneMargin = 0.98;  // autotuner: keep the current setting unless 2% faster
static constexpr uint32_t kBsgsMaxCycles = 1u << 20;  // giant cycles per d before the fallback walk
// Plans with fewer candidates than this walk every d to its centre (the
// search's table pool is not worth allocating for them).
static constexpr uint64_t kBsgsMinCands = (uint64_t)1 << 18;

static void record(cudaEvent_t ev, cudaStream_t s, bool capturing) {
    if (capturing)
        cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal);
    else
        cudaEventRecord(ev, s);
}

static int plan_enqueue(eis_plan *p, cudaStream_t s, bool capturing) {
    eis_ctx *c = p->ctx;
    const uint32_t nseg = (uint32_t)p->segs.size();
    const uint32_t ntiles = (uint32_t)p->tiles.size();
    const uint32_t limit = (uint32_t)std::min<int64_t>(c->step_limit, 0xffffffffll);
    int launches = 0;
    record(p->ev[0], s, capturing);
    EIS_CK(cudaMemsetAsync(p->d_flags, 0, p->nwords * 4, s));
    EIS_CK(cudaMemsetAsync(p->d_ctr, 0, 4 * sizeof(uint32_t), s));
    EIS_CK(cudaMemsetAsync(p->d_status, 0, sizeof(int), s));
    EIS_CK(cudaMemsetAsync(p->d_counts, 0, 2 * nseg * sizeof(unsigned long long) + 8, s));
    EIS_CK(cudaMemsetAsync(p->d_steps, 0, 4 * sizeof(unsigned long long), s));
    if (p->d_glog) EIS_CK(cudaMemsetAsync(p->d_glog, 0, p->total_cand, s));
    if (p->d_cls) EIS_CK(cudaMemsetAsync(p->d_cls, 0, 3 * nseg * sizeof(unsigned long long) + 8, s));
    if (ntiles > 0) {
        k_sieve<<<ntiles, 256, 0, s>>>(p->d_tiles, p->d_segs, c->d_primes, c->nprimes, p->d_sqfree,
                                       p->d_tile_pop, p->primes_only);
        ++launches;
        if (p->mode == EIS_MODE_PERSISTENT) {
            k_scan_tiles<<<1, 1024, 0, s>>>(p->d_tile_pop, p->d_tile_off, ntiles, p->d_ctr);
            k_compact<<<ntiles, 256, 0, s>>>(p->d_tiles, p->d_sqfree, p->d_tile_off, p->d_surv);
            launches += 2;
            record(p->ev[1], s, capturing);
            if (p->bsgs) {
                const uint32_t C = p->bsgs_chunk;
                for (uint32_t r = 0; r < p->bsgs_rounds; ++r) {
                    const uint32_t q_lo = r * C;
                    const uint32_t q_hi = (uint32_t)std::min<uint64_t>((uint64_t)q_lo + C, 0xffffffffull);
                    record(p->bev[3 * r], s, capturing);
                    EIS_CK(cudaMemsetAsync(p->d_bctr, 0, 8 * sizeof(uint32_t), s));
                    k_walk_record<<<p->bsgs_grid_a, 256, 0, s>>>(
                        p->d_segs, nseg, p->d_surv, p->d_ctr, q_lo, q_hi, p->d_bctr,
                        p->d_flags, p->d_glog, p->d_steps, p->d_status, limit, p->tt,
                        p->d_recs, p->d_bctr + 1, C, p->d_pool, p->d_steps + 3,
                        p->fast);
                    record(p->bev[3 * r + 1], s, capturing);
                    EIS_CK(launch_k_bsgs(p->bsgs_grid_b, s, p->fast, c->giant_compose, p->d_segs,
                                         nseg, p->d_recs, p->d_bctr + 1, C, p->d_bctr + 3, p->d_pool,
                                         p->d_flags, p->d_glog, p->d_steps + 1, p->d_status,
                                         p->d_fb, p->d_bctr + 4, C, p->tt, kBsgsMaxCycles,
                                         p->bsgs_walk_cap, p->bsgs_window));
                    k_walk_persistent<<<p->walk_grid, 256, 0, s>>>(
                        p->d_segs, nseg, p->d_fb, p->d_bctr + 4, p->d_bctr + 5, p->d_flags,
                        p->d_glog, p->d_steps, p->d_status, limit, 0u, nullptr, nullptr, 0u,
                        p->fast);
                    record(p->bev[3 * r + 2], s, capturing);
                    launches += 3;
                }
            } else {
                k_walk_persistent<<<p->walk_grid, 256, 0, s>>>(
                    p->d_segs, nseg, p->d_surv, p->d_ctr, p->d_ctr + 1, p->d_flags, p->d_glog,
                    p->d_steps, p->d_status, limit, p->defer_after, p->d_defer, p->d_ctr + 2,
                    p->defer_cap, p->fast);
                ++launches;
            }
            record(p->ev[2], s, capturing);
            if (p->d_defer) {
                const size_t smem = (size_t)8 << p->giant_log2n;
                k_giant<<<p->giant_grid, 32, smem, s>>>(
                    nullptr, p->d_segs, nseg, p->d_defer, p->d_ctr + 2, p->defer_cap,
                    p->d_ctr + 3, c->d_primes, c->d_sqtab, c->nprimes, nullptr, p->d_flags, p->d_glog,
                    p->d_steps + 1, p->d_status, p->giant_nbaby, p->giant_log2n, kGiantMaxRounds,
                    c->giant_compose, nullptr);
                ++launches;
            }
            record(p->ev[4], s, capturing);
        } else {
            record(p->ev[1], s, capturing);
            for (const PlainBlock &b : p->blocks) {
                const uint32_t grid = (b.ncand + 255) / 256;
                k_walk_plain<<<grid, 256, 0, s>>>(b.d_first, b.cand_first, b.ncand, p->d_sqfree,
                                                  p->d_flags, p->d_glog, p->d_steps, p->d_status,
                                                  limit);
                ++launches;
            }
            record(p->ev[2], s, capturing);
            record(p->ev[4], s, capturing);
        }
        k_count<<<ntiles, 256, 0, s>>>(p->d_tiles, p->d_flags, p->d_sqfree, p->d_counts, p->d_glog,
                                       p->d_cls);
        ++launches;
    } else {
        record(p->ev[1], s, capturing);
        record(p->ev[2], s, capturing);
        record(p->ev[4], s, capturing);
    }
    record(p->ev[3], s, capturing);
    EIS_CK(cudaGetLastError());
    p->launches = launches;
    return EIS_OK;
}

static void plan_free(eis_plan *p) {
    if (!p) return;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    for (auto &e : p->ev)
        if (e) cudaEventDestroy(e);
    for (auto &e : p->bev)
        if (e) cudaEventDestroy(e);
    if (p->d_pool && p->ctx) {
        // the pool goes to the context's cache; wait for any kernel still
        // using it (as cudaFree would)
        cudaDeviceSynchronize();
        pool_give(p->ctx, p->d_pool, p->pool_bytes);
        p->bytes -= std::min(p->bytes, p->pool_bytes);
        p->d_pool = nullptr;
    }
    void *bufs[] = {p->d_segs, p->d_tiles, p->d_sqfree, p->d_flags, p->d_tile_pop, p->d_tile_off,
                    p->d_surv, p->d_ctr, p->d_status, p->d_counts, p->d_steps, p->d_glog,
                    p->d_defer, p->d_cls, p->d_recs, p->d_pool, p->d_fb, p->d_bctr};
    for (void *b : bufs)
        if (b) cudaFree(b);
    if (p->ctx) ctx_release(p->ctx, p->bytes);
    delete p;
}

static int plan_build(eis_ctx *c, const uint64_t *lo, const uint64_t *hi, size_t n, int mode,
                      int with_log, eis_plan **out, uint32_t flags = 0) {
    EisNvtxRange range("eis.plan_build");
    if (flags & ~(uint32_t)(EIS_PLAN_CLASSES | EIS_PLAN_PRIMES)) return EIS_EINVAL;
    if (flags & EIS_PLAN_CLASSES) with_log = 1;
    if (!c || !out || (n && (!lo || !hi))) return EIS_EINVAL;
    if (mode != EIS_MODE_PLAIN && mode != EIS_MODE_PERSISTENT) return EIS_EINVAL;
    for (size_t i = 0; i < n; ++i) {
        if (lo[i] > hi[i]) return EIS_EINVAL;
        if (hi[i] > EIS_D_LIMIT) return EIS_ERANGE;
    }
    EIS_CK(cudaSetDevice(c->device));
    eis_plan *p = new eis_plan();
    p->ctx = c;
    p->mode = mode;
    p->n = n;
    p->primes_only = (flags & EIS_PLAN_PRIMES) ? 1 : 0;
    std::vector<uint64_t> d0(n), nc(n);
    for (size_t i = 0; i < n; ++i) nc[i] = num_candidates(lo[i], hi[i], &d0[i]);
    std::vector<uint32_t> order(n);
    std::iota(order.begin(), order.end(), 0u);
    std::stable_sort(order.begin(), order.end(),
                     [&](uint32_t a, uint32_t b) { return d0[a] < d0[b]; });
    p->word_off.assign(n, 0);
    uint64_t cur = 0;
    for (uint32_t u : order) {
        Seg s{d0[u], nc[u], cur};
        p->segs.push_back(s);
        p->user_of.push_back(u);
        p->word_off[u] = cur / 32;
        cur += (nc[u] + 31) / 32 * 32;
    }
    p->total_cand = cur;
    p->nwords = cur / 32;
    for (const Seg &sg : p->segs)
        if (sg.ncand && sg.d0 + 8 * (sg.ncand - 1) >= kFastDLimit) p->fast = 0;
    // Survivor indices are 32-bit and the queue head may overshoot by one
    // claim per warp.
    if (cur > 0xffffffffull - (1ull << 24)) {
        plan_free(p);
        return EIS_ENOMEM;
    }
    for (uint32_t si = 0; si < p->segs.size(); ++si) {
        const Seg &s = p->segs[si];
        for (uint64_t off = 0; off < s.ncand; off += kTileCands) {
            Tile t{s.cand0 + off, si, (uint32_t)std::min<uint64_t>(kTileCands, s.ncand - off)};
            p->tiles.push_back(t);
        }
        for (uint64_t off = 0; off < s.ncand; off += kPlainBlockCands) {
            PlainBlock b{s.d0 + 8 * off, s.cand0 + off,
                         (uint32_t)std::min<uint64_t>(kPlainBlockCands, s.ncand - off)};
            p->blocks.push_back(b);
        }
    }
    int rc = EIS_OK;
    const size_t nseg = p->segs.size(), ntiles = p->tiles.size();
#define EIS_ALLOC(ptr, bytes)                                             \
    do {                                                                  \
        rc = plan_alloc(p, (void **)&(ptr), (bytes));                     \
        if (rc != EIS_OK) {                                               \
            plan_free(p);                                                 \
            return rc;                                                    \
        }                                                                 \
    } while (0)
    EIS_ALLOC(p->d_segs, nseg * sizeof(Seg));
    EIS_ALLOC(p->d_tiles, ntiles * sizeof(Tile));
    EIS_ALLOC(p->d_sqfree, p->nwords * 4);
    EIS_ALLOC(p->d_flags, p->nwords * 4);
    EIS_ALLOC(p->d_tile_pop, ntiles * 4);
    EIS_ALLOC(p->d_tile_off, ntiles * 4);
    if (mode == EIS_MODE_PERSISTENT) EIS_ALLOC(p->d_surv, p->total_cand * 4);
    EIS_ALLOC(p->d_ctr, 4 * sizeof(uint32_t));
    EIS_ALLOC(p->d_status, sizeof(int));
    EIS_ALLOC(p->d_counts, 2 * nseg * sizeof(unsigned long long) + 8);
    EIS_ALLOC(p->d_steps, 4 * sizeof(unsigned long long));
    if (with_log) EIS_ALLOC(p->d_glog, p->total_cand);
    if (flags & EIS_PLAN_CLASSES) EIS_ALLOC(p->d_cls, 3 * nseg * sizeof(unsigned long long) + 8);
    // the settings each d of the plan takes: the context's tuning table, or
    // one row of EIS_OPT_GIANT_THRESHOLD / EIS_OPT_MARK_EVERY
    bool any_search = false;
    if (!c->tune.empty()) {
        p->tt.n = (uint32_t)c->tune.size();
        for (size_t r = 0; r < c->tune.size(); ++r) {
            p->tt.d_hi[r] = c->tune[r].d_hi;
            p->tt.nbaby[r] = (uint32_t)c->tune[r].nbaby;
            p->tt.tau[r] = 1.39f / (float)c->tune[r].mark_every;
            any_search |= c->tune[r].nbaby > 0;
        }
    } else {
        p->tt.n = 1;
        p->tt.d_hi[0] = EIS_D_LIMIT;
        p->tt.nbaby[0] = c->giant_kernel == EIS_GIANT_LANE
                             ? (uint32_t)std::min<int64_t>(c->giant_threshold, 0xffffffffll)
                             : 0u;
        p->tt.tau[0] = 1.39f / (float)c->mark_every;
        any_search = p->tt.nbaby[0] > 0;
    }
    if (mode == EIS_MODE_PERSISTENT && any_search && p->total_cand >= kBsgsMinCands) {
        // lane-per-d search: survivors in rounds of C queue positions; the
        // pool holds one table region per resident lane plus one per d a
        // round can hand on
        // round, smaller when the budget left cannot hold the default round;
        // without room for 2^16 survivors per round the plan walks instead
        const uint64_t lanes = (uint64_t)c->sm_count * c->occ_record * 256;
        const uint64_t per_d = kBsgsRegionBytes + sizeof(DRecord) + 4;
        const uint64_t used = c->in_use.load();
        const uint64_t cached = pool_cached_bytes(c);  // reclaimable
        const uint64_t left = c->budget + cached > used ? c->budget + cached - used : 0;
        const uint64_t fit = left / per_d > lanes + 64 ? left / per_d - lanes - 64 : 0;
        uint64_t C = std::min<uint64_t>((uint64_t)c->bsgs_chunk, (p->total_cand + 31) / 32 * 32);
        C = std::min<uint64_t>(C, fit / 32 * 32);
        if (C >= ((uint64_t)1 << 16) || C >= (p->total_cand + 31) / 32 * 32) {
            p->bsgs = 1;
            p->bsgs_walk_cap = (uint32_t)c->bsgs_walk_cap;
            p->bsgs_window = (uint32_t)(c->bsgs_window > 0 ? c->bsgs_window : c->bsgs_walk_cap);
            p->bsgs_chunk = (uint32_t)C;
            p->bsgs_rounds = (uint32_t)((p->total_cand + C - 1) / C);
            p->bsgs_grid_a = (uint32_t)(c->sm_count * c->occ_record);
            p->bsgs_grid_b = (uint32_t)(c->sm_count * c->occ_bsgs);
            const uint64_t pool_need = (lanes + C) * kBsgsRegionBytes;
            uint64_t got = 0;
            p->d_pool = pool_take(c, pool_need, &got);
            if (p->d_pool) {
                p->pool_bytes = got;  // its charge moves to this plan
                p->bytes += got;
            } else {
                EIS_ALLOC(p->d_pool, pool_need);
                p->pool_bytes = pool_need;
            }
            EIS_ALLOC(p->d_recs, C * sizeof(DRecord));
            EIS_ALLOC(p->d_fb, C * 4);
            EIS_ALLOC(p->d_bctr, 8 * sizeof(uint32_t));
            p->bev.assign(3 * (size_t)p->bsgs_rounds, nullptr);
        }
    } else if (mode == EIS_MODE_PERSISTENT && c->giant_threshold > 0 && c->tune.empty() &&
               c->giant_kernel == EIS_GIANT_WARP && p->total_cand > 0) {
        uint64_t dmax = 0;
        for (const Seg &sg : p->segs)
            if (sg.ncand) dmax = std::max(dmax, sg.d0 + 8 * (sg.ncand - 1));
        giant_params(dmax, c->giant_stride, p->giant_nbaby, p->giant_log2n);
        p->giant_log2n = std::min(p->giant_log2n, kGiantMaxLog2);
        p->defer_after = (uint32_t)std::min<int64_t>(c->giant_threshold, 0xffffffffll);
        p->defer_cap = (uint32_t)std::min<uint64_t>(p->total_cand, std::max<uint64_t>(1u << 16, p->total_cand / 4));
        EIS_ALLOC(p->d_defer, (size_t)p->defer_cap * 4);
        int occ = 0;
        const size_t smem = (size_t)8 << p->giant_log2n;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_giant, 32, smem) != cudaSuccess) {
            cudaGetLastError();
            occ = 1;
        }
        p->giant_grid = (uint32_t)(c->sm_count * std::max(1, occ));
    }
#undef EIS_ALLOC
    for (auto &e : p->ev) {
        if (cudaEventCreate(&e) != cudaSuccess) {
            plan_free(p);
            return EIS_EDEVICE;
        }
    }
    for (auto &e : p->bev) {
        if (cudaEventCreate(&e) != cudaSuccess) {
            plan_free(p);
            return EIS_EDEVICE;
        }
    }
    if (nseg && cudaMemcpy(p->d_segs, p->segs.data(), nseg * sizeof(Seg), cudaMemcpyHostToDevice) != cudaSuccess) {
        plan_free(p);
        return EIS_EDEVICE;
    }
    if (ntiles && cudaMemcpy(p->d_tiles, p->tiles.data(), ntiles * sizeof(Tile), cudaMemcpyHostToDevice) != cudaSuccess) {
        plan_free(p);
        return EIS_EDEVICE;
    }
    const int per_sm = c->ctas_per_sm > 0 ? c->ctas_per_sm : c->occ_persistent;
    p->walk_grid = (uint32_t)(c->sm_count * std::max(1, per_sm));
    if (c->use_graph) {
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            plan_free(p);
            return EIS_EDEVICE;
        }
        rc = plan_enqueue(p, c->stream, true);
        cudaError_t e = cudaStreamEndCapture(c->stream, &g);
        if (rc != EIS_OK || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            plan_free(p);
            return rc != EIS_OK ? rc : EIS_EDEVICE;
        }
        p->graph = g;
        if (cudaGraphInstantiate(&p->exec, g, 0) != cudaSuccess) {
            plan_free(p);
            return EIS_EDEVICE;
        }
    }
    *out = p;
    return EIS_OK;
}

static int plan_launch(eis_plan *p, cudaStream_t s) {
    EisNvtxRange range("eis.plan_launch");
    EIS_CK(cudaSetDevice(p->ctx->device));
    if (!s) s = p->ctx->stream;
    if (p->exec) {
        EIS_CK(cudaGraphLaunch(p->exec, s));
    } else {
        int rc = plan_enqueue(p, s, false);
        if (rc != EIS_OK) return rc;
    }
    p->last_stream = s;
    p->launched = true;
    return EIS_OK;
}

static int plan_wait(eis_plan *p) {
    if (!p->launched) return EIS_EINVAL;
    EIS_CK(cudaStreamSynchronize(p->last_stream));
    int status = 0;
    EIS_CK(cudaMemcpy(&status, p->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (status & (kErrSteps | kErrGiant)) return EIS_ESTEPS;
    return EIS_OK;
}

static int plan_fill_stats(eis_plan *p, eis_stats *st) {
    int rc = plan_wait(p);
    if (rc != EIS_OK) return rc;
    std::memset(st, 0, sizeof(*st));
    unsigned long long steps[4] = {0, 0, 0, 0};
    EIS_CK(cudaMemcpy(steps, p->d_steps, sizeof(steps), cudaMemcpyDeviceToHost));
    std::vector<unsigned long long> cnt(2 * p->segs.size() + 1);
    EIS_CK(cudaMemcpy(cnt.data(), p->d_counts, cnt.size() * sizeof(unsigned long long),
                      cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < p->segs.size(); ++i) {
        st->candidates += p->segs[i].ncand;
        st->in_E += cnt[2 * i];
        st->in_D += cnt[2 * i + 1];
    }
    st->baby_steps = steps[0] + steps[1];
    st->giant_steps = steps[2];
    uint32_t ctr[4] = {0, 0, 0, 0};
    EIS_CK(cudaMemcpy(ctr, p->d_ctr, sizeof(ctr), cudaMemcpyDeviceToHost));
    st->deferred = p->d_defer ? std::min(ctr[2], p->defer_cap) : 0;
    if (p->bsgs) {
        // steps[0]: baby steps of the recording and fallback walks, [1]: steps
        // of the search's walks, [2]: giant cycles, [3]: d handed on
        st->baby_steps = steps[0] + steps[1];
        st->search_steps = steps[1];
        st->giant_steps = steps[2];
        st->deferred = steps[3];
    }
    float ms = 0;
    if (cudaEventElapsedTime(&ms, p->ev[0], p->ev[3]) == cudaSuccess) st->ms_total = ms;
    if (cudaEventElapsedTime(&ms, p->ev[0], p->ev[1]) == cudaSuccess) st->ms_sieve = ms;
    if (cudaEventElapsedTime(&ms, p->ev[1], p->ev[2]) == cudaSuccess) st->ms_walk = ms;
    if (cudaEventElapsedTime(&ms, p->ev[2], p->ev[4]) == cudaSuccess) st->ms_giant = ms;
    if (p->bsgs) {
        double walk = 0, giant = 0;
        for (uint32_t r = 0; r < p->bsgs_rounds; ++r) {
            if (cudaEventElapsedTime(&ms, p->bev[3 * r], p->bev[3 * r + 1]) == cudaSuccess) walk += ms;
            if (cudaEventElapsedTime(&ms, p->bev[3 * r + 1], p->bev[3 * r + 2]) == cudaSuccess)
                giant += ms;
        }
        st->ms_walk = walk;
        st->ms_giant = giant;
    }
    cudaGetLastError();
    st->launches = p->launches;
    st->sm_count = p->ctx->sm_count;
    return EIS_OK;
}

static int plan_counts_user(eis_plan *p, uint64_t *counts_out) {
    int rc = plan_wait(p);
    if (rc != EIS_OK) return rc;
    std::vector<unsigned long long> cnt(2 * p->segs.size() + 1);
    EIS_CK(cudaMemcpy(cnt.data(), p->d_counts, cnt.size() * sizeof(unsigned long long),
                      cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < p->segs.size(); ++i) counts_out[p->user_of[i]] = cnt[2 * i];
    return EIS_OK;
}

// Run [lo, hi) in chunks of at most M candidates (M a multiple of the tile
// size, so chunk j starts at candidate j*M and at output word j*M/32).  The
// callback gets each finished chunk's plan and candidate offset.
template <class F>
static int run_chunks(eis_ctx *c, uint64_t lo, uint64_t hi, int with_log, cudaStream_t s,
                      eis_stats *acc, F &&on_chunk) {
    if (!c || lo > hi) return EIS_EINVAL;
    if (hi > EIS_D_LIMIT) return EIS_ERANGE;
    uint64_t d0;
    const uint64_t ntot = num_candidates(lo, hi, &d0);
    const uint64_t M = max_chunk_cands(c, with_log);
    if (M == 0) return EIS_ENOMEM;
    std::memset(acc, 0, sizeof(*acc));
    for (uint64_t off = 0; off < ntot || (off == 0 && ntot == 0); off += M) {
        const uint64_t a = lo + 8 * off;
        const uint64_t b = std::min(hi, lo + 8 * (off + M));
        eis_plan *p = nullptr;
        int rc = plan_build(c, &a, &b, 1, c->mode, with_log, &p);
        if (rc != EIS_OK) return rc;
        rc = plan_launch(p, s);
        eis_stats st{};
        if (rc == EIS_OK) rc = plan_fill_stats(p, &st);
        if (rc == EIS_OK) rc = on_chunk(p, off);
        plan_free(p);
        if (rc != EIS_OK) return rc;
        acc->candidates += st.candidates;
        acc->in_D += st.in_D;
        acc->in_E += st.in_E;
        acc->baby_steps += st.baby_steps;
        acc->giant_steps += st.giant_steps;
        acc->search_steps += st.search_steps;
        acc->deferred += st.deferred;
        acc->ms_total += st.ms_total;
        acc->ms_walk += st.ms_walk;
        acc->ms_sieve += st.ms_sieve;
        acc->ms_giant += st.ms_giant;
        acc->launches += st.launches;
        acc->sm_count = st.sm_count;
        if (ntot == 0) break;
    }
    return EIS_OK;
}

// ------------------------------------------------------------------ internal view

eis_ctx_view eis_ctx_get_view(eis_ctx *c) {
    eis_ctx_view v;
    v.device = c->device;
    v.d_primes = c->d_primes;
    v.d_sqtab = c->d_sqtab;
    v.nprimes = c->nprimes;
    const int per_sm = c->ctas_per_sm > 0 ? c->ctas_per_sm : c->occ_persistent;
    v.walk_grid = (uint32_t)(c->sm_count * std::max(1, per_sm));
    v.giant_grid = (uint32_t)(c->sm_count * 4);
    v.giant_compose = c->giant_compose;
    v.step_limit = (uint32_t)std::min<int64_t>(c->step_limit, 0xffffffffll);
    return v;
}

void eis_giant_params(uint64_t d, int64_t forced, int &nbaby, int &log2n) {
    giant_params(d, forced, nbaby, log2n);
    log2n = std::min(log2n, kGiantMaxLog2);
}

bool eis_ctx_reserve(eis_ctx *c, uint64_t bytes) { return ctx_reserve(c, bytes); }

void eis_ctx_release(eis_ctx *c, uint64_t bytes) { ctx_release(c, bytes); }

// ------------------------------------------------------------------ C-ABI

extern "C" {

const char *eis_strerror(int code) {
    switch (code) {
        case EIS_OK: return "ok";
        case EIS_EINVAL: return "invalid argument";
        case EIS_ENOTD: return "d is not a square-free d == 5 (mod 8)";
        case EIS_ERANGE: return "value above the supported limit 2^44";
        case EIS_ENOMEM: return "out of memory or over the context's budget";
        case EIS_ETIMEOUT: return "wait timed out";
        case EIS_EDEVICE: return "CUDA error";
        case EIS_ESTEPS: return "a walk ran past its step limit";
        case EIS_EBUSY: return "request not admitted";
        case EIS_ENOTFOUND: return "unknown request";
        case EIS_ECANCELED: return "request cancelled";
        case EIS_ETOOLARGE: return "range has more candidates than the no-allocation call's fixed scratch (2^20)";
        default: return "unknown error";
    }
}

int eis_create(eis_ctx **out, int device, uint64_t mem_budget_bytes) {
    if (!out) return EIS_EINVAL;
    *out = nullptr;
    int ndev = 0;
    EIS_CK(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return EIS_EINVAL;
    EIS_CK(cudaSetDevice(device));
    eis_ctx *c = new eis_ctx();
    c->device = device;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
        delete c;
        return EIS_EDEVICE;
    }
    c->sm_count = prop.multiProcessorCount;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        delete c;
        return EIS_EDEVICE;
    }
    c->budget = mem_budget_bytes ? mem_budget_bytes : (uint64_t)free_b / 4 * 3;
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete c;
        return EIS_EDEVICE;
    }
    std::vector<uint32_t> pr = odd_primes_below(1u << 22);
    c->nprimes = (uint32_t)pr.size();
    c->primes = pr;
    // Every table of the context is charged once: primes, the square-free
    // test table (16 B per prime), the single-query words.
    if (!ctx_reserve(c, pr.size() * 4 + pr.size() * 16 + 4 * sizeof(int) + 64)) {
        eis_destroy(c);
        return EIS_ENOMEM;
    }
    if (cudaMalloc(&c->d_primes, pr.size() * 4) != cudaSuccess ||
        cudaMalloc(&c->d_single, 4 * sizeof(int)) != cudaSuccess) {
        eis_destroy(c);
        return EIS_ENOMEM;
    }
    // Division-free square-free test table (Granlund & Montgomery, section 9):
    // for odd m = p^2, m | d iff d * m^(-1) mod 2^64 <= floor((2^64-1)/m).
    {
        std::vector<uint64_t> tab(2 * pr.size());
        for (size_t i = 0; i < pr.size(); ++i) {
            const uint64_t m = (uint64_t)pr[i] * pr[i];
            uint64_t x = m;  // m * m == 1 (mod 8)
            for (int k = 0; k < 5; ++k) x *= 2 - m * x;
            tab[2 * i] = x;
            tab[2 * i + 1] = UINT64_MAX / m;
        }
        if (cudaMalloc(&c->d_sqtab, tab.size() * 8) != cudaSuccess ||
            cudaMemcpy(c->d_sqtab, tab.data(), tab.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess) {
            eis_destroy(c);
            return EIS_ENOMEM;
        }
    }
    if (cudaMalloc(&c->d_query, 64) != cudaSuccess) {
        eis_destroy(c);
        return EIS_ENOMEM;
    }
    if (cudaFuncSetAttribute(k_giant, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(8u << kGiantMaxLog2)) != cudaSuccess) {
        eis_destroy(c);
        return EIS_EDEVICE;
    }
    if (cudaMemcpy(c->d_primes, pr.data(), pr.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
        eis_destroy(c);
        return EIS_EDEVICE;
    }
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_walk_persistent, 256, 0) != cudaSuccess)
        occ = 1;
    c->occ_persistent = std::max(1, occ);
    occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_walk_record, 256, 0) != cudaSuccess)
        occ = 1;
    c->occ_record = std::max(1, occ);
    occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_bsgs_kernel(1, EIS_COMPOSE_TEXTBOOK),
                                                      128, 0) != cudaSuccess)
        occ = 1;
    c->occ_bsgs = std::max(1, occ);
    cudaGetLastError();
    *out = c;
    return EIS_OK;
}

int eis_destroy(eis_ctx *c) {
    if (!c) return EIS_OK;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->d_primes) cudaFree(c->d_primes);
    if (c->d_single) cudaFree(c->d_single);
    if (c->d_query) cudaFree(c->d_query);
    if (c->d_sqtab) cudaFree(c->d_sqtab);
    if (c->pool_cache) cudaFree(c->pool_cache);
    if (c->stream) cudaStreamDestroy(c->stream);
    delete c;
    return EIS_OK;
}

int eis_set_option(eis_ctx *c, int key, int64_t v) {
    if (!c) return EIS_EINVAL;
    switch (key) {
        case EIS_OPT_MODE:
            if (v != EIS_MODE_PLAIN && v != EIS_MODE_PERSISTENT) return EIS_EINVAL;
            c->mode = (int)v;
            return EIS_OK;
        case EIS_OPT_CTAS_PER_SM:
            if (v < 0 || v > 64) return EIS_EINVAL;
            c->ctas_per_sm = (int)v;
            return EIS_OK;
        case EIS_OPT_THREADS:
            if (v != 256) return EIS_EINVAL;
            c->threads = (int)v;
            return EIS_OK;
        case EIS_OPT_STEP_LIMIT:
            if (v < 1 || v > 0xffffffffll) return EIS_EINVAL;
            c->step_limit = v;
            return EIS_OK;
        case EIS_OPT_USE_GRAPH:
            c->use_graph = v ? 1 : 0;
            return EIS_OK;
        case EIS_OPT_GIANT_THRESHOLD:
            if (v < 0) return EIS_EINVAL;
            c->giant_threshold = v;
            return EIS_OK;
        case EIS_OPT_GIANT_STRIDE:
            if (v < 0) return EIS_EINVAL;
            c->giant_stride = v;
            return EIS_OK;
        case EIS_OPT_GIANT_COMPOSE:
            if (v != EIS_COMPOSE_TEXTBOOK && v != EIS_COMPOSE_NUCOMP) return EIS_EINVAL;
            c->giant_compose = (int)v;
            return EIS_OK;
        case EIS_OPT_GIANT_KERNEL:
            if (v != EIS_GIANT_LANE && v != EIS_GIANT_WARP) return EIS_EINVAL;
            c->giant_kernel = (int)v;
            return EIS_OK;
        case EIS_OPT_MARK_EVERY:
            if (v < 2 || v > 4096) return EIS_EINVAL;
            c->mark_every = (int)v;
            return EIS_OK;
        case EIS_OPT_BSGS_CHUNK:
            if (v < 4096 || v > ((int64_t)1 << 28)) return EIS_EINVAL;
            c->bsgs_chunk = v;
            return EIS_OK;
        case EIS_OPT_BSGS_WALK_CAP:
            if (v < 1 || v > ((int64_t)1 << 24)) return EIS_EINVAL;
            c->bsgs_walk_cap = v;
            return EIS_OK;
        case EIS_OPT_BSGS_WINDOW:
            if (v < 0 || v > ((int64_t)1 << 24)) return EIS_EINVAL;
            c->bsgs_window = v;
            return EIS_OK;
        default:
            return EIS_EINVAL;
    }
}

int eis_get_option(eis_ctx *c, int key, int64_t *v) {
    if (!c || !v) return EIS_EINVAL;
    switch (key) {
        case EIS_OPT_MODE: *v = c->mode; return EIS_OK;
        case EIS_OPT_CTAS_PER_SM: *v = c->ctas_per_sm ? c->ctas_per_sm : c->occ_persistent; return EIS_OK;
        case EIS_OPT_THREADS: *v = c->threads; return EIS_OK;
        case EIS_OPT_STEP_LIMIT: *v = c->step_limit; return EIS_OK;
        case EIS_OPT_USE_GRAPH: *v = c->use_graph; return EIS_OK;
        case EIS_OPT_GIANT_THRESHOLD: *v = c->giant_threshold; return EIS_OK;
        case EIS_OPT_GIANT_STRIDE: *v = c->giant_stride; return EIS_OK;
        case EIS_OPT_GIANT_COMPOSE: *v = c->giant_compose; return EIS_OK;
        case EIS_OPT_GIANT_KERNEL: *v = c->giant_kernel; return EIS_OK;
        case EIS_OPT_MARK_EVERY: *v = c->mark_every; return EIS_OK;
        case EIS_OPT_BSGS_CHUNK: *v = c->bsgs_chunk; return EIS_OK;
        case EIS_OPT_BSGS_WALK_CAP: *v = c->bsgs_walk_cap; return EIS_OK;
        case EIS_OPT_BSGS_WINDOW: *v = c->bsgs_window; return EIS_OK;
        case EIS_OPT_MEM_BUDGET: *v = (int64_t)c->budget; return EIS_OK;
        case EIS_OPT_MEM_IN_USE: *v = (int64_t)c->in_use.load(); return EIS_OK;
        default: return EIS_EINVAL;
    }
}

int eis_get_stats(eis_ctx *c, eis_stats *out) {
    if (!c || !out) return EIS_EINVAL;
    *out = c->last;
    return EIS_OK;
}

int eis_plan_create(eis_ctx *c, const uint64_t *lo, const uint64_t *hi, size_t n, int mode,
                    eis_plan **out) {
    return plan_build(c, lo, hi, n, mode, 0, out);
}

int eis_plan_create_ex(eis_ctx *c, const uint64_t *lo, const uint64_t *hi, size_t n, int mode,
                       uint32_t flags, eis_plan **out) {
    return plan_build(c, lo, hi, n, mode, 0, out, flags);
}

int eis_plan_class_counts(eis_plan *p, uint64_t *out) {
    if (!p || (!out && p->n)) return EIS_EINVAL;
    if (!p->d_cls) return EIS_EINVAL;
    int rc = plan_wait(p);
    if (rc != EIS_OK) return rc;
    std::vector<unsigned long long> cnt(3 * p->segs.size() + 1);
    EIS_CK(cudaMemcpy(cnt.data(), p->d_cls, cnt.size() * sizeof(unsigned long long),
                      cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < p->segs.size(); ++i)
        for (int g = 0; g < 3; ++g) out[3 * p->user_of[i] + g] = cnt[3 * i + g];
    return EIS_OK;
}

int eis_class_counts(eis_ctx *c, uint64_t lo, uint64_t hi, int primes_only, uint64_t out[3]) {
    if (!c || !out) return EIS_EINVAL;
    if (lo > hi) return EIS_EINVAL;
    if (hi > EIS_D_LIMIT) return EIS_ERANGE;
    uint64_t d0;
    const uint64_t ntot = num_candidates(lo, hi, &d0);
    const uint64_t M = max_chunk_cands(c, 1);
    if (M == 0) return EIS_ENOMEM;
    uint64_t acc[3] = {0, 0, 0};
    const uint32_t flags = EIS_PLAN_CLASSES | (primes_only ? EIS_PLAN_PRIMES : 0u);
    for (uint64_t off = 0; off < ntot; off += M) {
        const uint64_t a = lo + 8 * off;
        const uint64_t b = std::min(hi, lo + 8 * (off + M));
        eis_plan *p = nullptr;
        int rc = plan_build(c, &a, &b, 1, c->mode == EIS_MODE_PLAIN ? EIS_MODE_PLAIN
                                                                     : EIS_MODE_PERSISTENT,
                            1, &p, flags);
        if (rc != EIS_OK) return rc;
        rc = plan_launch(p, c->stream);
        uint64_t part[3] = {0, 0, 0};
        if (rc == EIS_OK) rc = eis_plan_class_counts(p, part);
        plan_free(p);
        if (rc != EIS_OK) return rc;
        for (int g = 0; g < 3; ++g) acc[g] += part[g];
    }
    for (int g = 0; g < 3; ++g) out[g] = acc[g];
    return EIS_OK;
}

int eis_plan_launch(eis_plan *p, void *stream) {
    if (!p) return EIS_EINVAL;
    return plan_launch(p, (cudaStream_t)stream);
}

int eis_plan_counts(eis_plan *p, uint64_t *counts_out) {
    if (!p || (!counts_out && p->n)) return EIS_EINVAL;
    return plan_counts_user(p, counts_out);
}

int eis_plan_counts_D(eis_plan *p, uint64_t *counts_D_out) {
    if (!p || (!counts_D_out && p->n)) return EIS_EINVAL;
    int rc = plan_wait(p);
    if (rc != EIS_OK) return rc;
    std::vector<unsigned long long> cnt(2 * p->segs.size() + 1);
    EIS_CK(cudaMemcpy(cnt.data(), p->d_counts, cnt.size() * sizeof(unsigned long long),
                      cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < p->segs.size(); ++i) counts_D_out[p->user_of[i]] = cnt[2 * i + 1];
    return EIS_OK;
}

int eis_plan_bitmaps(eis_plan *p, const uint32_t **flags, const uint32_t **sqfree,
                     uint64_t *word_offset, uint64_t *total_words) {
    if (!p) return EIS_EINVAL;
    if (flags) *flags = p->d_flags;
    if (sqfree) *sqfree = p->d_sqfree;
    if (word_offset)
        for (size_t i = 0; i < p->n; ++i) word_offset[i] = p->word_off[i];
    if (total_words) *total_words = p->nwords;
    return EIS_OK;
}

int eis_plan_copy_bitmaps(eis_plan *p, uint32_t *flags_out, uint32_t *sqfree_out,
                          int out_on_device) {
    if (!p) return EIS_EINVAL;
    int rc = plan_wait(p);
    if (rc != EIS_OK) return rc;
    const cudaMemcpyKind kind = out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (flags_out && p->nwords) EIS_CK(cudaMemcpy(flags_out, p->d_flags, p->nwords * 4, kind));
    if (sqfree_out && p->nwords) EIS_CK(cudaMemcpy(sqfree_out, p->d_sqfree, p->nwords * 4, kind));
    return EIS_OK;
}

int eis_plan_stats(eis_plan *p, eis_stats *out) {
    if (!p || !out) return EIS_EINVAL;
    return plan_fill_stats(p, out);
}

int eis_plan_destroy(eis_plan *p) {
    if (!p) return EIS_OK;
    cudaSetDevice(p->ctx->device);
    if (p->launched) cudaStreamSynchronize(p->last_stream);
    plan_free(p);
    return EIS_OK;
}

static bool tune_rows_valid(const eis_tune_row *rows, size_t n) {
    if (n > EIS_TUNE_MAX_ROWS) return false;
    for (size_t r = 0; r < n; ++r) {
        if (rows[r].nbaby < 0 || rows[r].mark_every < 2 || rows[r].mark_every > 4096) return false;
        if (r && rows[r].d_hi <= rows[r - 1].d_hi) return false;
    }
    return true;
}

int eis_set_tune_table(eis_ctx *c, const eis_tune_row *rows, size_t n) {
    if (!c || (n && !rows) || !tune_rows_valid(rows, n)) return EIS_EINVAL;
    c->tune.assign(rows, rows + n);
    return EIS_OK;
}

int eis_get_tune_table(eis_ctx *c, eis_tune_row *rows, size_t cap, size_t *n_out) {
    if (!c || !n_out || (cap && !rows)) return EIS_EINVAL;
    *n_out = c->tune.size();
    for (size_t r = 0; r < c->tune.size() && r < cap; ++r) rows[r] = c->tune[r];
    return EIS_OK;
}

// Candidate (nbaby, mark_every) pairs of the decade tuner; {0, 16} is the
// walk alone.
static const eis_tune_row kTuneGrid[] = {
    {0, 0, 16},    {0, 1024, 16}, {0, 1536, 24}, {0, 2048, 24}, {0, 2048, 32},
    {0, 2048, 40}, {0, 2304, 48}, {0, 2560, 32}, {0, 3072, 32}, {0, 3072, 40},
    {0, 4096, 32}, {0, 4096, 48}, {0, 6144, 64}, {0, 8192, 64},
};

int eis_autotune_decades(eis_ctx *c, uint64_t d_lo, uint64_t d_hi, eis_tune_row *rows_out,
                         size_t cap, size_t *n_out) {
    EisNvtxRange range("eis.autotune_decades");
    if (!c || d_lo >= d_hi || (cap && !rows_out)) return EIS_EINVAL;
    if (d_hi > EIS_D_LIMIT) return EIS_ERANGE;
    const std::vector<eis_tune_row> saved = c->tune;
    const int saved_mode = c->mode;
    c->mode = EIS_MODE_PERSISTENT;
    std::vector<eis_tune_row> found;
    int rc = EIS_OK;
    uint64_t dec_lo = 1;
    while (dec_lo * 10 <= d_lo) dec_lo *= 10;
    for (; dec_lo < d_hi && rc == EIS_OK; dec_lo *= 10) {
        const uint64_t dec_hi = std::min<uint64_t>(dec_lo * 10, EIS_D_LIMIT);
        const uint64_t top = std::min(dec_hi, d_hi);
        const uint64_t bot = std::max(dec_lo, d_lo);
        if (bot >= top) continue;
        const uint64_t width = (uint64_t)8 << 22;  // 2^22 candidates
        const uint64_t slo = top - bot > width ? top - width : bot;
        uint64_t ref = 0;
        double best_ms = 1e300, walk_ms = 1e300;
        eis_tune_row best = kTuneGrid[0];
        for (const eis_tune_row &cand : kTuneGrid) {
            eis_tune_row one = cand;
            one.d_hi = EIS_D_LIMIT;
            c->tune.assign(1, one);
            eis_plan *p = nullptr;
            rc = plan_build(c, &slo, &top, 1, EIS_MODE_PERSISTENT, 0, &p);
            if (rc != EIS_OK) break;
            double ms = 1e300;
            uint64_t count = 0;
            for (int rep = 0; rep < 2 && rc == EIS_OK; ++rep) {
                rc = plan_launch(p, c->stream);
                eis_stats st{};
                if (rc == EIS_OK) rc = plan_fill_stats(p, &st);
                if (rc == EIS_OK) {
                    ms = std::min(ms, st.ms_total);
                    count = st.in_E;
                }
            }
            plan_free(p);
            if (rc != EIS_OK) break;
            if (cand.nbaby == 0) {
                ref = count;
                walk_ms = ms;
            } else if (count != ref) {  // every setting must give the same count
                rc = EIS_EDEVICE;
                break;
            }
            if (ms < best_ms) {
                best_ms = ms;
                best = cand;
            }
        }
        if (rc != EIS_OK) break;
        if (best.nbaby && !(best_ms < kTuneMargin * walk_ms)) best = kTuneGrid[0];
        best.d_hi = dec_hi;
        found.push_back(best);
    }
    c->mode = saved_mode;
    if (rc != EIS_OK) {
        c->tune = saved;
        return rc;
    }
    // merge: the rows found replace the saved rows of the same decades
    std::vector<eis_tune_row> table;
    const uint64_t lo_cov = found.empty() ? 0 : found.front().d_hi / 10;
    const uint64_t hi_cov = found.empty() ? 0 : found.back().d_hi;
    for (const eis_tune_row &r : saved)
        if (r.d_hi <= lo_cov) table.push_back(r);
    for (const eis_tune_row &r : found) table.push_back(r);
    for (const eis_tune_row &r : saved)
        if (r.d_hi > hi_cov) table.push_back(r);
    std::vector<eis_tune_row> merged;
    for (const eis_tune_row &r : table) {
        if (!merged.empty() && merged.back().nbaby == r.nbaby &&
            merged.back().mark_every == r.mark_every)
            merged.back().d_hi = r.d_hi;
        else
            merged.push_back(r);
    }
    // (the last row also covers every larger d; its d_hi stays its decade's
    // top so that later calls merge by decade)
    if (merged.size() > EIS_TUNE_MAX_ROWS) merged.resize(EIS_TUNE_MAX_ROWS);
    c->tune = merged;
    if (n_out) *n_out = found.size();
    for (size_t r = 0; r < found.size() && r < cap; ++r) rows_out[r] = found[r];
    return EIS_OK;
}

int eis_autotune(eis_ctx *c, uint64_t lo, uint64_t hi, eis_tune_result *out) {
    EisNvtxRange range("eis.autotune");
    if (!c || !out || lo >= hi) return EIS_EINVAL;
    if (hi > EIS_D_LIMIT) return EIS_ERANGE;
    // CTAs per SM of the walk; threads per d (0 = walk only, the lane search
    // at 1 thread per d, the warp-per-d kernel at 32) with its threshold;
    // and the round size of the lane search (the chunk of survivors whose
    // tables one round holds)
    struct Setting {
        int ctas;
        int kernel;
        int64_t thr, chunk;
    };
    const int occ = c->occ_persistent;
    std::vector<Setting> cands;
    for (int ctas : {occ, std::max(1, occ * 3 / 4), std::max(1, occ / 2)})
        cands.push_back({ctas, EIS_GIANT_LANE, 0, c->bsgs_chunk});
    for (int64_t thr : {(int64_t)32768, (int64_t)131072})
        cands.push_back({occ, EIS_GIANT_WARP, thr, c->bsgs_chunk});
    const int64_t lane_thr = c->giant_kernel == EIS_GIANT_LANE && c->giant_threshold > 0
                                 ? c->giant_threshold
                                 : 2048;
    for (int64_t chunk : {(int64_t)1 << 22, (int64_t)1 << 23, (int64_t)1 << 24, (int64_t)1 << 25})
        cands.push_back({occ, EIS_GIANT_LANE, lane_thr, chunk});
    const Setting prev{c->ctas_per_sm, c->giant_kernel, c->giant_threshold, c->bsgs_chunk};
    const int prev_mode = c->mode;
    const std::vector<eis_tune_row> saved_table = c->tune;
    c->tune.clear();  // the trials use the context's global settings
    c->mode = EIS_MODE_PERSISTENT;
    auto apply = [&](const Setting &st) {
        c->ctas_per_sm = st.ctas;
        c->giant_kernel = st.kernel;
        c->giant_threshold = st.thr;
        c->bsgs_chunk = st.chunk;
    };
    auto time_one = [&](const Setting &st, double &ms, uint64_t &count) -> int {
        apply(st);
        eis_plan *p = nullptr;
        int rc = plan_build(c, &lo, &hi, 1, EIS_MODE_PERSISTENT, 0, &p);
        if (rc != EIS_OK) return rc;
        double best = 1e300;
        for (int rep = 0; rep < 2 && rc == EIS_OK; ++rep) {
            rc = plan_launch(p, c->stream);
            eis_stats stt{};
            if (rc == EIS_OK) rc = plan_fill_stats(p, &stt);
            if (rc == EIS_OK) {
                best = std::min(best, stt.ms_total);
                count = stt.in_E;
            }
        }
        plan_free(p);
        ms = best;
        return rc;
    };
    double ms_prev = 0;
    uint64_t ref_count = 0, cnt = 0;
    int rc = time_one(prev, ms_prev, ref_count);
    Setting best = prev;
    double ms_best = ms_prev;
    int trials = 1;
    for (const Setting &st : cands) {
        if (rc != EIS_OK) break;
        double ms = 0;
        rc = time_one(st, ms, cnt);
        if (rc != EIS_OK) break;
        if (cnt != ref_count) {  // every setting must give the same count
            rc = EIS_EDEVICE;
            break;
        }
        ++trials;
        // A setting replaces the current one only when it is faster by more
        // than the sample's run-to-run noise (2%); the sample below the
        // window is not the window itself.
        if (ms < ms_best && ms < kTuneMargin * ms_prev) {
            ms_best = ms;
            best = st;
        }
    }
    c->mode = prev_mode;
    c->tune = saved_table;
    if (rc != EIS_OK) {
        apply(prev);
        return rc;
    }
    apply(best);
    out->ctas_per_sm = best.ctas > 0 ? best.ctas : occ;
    out->giant_threshold = best.thr;
    out->giant_stride = c->giant_stride;
    out->ms_best = ms_best;
    out->ms_default = ms_prev;
    out->trials = trials;
    out->giant_kernel = best.kernel;
    out->mark_every = c->mark_every;
    out->bsgs_chunk = best.chunk;
    return EIS_OK;
}

int eis_count_range(eis_ctx *c, uint64_t lo, uint64_t hi, uint64_t *count_out) {
    if (!c || !count_out) return EIS_EINVAL;
    eis_stats acc{};
    int rc = run_chunks(c, lo, hi, 0, c->stream, &acc, [](eis_plan *, uint64_t) { return EIS_OK; });
    if (rc != EIS_OK) return rc;
    c->last = acc;
    *count_out = acc.in_E;
    return EIS_OK;
}

int eis_classify_range(eis_ctx *c, uint64_t lo, uint64_t hi, uint32_t *flags_out,
                       uint32_t *sqfree_out, int out_on_device, uint64_t *count_out,
                       void *stream) {
    if (!c) return EIS_EINVAL;
    cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
    const cudaMemcpyKind kind = out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    eis_stats acc{};
    int rc = run_chunks(c, lo, hi, 0, s, &acc, [&](eis_plan *p, uint64_t off) -> int {
        const uint64_t w0 = off / 32;
        if (flags_out && p->nwords)
            EIS_CK(cudaMemcpyAsync(flags_out + w0, p->d_flags, p->nwords * 4, kind, s));
        if (sqfree_out && p->nwords)
            EIS_CK(cudaMemcpyAsync(sqfree_out + w0, p->d_sqfree, p->nwords * 4, kind, s));
        EIS_CK(cudaStreamSynchronize(s));
        return EIS_OK;
    });
    if (rc != EIS_OK) return rc;
    c->last = acc;
    if (count_out) *count_out = acc.in_E;
    return EIS_OK;
}

int eis_classify_range_u8(eis_ctx *c, uint64_t lo, uint64_t hi, uint8_t *codes_out,
                          int out_on_device, uint64_t *count_out, void *stream) {
    if (!c || !codes_out) return EIS_EINVAL;
    cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
    const cudaMemcpyKind kind = out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    uint64_t d0;
    const uint64_t ntot = num_candidates(lo, hi, &d0);
    eis_stats acc{};
    int rc = run_chunks(c, lo, hi, 1, s, &acc, [&](eis_plan *p, uint64_t off) -> int {
        const uint64_t n = std::min<uint64_t>(p->total_cand, ntot - off);
        if (n == 0) return EIS_OK;
        uint8_t *tmp = out_on_device ? codes_out + off : nullptr;
        if (!tmp) {
            if (cudaMalloc(&tmp, n) != cudaSuccess) {
                cudaGetLastError();
                return EIS_ENOMEM;
            }
        }
        const uint32_t grid = (uint32_t)std::min<uint64_t>((n + 255) / 256, 65535ull * 8);
        k_expand_codes<<<grid, 256, 0, s>>>(p->d_flags, p->d_sqfree, n, tmp);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess && !out_on_device)
            e = cudaMemcpyAsync(codes_out + off, tmp, n, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (!out_on_device) cudaFree(tmp);
        (void)kind;
        return e == cudaSuccess ? EIS_OK : EIS_EDEVICE;
    });
    if (rc != EIS_OK) return rc;
    c->last = acc;
    if (count_out) *count_out = acc.in_E;
    return EIS_OK;
}

int eis_classify_range_log(eis_ctx *c, uint64_t lo, uint64_t hi, uint8_t *log_out,
                           int out_on_device, void *stream) {
    if (!c || !log_out) return EIS_EINVAL;
    cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
    const cudaMemcpyKind kind = out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    uint64_t d0;
    const uint64_t ntot = num_candidates(lo, hi, &d0);
    eis_stats acc{};
    int rc = run_chunks(c, lo, hi, 1, s, &acc, [&](eis_plan *p, uint64_t off) -> int {
        const uint64_t n = std::min<uint64_t>(p->total_cand, ntot - off);
        if (n) EIS_CK(cudaMemcpyAsync(log_out + off, p->d_glog, n, kind, s));
        EIS_CK(cudaStreamSynchronize(s));
        return EIS_OK;
    });
    if (rc != EIS_OK) return rc;
    c->last = acc;
    return EIS_OK;
}

int eis_is_eisenstein(eis_ctx *c, uint64_t d, int *result_out) {
    EisNvtxRange range("eis.is_eisenstein");
    if (!c || !result_out) return EIS_EINVAL;
    if (d >= EIS_D_LIMIT) return EIS_ERANGE;
    if (d % 8 != 5) return EIS_ENOTD;
    EIS_CK(cudaSetDevice(c->device));
    const uint32_t limit = (uint32_t)std::min<int64_t>(c->step_limit, 0xffffffffll);
    std::memset(&c->last, 0, sizeof(c->last));
    c->last.candidates = 1;
    int res = 0;  // 0: not in D, else 1 + log eps_d
    // square-free test by the whole GPU (d_query[40], 0 = square-free)
    unsigned char *q = c->d_query;  // [0] d, [8] out, [12] status, [16] acc[2], [32] next, [40] flag
    uint32_t *sq_flag = reinterpret_cast<uint32_t *>(q + 40);
    EIS_CK(cudaMemsetAsync(q, 0, 64, c->stream));
    {
        // only odd primes with p^2 <= d can divide d: scan those, on as many
        // blocks as they fill (at most two per SM)
        uint64_t r = (uint64_t)std::sqrt((double)d);
        while (r * r > d) --r;
        while ((r + 1) * (r + 1) <= d) ++r;
        const uint32_t np = (uint32_t)(std::upper_bound(c->primes.begin(), c->primes.end(),
                                                        (uint32_t)std::min<uint64_t>(r, UINT32_MAX)) -
                                       c->primes.begin());
        const uint32_t blocks = std::max<uint32_t>(1u, std::min<uint32_t>((np + 255) / 256,
                                                                          (uint32_t)c->sm_count * 2));
        k_sqfree_one<<<blocks, 256, 0, c->stream>>>(d, c->d_sqtab, np, sq_flag);
    }
    EIS_CK(cudaGetLastError());
    if (c->mode == EIS_MODE_PLAIN) {
        // one lane walks the half period
        EIS_CK(cudaMemsetAsync(c->d_single, 0, 4 * sizeof(int), c->stream));
        k_walk_single<<<1, 32, 0, c->stream>>>(d, c->d_primes, c->d_sqtab, c->nprimes, c->d_single,
                                               c->d_single + 2, limit, sq_flag);
        EIS_CK(cudaGetLastError());
        int h[4] = {0, 0, 0, 0};
        EIS_CK(cudaMemcpyAsync(h, c->d_single, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
        EIS_CK(cudaStreamSynchronize(c->stream));
        if (h[2] & kErrSteps) return EIS_ESTEPS;
        c->last.baby_steps = (uint64_t)h[1];
        res = h[0];
    } else {
        // one warp: baby steps into a shared-memory table, 32 lanes of giant steps
        int nbaby, log2n;
        giant_params(d, c->giant_stride, nbaby, log2n);
        log2n = std::min(log2n, kGiantMaxLog2);
        EIS_CK(cudaMemcpyAsync(q, &d, sizeof(d), cudaMemcpyHostToDevice, c->stream));
        k_giant<<<1, 32, (size_t)8 << log2n, c->stream>>>(
            reinterpret_cast<const uint64_t *>(q), nullptr, 0, nullptr, nullptr, 1,
            reinterpret_cast<uint32_t *>(q + 32), c->d_primes, c->d_sqtab, c->nprimes,
            reinterpret_cast<int8_t *>(q + 8), nullptr, nullptr,
            reinterpret_cast<unsigned long long *>(q + 16), reinterpret_cast<int *>(q + 12), nbaby,
            log2n, kGiantMaxRounds, c->giant_compose, sq_flag);
        EIS_CK(cudaGetLastError());
        unsigned char h[64];
        EIS_CK(cudaMemcpyAsync(h, q, 64, cudaMemcpyDeviceToHost, c->stream));
        EIS_CK(cudaStreamSynchronize(c->stream));
        int status = 0;
        int8_t out = 0;
        unsigned long long acc[2] = {0, 0};
        std::memcpy(&out, h + 8, 1);
        std::memcpy(&status, h + 12, sizeof(int));
        std::memcpy(acc, h + 16, sizeof(acc));
        if ((status & kErrGiant) || out < 0) return EIS_ESTEPS;
        c->last.baby_steps = acc[0];
        c->last.giant_steps = acc[1];
        res = out;
    }
    if (res == 0) return EIS_ENOTD;
    c->last.in_D = 1;
    c->last.in_E = (res == 1);
    *result_out = (res == 1) ? 1 : 0;
    return EIS_OK;
}

int eis_count_batch(eis_ctx *c, const uint64_t *lo, const uint64_t *hi, size_t n,
                    uint64_t *counts_out) {
    if (!c || (n && (!lo || !hi || !counts_out))) return EIS_EINVAL;
    for (size_t i = 0; i < n; ++i) {
        if (lo[i] > hi[i]) return EIS_EINVAL;
        if (hi[i] > EIS_D_LIMIT) return EIS_ERANGE;
    }
    const uint64_t M = max_chunk_cands(c, 0);
    if (M == 0) return EIS_ENOMEM;
    eis_stats acc{};
    // Group intervals into plans of at most M candidates; an interval larger
    // than M is counted on its own in chunks.
    size_t i = 0;
    while (i < n) {
        std::vector<uint64_t> glo, ghi;
        std::vector<size_t> gidx;
        uint64_t tot = 0;
        while (i < n) {
            uint64_t d0;
            const uint64_t nc = (num_candidates(lo[i], hi[i], &d0) + 31) / 32 * 32;
            if (nc > M) {
                if (!gidx.empty()) break;
                uint64_t v = 0;
                int rc = eis_count_range(c, lo[i], hi[i], &v);
                if (rc != EIS_OK) return rc;
                counts_out[i] = v;
                const eis_stats st = c->last;
                acc.candidates += st.candidates;
                acc.in_D += st.in_D;
                acc.in_E += st.in_E;
                acc.baby_steps += st.baby_steps;
                acc.ms_total += st.ms_total;
                acc.ms_walk += st.ms_walk;
                acc.ms_sieve += st.ms_sieve;
                acc.launches += st.launches;
                ++i;
                continue;
            }
            if (tot + nc > M) break;
            tot += nc;
            glo.push_back(lo[i]);
            ghi.push_back(hi[i]);
            gidx.push_back(i);
            ++i;
        }
        if (gidx.empty()) continue;
        eis_plan *p = nullptr;
        int rc = plan_build(c, glo.data(), ghi.data(), glo.size(), c->mode, 0, &p);
        if (rc != EIS_OK) return rc;
        rc = plan_launch(p, c->stream);
        std::vector<uint64_t> cnt(gidx.size());
        eis_stats st{};
        if (rc == EIS_OK) rc = plan_counts_user(p, cnt.data());
        if (rc == EIS_OK) rc = plan_fill_stats(p, &st);
        plan_free(p);
        if (rc != EIS_OK) return rc;
        for (size_t k = 0; k < gidx.size(); ++k) counts_out[gidx[k]] = cnt[k];
        acc.candidates += st.candidates;
        acc.in_D += st.in_D;
        acc.in_E += st.in_E;
        acc.baby_steps += st.baby_steps;
        acc.ms_total += st.ms_total;
        acc.ms_walk += st.ms_walk;
        acc.ms_sieve += st.ms_sieve;
        acc.launches += st.launches;
        acc.sm_count = st.sm_count;
    }
    c->last = acc;
    return EIS_OK;
}

}  // extern "C"
