// eis_serve.cu -- continuous-batching request server over the classification
// pipeline.
//
// Requests are range counts #E cap [lo, hi) and membership queries "is d in
// E".  A dispatcher thread owns `slots` batch slots; each slot has its own
// stream, device buffers sized once at creation (its memory share of the
// context budget) and pinned host tables.  Whenever a slot is free the
// dispatcher packs as many queued request parts as fit (candidates and
// segment count) into one batch and launches the whole pipeline -- sieve,
// compaction, persistent walk, count -- on the slot's stream.  Requests that
// arrive while batches run queue on the host and go out in the next free
// slot, so up to `slots` batches overlap on the device: a persistent walk
// CTA exits as soon as its lanes run out of work, and the next batch's CTAs
// take its SMs.  A membership query is a one-candidate segment [d, d+1).
// Completion is detected with cudaEventQuery; every wait on the host has a
// timeout (EIS_ETIMEOUT).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "eis.h"
#include "eis_internal.h"
#include "eis_kernels.h"

using namespace eis;
using Clock = std::chrono::steady_clock;

namespace {

struct Part {
    uint64_t req;
    uint64_t lo, hi;  // half-open, at most slot_candidates candidates
    uint64_t ncand;
    uint64_t d0;
    bool member;      // a single d answered by the giant-step kernel
};

struct Request {
    int kind = EIS_REQ_COUNT;
    uint32_t parts_left = 0;
    uint64_t sumE = 0, sumD = 0;
    int status = EIS_OK;
    bool done = false;
    bool cancelled = false;
    Clock::time_point t_submit, t_done;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done_ev = nullptr;
    // device
    Seg *d_segs = nullptr;
    Tile *d_tiles = nullptr;
    uint32_t *d_sqfree = nullptr, *d_flags = nullptr, *d_tile_pop = nullptr, *d_tile_off = nullptr;
    uint32_t *d_surv = nullptr, *d_ctr = nullptr;
    int *d_status = nullptr;
    unsigned long long *d_counts = nullptr, *d_steps = nullptr;
    // pinned host
    Seg *h_segs = nullptr;
    Tile *h_tiles = nullptr;
    unsigned long long *h_counts = nullptr;
    int *h_status = nullptr;
    uint32_t *h_ctr = nullptr;   // the batch's counters: [2] walks handed to k_giant
    // membership queries of the batch (one warp each in k_giant)
    uint64_t *d_mem_d = nullptr, *h_mem_d = nullptr;
    int8_t *d_mem_out = nullptr, *h_mem_out = nullptr;
    unsigned char *d_mem_ctl = nullptr;  // [0] next, [8] acc[2], [24] status
    uint32_t *d_defer = nullptr;         // long walks handed to k_giant
    std::vector<Part> items;     // range segments
    std::vector<Part> members;   // membership queries
    bool busy = false;
};

}  // namespace

struct eis_server {
    eis_ctx *ctx = nullptr;
    eis_server_config cfg{};
    std::vector<Slot> slots;
    uint32_t max_tiles = 0;
    uint32_t grid = 0;
    uint32_t giant_grid = 0;
    uint32_t step_limit = 1u << 26;
    // walks longer than this many baby steps go to the giant-step kernel, which
    // finishes one long walk far sooner than a single lane (0: never)
    uint32_t defer_after = 131072;  // from eis_server_config.giant_after
    uint32_t defer_cap = 0;
    std::mutex mu;
    std::condition_variable cv_work;  // dispatcher: new parts or stop
    std::condition_variable cv_done;  // waiters: a request finished
    std::deque<Part> pending;
    std::unordered_map<uint64_t, Request> reqs;
    uint64_t next_id = 1;
    bool stop = false;
    std::thread th;
    eis_server_counters st{};
    bool failed = false;
    uint32_t fail_left = 0;  // eis_server_config.fail_launches still to fake
};

namespace {

int slot_alloc(eis_server *s, Slot &sl) {
    const uint64_t M = s->cfg.slot_candidates;
    const uint32_t S = s->cfg.slot_requests;
    const uint64_t words = M / 32 + S + 1;  // each segment padded to whole words
    const uint64_t cands = words * 32;
    if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.done_ev, cudaEventDisableTiming) != cudaSuccess)
        return EIS_EDEVICE;
    bool ok = cudaMalloc(&sl.d_segs, S * sizeof(Seg)) == cudaSuccess &&
              cudaMalloc(&sl.d_tiles, s->max_tiles * sizeof(Tile)) == cudaSuccess &&
              cudaMalloc(&sl.d_sqfree, words * 4) == cudaSuccess &&
              cudaMalloc(&sl.d_flags, words * 4) == cudaSuccess &&
              cudaMalloc(&sl.d_tile_pop, s->max_tiles * 4) == cudaSuccess &&
              cudaMalloc(&sl.d_tile_off, s->max_tiles * 4) == cudaSuccess &&
              cudaMalloc(&sl.d_surv, cands * 4) == cudaSuccess &&
              cudaMalloc(&sl.d_ctr, 16) == cudaSuccess &&
              cudaMalloc(&sl.d_status, sizeof(int)) == cudaSuccess &&
              cudaMalloc(&sl.d_counts, (2 * S + 1) * sizeof(unsigned long long)) == cudaSuccess &&
              cudaMalloc(&sl.d_steps, 4 * sizeof(unsigned long long)) == cudaSuccess &&
              cudaHostAlloc(&sl.h_segs, S * sizeof(Seg), cudaHostAllocDefault) == cudaSuccess &&
              cudaHostAlloc(&sl.h_tiles, s->max_tiles * sizeof(Tile), cudaHostAllocDefault) == cudaSuccess &&
              cudaHostAlloc(&sl.h_counts, (2 * S + 1) * sizeof(unsigned long long), cudaHostAllocDefault) == cudaSuccess &&
              cudaHostAlloc(&sl.h_status, sizeof(int), cudaHostAllocDefault) == cudaSuccess &&
              cudaHostAlloc(&sl.h_ctr, 16, cudaHostAllocDefault) == cudaSuccess &&
              cudaMalloc(&sl.d_mem_d, S * sizeof(uint64_t)) == cudaSuccess &&
              cudaMalloc(&sl.d_mem_out, S) == cudaSuccess &&
              cudaMalloc(&sl.d_mem_ctl, 64) == cudaSuccess &&
              cudaMalloc(&sl.d_defer, (size_t)s->defer_cap * 4 + 4) == cudaSuccess &&
              cudaHostAlloc(&sl.h_mem_d, S * sizeof(uint64_t), cudaHostAllocDefault) == cudaSuccess &&
              cudaHostAlloc(&sl.h_mem_out, S, cudaHostAllocDefault) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        return EIS_ENOMEM;
    }
    return EIS_OK;
}

void slot_free(Slot &sl) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    void *dev[] = {sl.d_segs, sl.d_tiles, sl.d_sqfree, sl.d_flags, sl.d_tile_pop, sl.d_tile_off,
                   sl.d_surv, sl.d_ctr, sl.d_status, sl.d_counts, sl.d_steps,
                   sl.d_mem_d, sl.d_mem_out, sl.d_mem_ctl, sl.d_defer};
    for (void *p : dev)
        if (p) cudaFree(p);
    void *host[] = {sl.h_segs, sl.h_tiles, sl.h_counts, sl.h_status, sl.h_ctr, sl.h_mem_d,
                    sl.h_mem_out};
    for (void *p : host)
        if (p) cudaFreeHost(p);
    if (sl.done_ev) cudaEventDestroy(sl.done_ev);
    if (sl.stream) cudaStreamDestroy(sl.stream);
}

uint64_t slot_bytes(const eis_server_config &c, uint32_t max_tiles, uint32_t defer_cap) {
    const uint64_t words = c.slot_candidates / 32 + c.slot_requests + 1;
    return words * 4 * 2 + words * 32 * 4 + (uint64_t)defer_cap * 4 +
           (uint64_t)max_tiles * (sizeof(Tile) + 8) +
           (uint64_t)c.slot_requests * (sizeof(Seg) + 16 + 9) + 320;
}

// Launch one batch (the slot's items) on the slot's stream.  False when any
// call fails; the batch's results are then not to be read.
bool launch_batch(eis_server *s, Slot &sl) {
    EisNvtxRange range("eis.server.batch");
    if (s->fail_left > 0) {  // test hook: fail before anything is enqueued
        --s->fail_left;
        return false;
    }
    eis_ctx_view cv = eis_ctx_get_view(s->ctx);
    bool ok = true;
    auto ck = [&ok](cudaError_t e) { ok &= (e == cudaSuccess); };
    std::sort(sl.items.begin(), sl.items.end(),
              [](const Part &a, const Part &b) { return a.d0 < b.d0; });
    uint64_t cur = 0;
    uint32_t nt = 0;
    for (size_t i = 0; i < sl.items.size(); ++i) {
        const Part &p = sl.items[i];
        sl.h_segs[i] = Seg{p.d0, p.ncand, cur};
        for (uint64_t off = 0; off < p.ncand; off += kTileCands)
            sl.h_tiles[nt++] = Tile{cur + off, (uint32_t)i,
                                    (uint32_t)std::min<uint64_t>(kTileCands, p.ncand - off)};
        cur += (p.ncand + 31) / 32 * 32;
    }
    const uint32_t nseg = (uint32_t)sl.items.size();
    const uint64_t nwords = cur / 32;
    cudaStream_t st = sl.stream;
    ck(cudaMemcpyAsync(sl.d_segs, sl.h_segs, nseg * sizeof(Seg), cudaMemcpyHostToDevice, st));
    ck(cudaMemcpyAsync(sl.d_tiles, sl.h_tiles, nt * sizeof(Tile), cudaMemcpyHostToDevice, st));
    ck(cudaMemsetAsync(sl.d_flags, 0, nwords * 4 + 4, st));
    ck(cudaMemsetAsync(sl.d_ctr, 0, 16, st));
    ck(cudaMemsetAsync(sl.d_status, 0, sizeof(int), st));
    ck(cudaMemsetAsync(sl.d_counts, 0, (2 * nseg + 1) * sizeof(unsigned long long), st));
    ck(cudaMemsetAsync(sl.d_steps, 0, 4 * sizeof(unsigned long long), st));
    uint64_t dmax = 0;
    for (const Part &p : sl.items) dmax = std::max(dmax, p.d0 + 8 * (p.ncand - 1));
    if (nt > 0) {
        k_sieve<<<nt, 256, 0, st>>>(sl.d_tiles, sl.d_segs, cv.d_primes, cv.nprimes, sl.d_sqfree,
                                    sl.d_tile_pop, 0);
        k_scan_tiles<<<1, 1024, 0, st>>>(sl.d_tile_pop, sl.d_tile_off, nt, sl.d_ctr);
        k_compact<<<nt, 256, 0, st>>>(sl.d_tiles, sl.d_sqfree, sl.d_tile_off, sl.d_surv);
        k_walk_persistent<<<s->grid, 256, 0, st>>>(sl.d_segs, nseg, sl.d_surv, sl.d_ctr,
                                                   sl.d_ctr + 1, sl.d_flags, nullptr, sl.d_steps,
                                                   sl.d_status, s->step_limit, s->defer_after,
                                                   sl.d_defer, sl.d_ctr + 2, s->defer_cap,
                                                   dmax < kFastDLimit ? 1 : 0);
        if (s->defer_after) {
            int nbaby, log2n;
            eis_giant_params(dmax, 0, nbaby, log2n);
            k_giant<<<s->giant_grid, 32, (size_t)8 << log2n, st>>>(
                nullptr, sl.d_segs, nseg, sl.d_defer, sl.d_ctr + 2, s->defer_cap, sl.d_ctr + 3,
                cv.d_primes, cv.d_sqtab, cv.nprimes, nullptr, sl.d_flags, nullptr, sl.d_steps + 1,
                sl.d_status, nbaby, log2n, 1u << 20, cv.giant_compose, nullptr);
        }
        k_count<<<nt, 256, 0, st>>>(sl.d_tiles, sl.d_flags, sl.d_sqfree, sl.d_counts, nullptr,
                                    nullptr);
    }
    const uint32_t nmem = (uint32_t)sl.members.size();
    if (nmem > 0) {
        uint64_t dmax = 0;
        for (uint32_t i = 0; i < nmem; ++i) {
            sl.h_mem_d[i] = sl.members[i].d0;
            dmax = std::max(dmax, sl.members[i].d0);
        }
        int nbaby, log2n;
        eis_giant_params(dmax, 0, nbaby, log2n);
        ck(cudaMemcpyAsync(sl.d_mem_d, sl.h_mem_d, nmem * sizeof(uint64_t), cudaMemcpyHostToDevice,
                           st));
        ck(cudaMemsetAsync(sl.d_mem_ctl, 0, 64, st));
        k_giant<<<std::min<uint32_t>(nmem, s->giant_grid), 32, (size_t)8 << log2n, st>>>(
            sl.d_mem_d, nullptr, 0, nullptr, nullptr, nmem,
            reinterpret_cast<uint32_t *>(sl.d_mem_ctl), cv.d_primes, cv.d_sqtab, cv.nprimes,
            sl.d_mem_out,
            nullptr, nullptr, reinterpret_cast<unsigned long long *>(sl.d_mem_ctl + 8),
            reinterpret_cast<int *>(sl.d_mem_ctl + 24), nbaby, log2n, 1u << 20, cv.giant_compose,
            nullptr);
        ck(cudaGetLastError());
        ck(cudaMemcpyAsync(sl.h_mem_out, sl.d_mem_out, nmem, cudaMemcpyDeviceToHost, st));
    }
    ck(cudaGetLastError());
    ck(cudaMemcpyAsync(sl.h_counts, sl.d_counts, 2 * nseg * sizeof(unsigned long long),
                       cudaMemcpyDeviceToHost, st));
    ck(cudaMemcpyAsync(sl.h_status, sl.d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    ck(cudaMemcpyAsync(sl.h_ctr, sl.d_ctr, 16, cudaMemcpyDeviceToHost, st));
    ck(cudaEventRecord(sl.done_ev, st));
    return ok;
}

void finish_request(eis_server *s, uint64_t id, Request &r) {
    r.done = true;
    r.t_done = Clock::now();
    if (r.status == EIS_OK && r.kind == EIS_REQ_MEMBER && r.sumD == 0) r.status = EIS_ENOTD;
    s->st.requests_done++;
    (void)id;
}

// A batch that could not be launched: every request part it held completes
// with EIS_EDEVICE (its counts were never written), and the slot is left
// idle.  Called with s->mu held.
void fail_batch(eis_server *s, Slot &sl) {
    for (const std::vector<Part> *v : {&sl.items, &sl.members}) {
        for (const Part &p : *v) {
            auto it = s->reqs.find(p.req);
            if (it == s->reqs.end()) continue;
            Request &r = it->second;
            if (r.status == EIS_OK) r.status = EIS_EDEVICE;
            if (--r.parts_left == 0) finish_request(s, it->first, r);
        }
    }
    sl.items.clear();
    sl.members.clear();
    sl.busy = false;
    s->failed = true;
}

void dispatcher(eis_server *s) {
    cudaSetDevice(eis_ctx_get_view(s->ctx).device);
    for (;;) {
        bool progressed = false;
        // 1. completed batches
        for (Slot &sl : s->slots) {
            if (!sl.busy) continue;
            cudaError_t q = cudaEventQuery(sl.done_ev);
            if (q == cudaErrorNotReady) continue;
            std::lock_guard<std::mutex> lk(s->mu);
            const int bstatus = (q != cudaSuccess) ? EIS_EDEVICE
                                : ((*sl.h_status & (kErrSteps | kErrGiant)) ? EIS_ESTEPS : EIS_OK);
            if (q != cudaSuccess) s->failed = true;
            if (q == cudaSuccess && s->defer_after && !sl.items.empty())
                s->st.deferred += std::min(sl.h_ctr[2], s->defer_cap);
            for (size_t i = 0; i < sl.items.size(); ++i) {
                auto it = s->reqs.find(sl.items[i].req);
                if (it == s->reqs.end()) continue;
                Request &r = it->second;
                r.sumE += sl.h_counts[2 * i];
                r.sumD += sl.h_counts[2 * i + 1];
                if (bstatus != EIS_OK && r.status == EIS_OK) r.status = bstatus;
                if (--r.parts_left == 0) finish_request(s, it->first, r);
            }
            for (size_t i = 0; i < sl.members.size(); ++i) {
                auto it = s->reqs.find(sl.members[i].req);
                if (it == s->reqs.end()) continue;
                Request &r = it->second;
                const int8_t o = sl.h_mem_out[i];
                if (q != cudaSuccess) {
                    if (r.status == EIS_OK) r.status = EIS_EDEVICE;
                } else if (o < 0) {
                    if (r.status == EIS_OK) r.status = EIS_ESTEPS;
                } else if (o > 0) {
                    r.sumD += 1;
                    r.sumE += (o == 1);
                }
                if (--r.parts_left == 0) finish_request(s, it->first, r);
            }
            sl.items.clear();
            sl.members.clear();
            sl.busy = false;
            progressed = true;
            s->cv_done.notify_all();
        }
        // 2. dispatch queued parts into free slots
        for (Slot &sl : s->slots) {
            if (sl.busy) continue;
            {
                std::lock_guard<std::mutex> lk(s->mu);
                if (s->pending.empty() || s->failed) break;
                uint64_t cand = 0;
                uint32_t tiles = 0;
                while (!s->pending.empty() && sl.items.size() < s->cfg.slot_requests &&
                       sl.members.size() < s->cfg.slot_requests) {
                    const Part &p = s->pending.front();
                    if (p.member) {
                        auto itm = s->reqs.find(p.req);
                        if (itm != s->reqs.end() && itm->second.cancelled) {
                            if (--itm->second.parts_left == 0) finish_request(s, itm->first, itm->second);
                        } else {
                            sl.members.push_back(p);
                        }
                        s->pending.pop_front();
                        continue;
                    }
                    const uint64_t c = (p.ncand + 31) / 32 * 32;
                    const uint32_t t = (uint32_t)((p.ncand + kTileCands - 1) / kTileCands);
                    if (!sl.items.empty() &&
                        (cand + c > s->cfg.slot_candidates || tiles + t > s->max_tiles))
                        break;
                    auto it = s->reqs.find(p.req);
                    if (it != s->reqs.end() && it->second.cancelled) {
                        // cancelled before dispatch: count the part as done
                        Request &r = it->second;
                        if (--r.parts_left == 0) finish_request(s, it->first, r);
                        s->pending.pop_front();
                        continue;
                    }
                    cand += c;
                    tiles += t;
                    sl.items.push_back(p);
                    s->pending.pop_front();
                }
                if (sl.items.empty() && sl.members.empty()) continue;
                s->st.batches++;
                s->st.parts += sl.items.size() + sl.members.size();
                s->st.max_batch_parts = std::max<uint64_t>(s->st.max_batch_parts,
                                                           sl.items.size() + sl.members.size());
            }
            progressed = true;
            if (!launch_batch(s, sl)) {
                std::lock_guard<std::mutex> lk(s->mu);
                fail_batch(s, sl);
                s->cv_done.notify_all();
                continue;
            }
            sl.busy = true;
        }
        {
            std::unique_lock<std::mutex> lk(s->mu);
            bool any_busy = false;
            for (Slot &sl : s->slots) any_busy |= sl.busy;
            if (s->stop && s->pending.empty() && !any_busy) break;
            if (s->failed) {
                // fail everything still queued; in-flight batches finish above
                while (!s->pending.empty()) {
                    const Part p = s->pending.front();
                    s->pending.pop_front();
                    auto it = s->reqs.find(p.req);
                    if (it == s->reqs.end()) continue;
                    it->second.status = EIS_EDEVICE;
                    if (--it->second.parts_left == 0) finish_request(s, it->first, it->second);
                }
                s->cv_done.notify_all();
            }
            if (!progressed) {
                if (any_busy)
                    s->cv_work.wait_for(lk, std::chrono::microseconds(20));
                else
                    s->cv_work.wait_for(lk, std::chrono::milliseconds(5));
            }
        }
    }
}

}  // namespace

extern "C" {

int eis_server_create(eis_ctx *ctx, const eis_server_config *cfg, eis_server **out) {
    if (!ctx || !out) return EIS_EINVAL;
    *out = nullptr;
    eis_server_config c{};
    c.slots = 4;
    c.slot_candidates = (uint64_t)1 << 22;
    c.slot_requests = 4096;
    c.max_pending = 1u << 20;
    if (cfg) {
        if (cfg->slots) c.slots = cfg->slots;
        if (cfg->slot_candidates) c.slot_candidates = cfg->slot_candidates;
        if (cfg->slot_requests) c.slot_requests = cfg->slot_requests;
        if (cfg->max_pending) c.max_pending = cfg->max_pending;
        c.giant_after = cfg->giant_after;
        c.giant_max = cfg->giant_max;
        c.fail_launches = cfg->fail_launches;
    }
    if (c.giant_after == 0) c.giant_after = 131072;
    if (c.slots > 64 || c.slot_candidates < 64 || c.slot_candidates > ((uint64_t)1 << 30) ||
        c.slot_requests < 1)
        return EIS_EINVAL;
    c.slot_candidates = (c.slot_candidates + 31) / 32 * 32;
    eis_ctx_view v = eis_ctx_get_view(ctx);
    if (cudaSetDevice(v.device) != cudaSuccess) return EIS_EDEVICE;
    eis_server *s = new eis_server();
    s->ctx = ctx;
    s->cfg = c;
    s->max_tiles = (uint32_t)(c.slot_candidates / kTileCands) + c.slot_requests + 1;
    s->grid = v.walk_grid;
    s->giant_grid = v.giant_grid;
    s->defer_after = c.giant_after == 0xffffffffu ? 0u : c.giant_after;
    s->fail_left = c.fail_launches;
    s->step_limit = v.step_limit;
    // At most giant_max walks of a batch go to the giant-step kernel (default:
    // an eighth of a slot, in practice every walk past giant_after; capping
    // lower measured no better at p99).
    s->defer_cap = c.giant_max ? c.giant_max
                               : (uint32_t)std::max<uint64_t>(1024, c.slot_candidates / 8);
    const uint64_t need = slot_bytes(c, s->max_tiles, s->defer_cap) * c.slots;
    if (!eis_ctx_reserve(ctx, need)) {
        delete s;
        return EIS_ENOMEM;
    }
    s->st.reserved_bytes = need;
    s->slots.resize(c.slots);
    for (Slot &sl : s->slots) {
        int rc = slot_alloc(s, sl);
        if (rc != EIS_OK) {
            for (Slot &x : s->slots) slot_free(x);
            eis_ctx_release(ctx, need);
            delete s;
            return rc;
        }
    }
    s->th = std::thread(dispatcher, s);
    *out = s;
    return EIS_OK;
}

int eis_server_submit(eis_server *s, int kind, uint64_t lo, uint64_t hi, uint64_t *id_out) {
    if (!s || !id_out) return EIS_EINVAL;
    if (kind == EIS_REQ_MEMBER) hi = lo + 1;
    else if (kind != EIS_REQ_COUNT) return EIS_EINVAL;
    if (lo > hi) return EIS_EINVAL;
    if (hi > EIS_D_LIMIT) return EIS_ERANGE;
    std::vector<Part> parts;
    uint64_t d0 = lo + ((13 - lo % 8) % 8);
    const uint64_t n = hi > d0 ? (hi - d0 + 7) / 8 : 0;
    const uint64_t M = s->cfg.slot_candidates;
    for (uint64_t off = 0; off < n; off += M) {
        const uint64_t a = d0 + 8 * off;
        const uint64_t b = std::min(hi, d0 + 8 * (off + M));
        parts.push_back(Part{0, a, b, std::min<uint64_t>(M, n - off), a, kind == EIS_REQ_MEMBER});
    }
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return EIS_EINVAL;
    if (s->pending.size() + parts.size() > s->cfg.max_pending) {
        s->st.rejected++;
        return EIS_EBUSY;
    }
    const uint64_t id = s->next_id++;
    Request &r = s->reqs[id];
    r.kind = kind;
    r.t_submit = Clock::now();
    r.parts_left = (uint32_t)parts.size();
    s->st.requests_submitted++;
    if (kind == EIS_REQ_MEMBER && lo % 8 != 5) {
        r.status = EIS_ENOTD;
        r.parts_left = 0;
    }
    if (r.parts_left == 0) {
        finish_request(s, id, r);
        s->cv_done.notify_all();
    } else {
        for (Part &p : parts) {
            p.req = id;
            s->pending.push_back(p);
        }
        s->cv_work.notify_one();
    }
    *id_out = id;
    return EIS_OK;
}

int eis_server_poll(eis_server *s, uint64_t id, int *done_out) {
    if (!s || !done_out) return EIS_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return EIS_ENOTFOUND;
    *done_out = it->second.done ? 1 : 0;
    return EIS_OK;
}

int eis_server_wait(eis_server *s, uint64_t id, double timeout_ms, uint64_t *result_out,
                    double *latency_us_out) {
    if (!s) return EIS_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return EIS_ENOTFOUND;
    const auto deadline = Clock::now() + std::chrono::microseconds((int64_t)(timeout_ms * 1e3));
    while (!it->second.done) {
        if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && !it->second.done)
            return EIS_ETIMEOUT;
        it = s->reqs.find(id);
        if (it == s->reqs.end()) return EIS_ENOTFOUND;
    }
    Request r = it->second;
    s->reqs.erase(it);
    if (result_out) *result_out = r.sumE;
    if (latency_us_out)
        *latency_us_out = std::chrono::duration<double, std::micro>(r.t_done - r.t_submit).count();
    return r.status;
}

int eis_server_cancel(eis_server *s, uint64_t id) {
    if (!s) return EIS_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return EIS_ENOTFOUND;
    if (!it->second.done) {
        it->second.cancelled = true;
        it->second.status = EIS_ECANCELED;
    }
    return EIS_OK;
}

int eis_server_stats(eis_server *s, eis_server_counters *out) {
    if (!s || !out) return EIS_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->st;
    out->pending_parts = s->pending.size();
    return EIS_OK;
}

int eis_server_destroy(eis_server *s) {
    if (!s) return EIS_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->th.joinable()) s->th.join();
    for (Slot &sl : s->slots) slot_free(sl);
    eis_ctx_release(s->ctx, s->st.reserved_bytes);
    delete s;
    return EIS_OK;
}

int eis_server_replay(eis_server *s, size_t n, const double *t_arrival_s, const int *kind,
                      const uint64_t *lo, const uint64_t *hi, uint64_t *results_out,
                      int *status_out, double *latency_us_out, double *wall_s_out) {
    if (!s || (n && (!t_arrival_s || !kind || !lo || !hi))) return EIS_EINVAL;
    std::vector<uint64_t> ids(n, 0);
    std::vector<int> sub_rc(n, EIS_OK);
    std::vector<Clock::time_point> t_arr(n);
    const Clock::time_point t0 = Clock::now();
    std::atomic<size_t> submitted{0};
    // Client: submit each request at its arrival time.
    std::thread client([&] {
        for (size_t i = 0; i < n; ++i) {
            const auto due = t0 + std::chrono::nanoseconds((int64_t)(t_arrival_s[i] * 1e9));
            while (Clock::now() < due) {
                const auto left = due - Clock::now();
                if (left > std::chrono::microseconds(200))
                    std::this_thread::sleep_for(left - std::chrono::microseconds(100));
            }
            t_arr[i] = due;
            uint64_t id = 0;
            int rc;
            do {
                rc = eis_server_submit(s, kind[i], lo[i], hi[i], &id);
                if (rc == EIS_EBUSY) std::this_thread::sleep_for(std::chrono::microseconds(50));
            } while (rc == EIS_EBUSY);
            sub_rc[i] = rc;
            ids[i] = id;
            submitted.store(i + 1, std::memory_order_release);
        }
    });
    // Collector: wait for each request in order (latency = done - arrival).
    int first_err = EIS_OK;
    for (size_t i = 0; i < n; ++i) {
        while (submitted.load(std::memory_order_acquire) <= i)
            std::this_thread::sleep_for(std::chrono::microseconds(20));
        if (sub_rc[i] != EIS_OK) {
            if (status_out) status_out[i] = sub_rc[i];
            if (first_err == EIS_OK) first_err = sub_rc[i];
            continue;
        }
        uint64_t res = 0;
        double lat = 0;
        int rc;
        Clock::time_point t_done;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            auto it = s->reqs.find(ids[i]);
            const auto deadline = Clock::now() + std::chrono::seconds(600);
            while (it != s->reqs.end() && !it->second.done) {
                if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) break;
                it = s->reqs.find(ids[i]);
            }
            if (it == s->reqs.end()) {
                rc = EIS_ENOTFOUND;
            } else if (!it->second.done) {
                rc = EIS_ETIMEOUT;
            } else {
                rc = it->second.status;
                res = it->second.sumE;
                t_done = it->second.t_done;
                s->reqs.erase(it);
                lat = std::chrono::duration<double, std::micro>(t_done - t_arr[i]).count();
            }
        }
        if (results_out) results_out[i] = res;
        if (status_out) status_out[i] = rc;
        if (latency_us_out) latency_us_out[i] = lat;
        if (rc != EIS_OK && rc != EIS_ENOTD && first_err == EIS_OK) first_err = rc;
    }
    client.join();
    if (wall_s_out) *wall_s_out = std::chrono::duration<double>(Clock::now() - t0).count();
    return first_err;
}

}  // extern "C"
