// k_bsgs.cu -- the lane-per-d infrastructure search of the batch path
// (Algorithm 1 with the sparse baby table of eis_bsgs.cuh).
//
//  k_walk_record  the persistent baby walk (k_walk.cu's lean step, ten steps
//                 per warp vote, work stealing from the survivor queue) that
//                 also stores every marked state, as the step reaches it,
//                 into the lane's table region.  A d whose centre does not
//                 come within nbaby steps (or whose table fills) is handed on
//                 as a DRecord; a warp stops to hand on and refill at most
//                 every kRecEpoch steps, so a lane may record a little past
//                 nbaby.  The lane then takes the region that belongs to that
//                 record's slot for its next d.
//  k_bsgs_t       one d per lane, lanes refilled from the records (the warp
//                 loads a fresh lane's table coalesced and indexes it as
//                 fingerprints in that lane's shared memory): each cycle
//                 composes mu <- reduce(mu * G), walks baby steps to the
//                 first marked state x and one step beyond, and looks x up
//                 under its direct and mirror keys (shared-memory probes; a
//                 fingerprint match is settled by a warp-wide exact scan of
//                 the entries); the next cycle composes from state x + 1.
//                 A d the search cannot finish (reduction or walk past its
//                 limits) goes to a fallback list that the plain persistent
//                 walk finishes.
#include "eis.h"
#include "eis_bsgs.cuh"
#include "eis_common.cuh"
#include "eis_kernels.h"

namespace eis {

namespace {

__device__ __forceinline__ void record_flag(uint32_t *__restrict__ flags, uint8_t *__restrict__ glog,
                                            uint64_t cand, int g) {
    if (g == 0) atomicOr(&flags[cand >> 5], 1u << (cand & 31));
    if (glog) glog[cand] = (uint8_t)(1 + g);
}

__device__ __forceinline__ void warp_add(unsigned long long *acc, unsigned long long v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(acc, v);
}

__device__ __forceinline__ DEntry *region_entries(unsigned char *pool, uint32_t region) {
    return reinterpret_cast<DEntry *>(pool + (size_t)region * kBsgsRegionBytes);
}

// An entry: Q, num (fp32 bits), S (class, reduced by the reader), position j.
__device__ __forceinline__ void store_entry(DEntry *e, float Q, float num, uint32_t S, uint32_t j) {
    *reinterpret_cast<uint4 *>(e) = make_uint4(__float_as_uint(Q), __float_as_uint(num), S, j);
}

constexpr int kRecGroup = 10;  // steps per warp vote in the recording walk
constexpr uint32_t kRecEpoch = 256;  // least steps between hand-offs of a warp's lanes

// The recording baby walk.  Queue positions [q_lo, min(q_hi, n_surv)) are
// taken from the end of the survivor queue (largest d first), as in the
// plain persistent walk.
template <bool kFast>
__device__ __forceinline__ void walk_record_body(
    const Seg *__restrict__ segs, uint32_t nseg, const uint32_t *__restrict__ surv,
    const uint32_t *__restrict__ n_surv_ptr, uint32_t q_lo, uint32_t q_hi,
    uint32_t *__restrict__ next_ptr, uint32_t *__restrict__ flags, uint8_t *__restrict__ glog,
    unsigned long long *__restrict__ steps_acc, int *__restrict__ status, uint32_t step_limit,
    const TuneTab &tt, DRecord *__restrict__ recs, uint32_t *__restrict__ nrec, uint32_t rec_cap,
    unsigned char *__restrict__ pool, unsigned long long *__restrict__ handed_acc) {
    const uint32_t n_total = *n_surv_ptr;
    const uint32_t q_end = min(n_total, q_hi);
    const int lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    uint32_t region = blockIdx.x * blockDim.x + threadIdx.x;  // this lane's first region
    DEntry *tab = region_entries(pool, region);
    LeanState w;
    float C;
    lean_park_idle(w, C);
    float T = 0.0f;          // marking threshold of the current d
    uint32_t nbaby = 0;      // baby steps of the current d before it is handed on
    uint32_t k = 0;          // entries recorded
    uint32_t jl = 0;         // position of the last marked state recorded
    bool rec_on = false;     // recording (and handing on) still possible for this d
    bool active = false;
    bool exhausted = q_lo >= q_end;  // warp-uniform
    uint32_t cand = 0;
    uint32_t done = 0;       // steps walked by the current d
    unsigned long long my_steps = 0, my_handed = 0;
    for (;;) {
        for (;;) {
            const unsigned need = __ballot_sync(kFull, !active);
            if (need == 0 || exhausted) break;
            const int leader = __ffs(need) - 1;
            uint32_t base = 0;
            if (lane == leader) base = atomicAdd(next_ptr, (uint32_t)__popc(need));
            base = __shfl_sync(kFull, base, leader) + q_lo;
            if ((uint64_t)base + __popc(need) >= q_end) exhausted = true;
            if (!active) {
                const uint32_t idx = base + __popc(need & lt);
                if (idx < q_end) {
                    cand = surv[n_total - 1 - idx];
                    const uint64_t d = cand_to_d(segs, nseg, cand);
                    int g;
                    my_steps += 1;
                    if (lean_init<kFast>(d, w, C, g)) {
                        record_flag(flags, glog, cand, g);
                        lean_park_idle(w, C);
                    } else {
                        active = true;
                        done = 0;
                        const int row = tune_row(tt, d);
                        nbaby = tt.nbaby[row];
                        // s = (C - 1)/2 (fast) or C/2, exactly; T = tau * s as bsgs_threshold
                        T = __fmul_rn(tt.tau[row], __fmul_rn(kFast ? __fsub_rn(C, 1.0f) : C, 0.5f));
                        k = 1;
                        jl = 0;
                        rec_on = nbaby > 0;
                        if (rec_on) {
                            // entry 0: a_l = O_K again, (2, P_1), class 0
                            store_entry(tab, 2.0f, w.num, 0u, 0u);
                            if (w.Q < T) {  // state 1 itself (S_1 = acc)
                                store_entry(tab + 1, w.Q, w.num, (uint32_t)w.acc, 1u);
                                k = 2;
                                jl = 1;
                            }
                        }
                    }
                }
            }
        }
        if (!__any_sync(kFull, active)) break;
        // Steps before the warp next stops to hand d on or refill: at least
        // kRecEpoch, so that lanes hand on together (a lane past nbaby keeps
        // recording: a longer table only lengthens the stride), but never past
        // a lane's step limit.
        uint32_t rem_rec = (active && rec_on) ? nbaby - min(done, nbaby) : 0xffffffffu;
        uint32_t rem_lim = active ? step_limit - min(done, step_limit) : 0xffffffffu;
        for (int o = 16; o > 0; o >>= 1) {
            rem_rec = min(rem_rec, __shfl_xor_sync(kFull, rem_rec, o));
            rem_lim = min(rem_lim, __shfl_xor_sync(kFull, rem_lim, o));
        }
        const uint32_t room = min(max(rem_rec, kRecEpoch), rem_lim);
        uint32_t n = 0, back = 0;
        bool hit = false, full = false;
        for (;;) {
            // ws[i] is position done + n + i + 2 (state 1 had 0 steps); a marked
            // state is stored as it is reached, with S = acc_i + steps_i (mod 3,
            // reduced by the reader)
            const uint32_t st0 = done + n + 1;
            LeanState ws[kRecGroup];
            bool any = false, c0 = false;
            int a = w.acc;
            // a group records only while the table has room for all its steps,
            // so each step needs a single compare; a table that cannot take a
            // whole group is full (every marked state up to jl is in it)
            const bool rec_g = rec_on && k + (uint32_t)kRecGroup <= (uint32_t)kBsgsKmax;
#pragma unroll
            for (int i = 0; i < kRecGroup; ++i) {
                ws[i] = i ? ws[i - 1] : w;
                const bool ci = lean_step<kFast>(ws[i], C);
                if (i == 0) c0 = ci;
                any |= ci;
                a += ws[i].x;
                if (rec_g && ws[i].Q < T) {
                    jl = st0 + (uint32_t)i + 1;
                    store_entry(tab + k, ws[i].Q, ws[i].num, (uint32_t)a + st0 + (uint32_t)i, jl);
                    ++k;
                }
            }
            n += kRecGroup;
            const int acc = a;
            w = ws[kRecGroup - 1];
            w.acc = acc;
            full = rec_on && k + (uint32_t)kRecGroup > (uint32_t)kBsgsKmax;
            if (__any_sync(kFull, any)) {
                hit = any;
                int post = 0;
#pragma unroll
                for (int i = kRecGroup - 1; i >= 0; --i) {
                    const bool c = i ? (any &&
                                        ((__float_as_int(ws[i].Q) == __float_as_int(ws[i - 1].Q)) |
                                         (__float_as_int(ws[i].num) == __float_as_int(ws[i - 1].num))))
                                     : c0;
                    if (c) {
                        w = ws[i];
                        w.acc = acc - post;
                        back = (uint32_t)(kRecGroup - 1 - i);
                    }
                    post += ws[i].x;
                }
                break;
            }
            if (n >= room || __any_sync(kFull, full)) break;
        }
        if (active) {
            done += n - back;
            if (hit) {
                record_flag(flags, glog, cand, lean_finish(w, done));
                my_steps += done;
                active = false;
                lean_park_idle(w, C);
            } else if (rec_on && (done >= nbaby || full)) {
                bool handed = false;
                if (jl >= (uint32_t)kBsgsMinJl) {
                    const uint32_t slot = atomicAdd(nrec, 1u);
                    if (slot < rec_cap) {
                        // s = floor(sqrt d) from C = 2s (+1), exactly
                        const uint32_t sv = (uint32_t)__fmul_rn(kFast ? __fsub_rn(C, 1.0f) : C, 0.5f);
                        *reinterpret_cast<uint4 *>(recs + slot) = make_uint4(cand, k, region, sv);
                        // regions 0 .. lanes-1 are the lanes' first ones;
                        // region lanes + slot belongs to record slot `slot`,
                        // whose d has just left its region: the lane takes it
                        region = gridDim.x * blockDim.x + slot;
                        tab = region_entries(pool, region);
                        handed = true;
                    }
                }
                if (handed) {
                    my_steps += done;
                    ++my_handed;
                    active = false;
                    lean_park_idle(w, C);
                } else {
                    rec_on = false;  // too few marked states (or no record slot): walk on
                }
            } else if (done >= step_limit) {
                atomicOr(status, kErrSteps);
                my_steps += done;
                active = false;
                lean_park_idle(w, C);
            }
        }
    }
    warp_add(steps_acc, my_steps);
    warp_add(handed_acc, my_handed);
}

}  // namespace

__global__ void __launch_bounds__(256, 3) k_walk_record(
    const Seg *__restrict__ segs, uint32_t nseg, const uint32_t *__restrict__ surv,
    const uint32_t *__restrict__ n_surv_ptr, uint32_t q_lo, uint32_t q_hi,
    uint32_t *__restrict__ next_ptr, uint32_t *__restrict__ flags, uint8_t *__restrict__ glog,
    unsigned long long *__restrict__ steps_acc, int *__restrict__ status, uint32_t step_limit,
    const __grid_constant__ TuneTab tt, DRecord *__restrict__ recs, uint32_t *__restrict__ nrec,
    uint32_t rec_cap, unsigned char *__restrict__ pool, unsigned long long *__restrict__ handed_acc,
    int fast) {
    if (fast)
        walk_record_body<true>(segs, nseg, surv, n_surv_ptr, q_lo, q_hi, next_ptr, flags, glog,
                               steps_acc, status, step_limit, tt, recs, nrec, rec_cap, pool,
                               handed_acc);
    else
        walk_record_body<false>(segs, nseg, surv, n_surv_ptr, q_lo, q_hi, next_ptr, flags, glog,
                                steps_acc, status, step_limit, tt, recs, nrec, rec_cap, pool,
                                handed_acc);
}

namespace {

// Steps per warp vote while the lanes walk to their marked states.
constexpr int kBsgsGroup = 2;

__device__ __forceinline__ void fallback(uint32_t *fb_list, uint32_t *fb_count, uint32_t fb_cap,
                                         uint32_t cand, int *status) {
    const uint32_t slot = atomicAdd(fb_count, 1u);
    if (slot < fb_cap)
        fb_list[slot] = cand;
    else
        atomicOr(status, kErrGiant);
}

// Per-lane fingerprint index of a d's table in shared memory: 256 slots of
// one byte, 0 = empty, else an 8-bit fingerprint (1..255) of the key stored at
// the slot its probe sequence reached.  A key whose probe meets no slot with
// its fingerprint before an empty one is not in the table; a fingerprint
// match is settled by an exact scan of the entries.
constexpr int kFpWords = kBsgsSlots / 4;

__device__ __forceinline__ uint32_t fp_of(uint32_t q, uint32_t num) {
    const uint32_t h = (q * 0x2545F491u) ^ (num * 0x9E3779B9u) ^ (q >> 11);
    const uint32_t f = (h * 0x85EBCA6Bu) >> 24;
    return f ? f : 1u;
}

// Each failed compare-and-swap means another lane's insert landed in that
// word, so with at most kBsgsKmax entries in kBsgsSlots slots an insert takes
// fewer than kBsgsSlots + kBsgsKmax iterations; the bound is above that.
__device__ __forceinline__ void fp_insert(uint32_t *sl, uint32_t q, uint32_t num) {
    uint32_t p = bsgs_slot(q, num);
    const uint32_t f = fp_of(q, num);
    for (int n = 0; n < 2 * kBsgsSlots; ++n) {
        const uint32_t w = p >> 2, sh = 8 * (p & 3);
        const uint32_t cur = sl[w];
        if ((cur >> sh) & 0xFFu) {
            p = (p + 1) & (kBsgsSlots - 1);  // taken: next slot
            continue;
        }
        if (atomicCAS(&sl[w], cur, cur | (f << sh)) == cur) return;  // else the word changed: retry
    }
}

// True when (q, num) may be in the table (a slot on its probe sequence holds
// its fingerprint), false when it certainly is not.
__device__ __forceinline__ bool fp_maybe(const uint32_t *sl, uint32_t q, uint32_t num) {
    uint32_t p = bsgs_slot(q, num);
    const uint32_t f = fp_of(q, num);
    for (int n = 0; n < kBsgsSlots; ++n) {
        const uint32_t b = (sl[p >> 2] >> (8 * (p & 3))) & 0xFFu;
        if (b == 0) return false;
        if (b == f) return true;
        p = (p + 1) & (kBsgsSlots - 1);
    }
    return true;
}

struct SIdeal {
    int32_t a, b, g;
};

template <bool kFast, int kCompose>
__device__ __forceinline__ void bsgs_body(
    const Seg *__restrict__ segs, uint32_t nseg, const DRecord *__restrict__ recs,
    const uint32_t *__restrict__ nrec, uint32_t rec_cap, uint32_t *__restrict__ next_ptr,
    const unsigned char *__restrict__ pool, uint32_t *__restrict__ flags, uint8_t *__restrict__ glog,
    unsigned long long *__restrict__ acc, int *__restrict__ status, uint32_t *__restrict__ fb_list,
    uint32_t *__restrict__ fb_count, uint32_t fb_cap, const TuneTab &tt, uint32_t max_cycles,
    uint32_t walk_cap, uint32_t walk_window, uint32_t *__restrict__ fp_all) {
    const uint32_t n = min(*nrec, rec_cap);
    const uint32_t groups = (walk_window + kBsgsGroup - 1) / kBsgsGroup;
    const int lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    uint32_t *fp_warp = fp_all + (threadIdx.x & ~31u) * kFpWords;  // lane t's words at t * kFpWords
    uint32_t *fp_mine = fp_warp + lane * kFpWords;
    bool active = false, exhausted = false;
    uint32_t cand = 0, cycles = 0, k = 0;
    int64_t d = 0;
    int32_t s = 0, L = 0;  // floor(sqrt d) < 2^22 and its square root
    float T = 0.0f, C = 0.0f;
    const uint4 *tab = nullptr;
    // G = a_jl starts the search; the stride Y is reduce(a_jl * a_j') (taken
    // by the first cycle from Y = a_j', `first`), or a_jl when no table state
    // lies kBsgsWideGap steps before jl
    // reduced ideals of the lane's d, every coefficient below 2^22: held in
    // 32 bits and widened for the product
    SIdeal G{1, 1, 0}, mu{1, 1, 0}, Y{1, 1, 0};
    int32_t wY = 0, wmu = 0;  // third form coefficients (b^2 - d)/(4a) of Y and mu
    bool first = false;
    // the lane's walk, carried across iterations: it composes when its last
    // walk has ended (compose_now), else walks on
    LeanState w;
    float Cw = 0.0f;
    lean_park_idle(w, Cw);
    int gc = 0;
    bool at_x = false, compose_now = false;
    float numx = 0.0f;
    uint32_t walked = 0;
    uint32_t my_cycles = 0, my_walk = 0;
    for (;;) {
        // ---- refill idle lanes from the records
        const unsigned need = __ballot_sync(kFull, !active);
        bool fresh = false;
        if (need && !exhausted) {
            const int leader = __ffs(need) - 1;
            uint32_t base = 0;
            if (lane == leader) base = atomicAdd(next_ptr, (uint32_t)__popc(need));
            base = __shfl_sync(kFull, base, leader);
            if ((uint64_t)base + __popc(need) >= n) exhausted = true;
            if (!active) {
                const uint32_t idx = base + __popc(need & lt);
                if (idx < n) {
                    const uint4 r0 = *reinterpret_cast<const uint4 *>(recs + idx);  // cand, k, region, s
                    cand = r0.x;
                    k = r0.y;
                    tab = reinterpret_cast<const uint4 *>(pool + (size_t)r0.z * kBsgsRegionBytes);
                    s = (int32_t)r0.w;
                    fresh = true;
                }
            }
        }
        // ---- the whole warp indexes each fresh lane's table: entries loaded
        // coalesced, fingerprints inserted into that lane's slots
        unsigned pend = __ballot_sync(kFull, fresh);
        while (pend) {
            const int src = __ffs(pend) - 1;
            pend &= pend - 1;
            const uint32_t kk = __shfl_sync(kFull, k, src);
            const uint4 *e = reinterpret_cast<const uint4 *>(
                __shfl_sync(kFull, reinterpret_cast<unsigned long long>(tab), src));
            uint32_t *sl = fp_warp + src * kFpWords;
            uint4 v[kBsgsKmax / 32];
#pragma unroll
            for (int t = 0; t < kBsgsKmax / 32; ++t) {
                const uint32_t i = lane + 32 * t;
                v[t] = i < kk ? e[i] : make_uint4(0u, 0u, 0u, 0u);
            }
            sl[lane] = 0u;
            sl[lane + 32] = 0u;
            __syncwarp();
#pragma unroll
            for (int t = 0; t < kBsgsKmax / 32; ++t)
                if (lane + 32 * t < kk) fp_insert(sl, v[t].x, v[t].y);
            // G = entry kk-1, held by lane (kk-1) % 32 in v[(kk-1) / 32]
            const uint32_t tg = (kk - 1) >> 5;
            uint32_t gx = 0, gy = 0, gz = 0;
#pragma unroll
            for (int t = 0; t < kBsgsKmax / 32; ++t) {
                if ((uint32_t)t == tg) {
                    gx = v[t].x;
                    gy = v[t].y;
                    gz = v[t].z;
                }
            }
            gx = __shfl_sync(kFull, gx, (kk - 1) & 31);
            gy = __shfl_sync(kFull, gy, (kk - 1) & 31);
            gz = __shfl_sync(kFull, gz, (kk - 1) & 31);
            const uint32_t jlast = __shfl_sync(kFull, (tg == 0 ? v[0].w : tg == 1 ? v[1].w
                                                       : tg == 2 ? v[2].w : v[3].w), (kk - 1) & 31);
            // j' = the last entry (not entry 0, not jl itself) at least
            // kBsgsWideGap steps before jl
            uint32_t ej = 0;
#pragma unroll
            for (int t = 0; t < kBsgsKmax / 32; ++t) {
                const uint32_t i = lane + 32 * t;
                if (i >= 1 && i + 1 < kk && v[t].w + kBsgsWideGap <= jlast) ej = max(ej, i);
            }
            ej = __reduce_max_sync(kFull, ej);
            const uint32_t tj = ej >> 5;
            uint32_t jx = 0, jy = 0, jz = 0;
#pragma unroll
            for (int t = 0; t < kBsgsKmax / 32; ++t) {
                if ((uint32_t)t == tj) {
                    jx = v[t].x;
                    jy = v[t].y;
                    jz = v[t].z;
                }
            }
            jx = __shfl_sync(kFull, jx, ej & 31);
            jy = __shfl_sync(kFull, jy, ej & 31);
            jz = __shfl_sync(kFull, jz, ej & 31);
            if (lane == src) {
                G.a = (int32_t)__uint_as_float(gx) / 2;
                G.b = (int32_t)__uint_as_float(gy) - s;  // floor(P + s (+ 1/2)) - s = P
                G.g = (int)(gz % 3u);
                first = ej > 0;
                if (first) {
                    Y.a = (int32_t)__uint_as_float(jx) / 2;
                    Y.b = (int32_t)__uint_as_float(jy) - s;
                    Y.g = (int)(jz % 3u);
                } else {
                    Y = G;
                }
            }
            __syncwarp();
        }
        if (fresh) {
            d = (int64_t)cand_to_d(segs, nseg, cand);
            if (kCompose == 1) {
                L = (int32_t)isqrt44((uint64_t)s);
                wmu = (int32_t)lean_cG(Ideal{G.a, G.b, G.g}, d);
            }
            wY = (int32_t)lean_cG(Ideal{Y.a, Y.b, Y.g}, d);
            C = __uint2float_rn((uint32_t)(kFast ? 2 * s + 1 : 2 * s));
            Cw = C;
            T = __fmul_rn(tt.tau[tune_row(tt, (uint64_t)d)], __uint2float_rn((uint32_t)s));
            mu = G;
            cycles = 0;
            active = true;
            compose_now = true;
        }
        if (!__any_sync(kFull, active)) break;
        // ---- giant step for the lanes whose last walk has ended:
        // mu <- reduce(mu * Y), with Q_{-1} of the result, and a new walk
        if (active && compose_now) {
            Ideal nx{1, 1, 0};
            int64_t Qm = 2;
            const bool ok = bsgs_giant(kCompose, Ideal{mu.a, mu.b, mu.g}, wmu, Ideal{Y.a, Y.b, Y.g}, wY, d,
                                       s, L, nx, Qm) &&
                            ++cycles <= max_cycles;
            if (!ok) {
                fallback(fb_list, fb_count, fb_cap, cand, status);
                my_cycles += cycles;
                active = false;
            } else {
                if (first) {  // the first landing, reduce(a_jl * a_j'), is the stride
                    first = false;
                    Y = SIdeal{(int32_t)nx.a, (int32_t)nx.b, nx.g};
                    wY = (int32_t)(-Qm / 2);  // (b^2 - d)/(4a) = -Q_{-1}/2
                }
                w.num = bsgs_num(nx.b, s, kFast);
                w.Q = __uint2float_rn((uint32_t)(2 * nx.a));
                w.Qp = __uint2float_rn((uint32_t)Qm);
                w.x = (int)((nx.b >> 1) & 1);
                w.acc = 0;
                gc = nx.g;
                at_x = false;
                walked = 0;
                compose_now = false;
            }
        }
        // ---- walk at most walk_window steps toward the first marked state x
        // and one step beyond (a lane stops at x + 1); a walk that needs more
        // goes on next iteration while the other lanes compose
        bool walking = active && !compose_now;
        if (!walking) lean_park_idle(w, Cw);  // idle lanes step NaN states
        uint32_t stepped = 0;
        for (uint32_t grp = 0; grp < groups && __any_sync(kFull, walking); ++grp) {
#pragma unroll
            for (int i = 0; i < kBsgsGroup; ++i) {
                if (walking) {
                    lean_step<kFast>(w, Cw);
                    gc += 1 + w.x;
                    ++walked;
                    ++stepped;
                    if (at_x) {
                        walking = false;  // at x + 1
                        compose_now = true;
                    } else if (w.Q < T) {
                        at_x = true;      // at x
                        numx = w.num;
                    }
                }
            }
        }
        my_walk += stepped;
        if (active && !compose_now && walked >= walk_cap) {
            // no marked state within walk_cap steps: the fallback walk finishes it
            fallback(fb_list, fb_count, fb_cap, cand, status);
            my_cycles += cycles;
            active = false;
        }
        // ---- look x up for the lanes that reached x + 1: direct key
        // (Q_x, P_x) and mirror key (Q_x, P_{x+1}); the lane stands at x + 1,
        // so Q_x = w.Qp and g_x = gc - 1 - x_{x+1}
        const bool at_end = active && compose_now;
        const uint32_t kq = __float_as_uint(w.Qp), kd = __float_as_uint(numx),
                       km = __float_as_uint(w.num);
        const bool maybe = at_end && (fp_maybe(fp_mine, kq, kd) || fp_maybe(fp_mine, kq, km));
        int g = -1;
        // exact scan of the tables of the lanes with a fingerprint match, by
        // the whole warp
        unsigned scan = __ballot_sync(kFull, maybe);
        while (scan) {
            const int src = __ffs(scan) - 1;
            scan &= scan - 1;
            const uint32_t kk = __shfl_sync(kFull, k, src);
            const uint4 *e = reinterpret_cast<const uint4 *>(
                __shfl_sync(kFull, reinterpret_cast<unsigned long long>(tab), src));
            const uint32_t sq = __shfl_sync(kFull, kq, src), sd = __shfl_sync(kFull, kd, src),
                           sm = __shfl_sync(kFull, km, src);
            int jd = 0x7fffffff, jm = 0x7fffffff;
            uint32_t Sd = 0, Sm = 0;
#pragma unroll
            for (int t = 0; t < kBsgsKmax / 32; ++t) {
                const uint32_t i = lane + 32 * t;
                if (i < kk) {
                    const uint4 v = e[i];
                    if (v.x == sq && v.y == sd && (int)i < jd) {
                        jd = (int)i;
                        Sd = v.z;
                    }
                    if (v.x == sq && v.y == sm && (int)i < jm) {
                        jm = (int)i;
                        Sm = v.z;
                    }
                }
            }
            const unsigned hd = __ballot_sync(kFull, jd != 0x7fffffff);
            const unsigned hm = __ballot_sync(kFull, jm != 0x7fffffff);
            const uint32_t Sd0 = __shfl_sync(kFull, Sd, hd ? __ffs(hd) - 1 : 0);
            const uint32_t Sm0 = __shfl_sync(kFull, Sm, hm ? __ffs(hm) - 1 : 0);
            if (lane == src) {
                const int gx = gc - 1 - w.x;
                if (hd)
                    g = (gx - (int)(Sd0 % 3u) + 3 * 4) % 3;  // x = l + j
                else if (hm)
                    g = (gx + (int)(Sm0 % 3u)) % 3;          // x = l - j
            }
        }
        if (!at_end) continue;
        if (g >= 0) {
            record_flag(flags, glog, cand, g);
            my_cycles += cycles;
            active = false;
        } else {  // the next giant step starts from x + 1
            mu.a = (int32_t)w.Q / 2;
            mu.b = (int32_t)w.num - s;
            mu.g = gc % 3;
            wmu = -(int32_t)w.Qp / 2;  // Q_{-1} of x + 1 is Q_x
        }
    }
    warp_add(&acc[0], my_walk);
    warp_add(&acc[1], my_cycles);
}

}  // namespace

template <bool kFast, int kCompose>
__global__ void __launch_bounds__(128) k_bsgs_t(
    const Seg *__restrict__ segs, uint32_t nseg, const DRecord *__restrict__ recs,
    const uint32_t *__restrict__ nrec, uint32_t rec_cap, uint32_t *__restrict__ next_ptr,
    const unsigned char *__restrict__ pool, uint32_t *__restrict__ flags, uint8_t *__restrict__ glog,
    unsigned long long *__restrict__ acc, int *__restrict__ status, uint32_t *__restrict__ fb_list,
    uint32_t *__restrict__ fb_count, uint32_t fb_cap, const __grid_constant__ TuneTab tt,
    uint32_t max_cycles, uint32_t walk_cap, uint32_t walk_window) {
    __shared__ uint32_t fp_all[128 * kFpWords];  // 32 KB: 256 fingerprint slots per lane
    bsgs_body<kFast, kCompose>(segs, nseg, recs, nrec, rec_cap, next_ptr, pool, flags, glog, acc,
                               status, fb_list, fb_count, fb_cap, tt, max_cycles, walk_cap,
                               walk_window, fp_all);
}

// One instantiation per (quotient, composition), so that each kernel holds
// only the code it runs.
const void *k_bsgs_kernel(int fast, int compose) {
    if (fast) {
        if (compose == EIS_COMPOSE_NUCOMP) return reinterpret_cast<const void *>(&k_bsgs_t<true, 1>);
        return reinterpret_cast<const void *>(&k_bsgs_t<true, 0>);
    }
    if (compose == EIS_COMPOSE_NUCOMP) return reinterpret_cast<const void *>(&k_bsgs_t<false, 1>);
    return reinterpret_cast<const void *>(&k_bsgs_t<false, 0>);
}

cudaError_t launch_k_bsgs(uint32_t grid, cudaStream_t st, int fast, int compose, const Seg *segs,
                          uint32_t nseg, const DRecord *recs, const uint32_t *nrec, uint32_t rec_cap,
                          uint32_t *next_ptr, const unsigned char *pool, uint32_t *flags,
                          uint8_t *glog, unsigned long long *acc, int *status, uint32_t *fb_list,
                          uint32_t *fb_count, uint32_t fb_cap, const TuneTab &tt,
                          uint32_t max_cycles, uint32_t walk_cap, uint32_t walk_window) {
    TuneTab t = tt;
    void *args[] = {&segs, &nseg, &recs, &nrec, &rec_cap, &next_ptr, &pool, &flags, &glog,
                    &acc, &status, &fb_list, &fb_count, &fb_cap, &t, &max_cycles, &walk_cap,
                    &walk_window};
    return cudaLaunchKernel(k_bsgs_kernel(fast, compose), dim3(grid), dim3(128), args, 0, st);
}

}  // namespace eis
