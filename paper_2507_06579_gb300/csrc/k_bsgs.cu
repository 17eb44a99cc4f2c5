// k_bsgs.cu -- the lane-per-d infrastructure search of the batch path
// (Algorithm 1 with the sparse baby table of eis_bsgs.cuh).
//
//  k_walk_record  the persistent baby walk (k_walk.cu's lean step, ten steps
//                 per warp vote, work stealing from the survivor queue) that
//                 also records every marked state into the lane's table
//                 region.  A d whose centre does not come within nbaby steps
//                 (or whose table fills) is handed on as a DRecord, and the
//                 lane takes the region that belongs to that record's slot
//                 for its next d.
//  k_bsgs_index   one thread per handed-on d: the table's hash index, built
//                 in shared memory and copied next to the entries.
//  k_bsgs         one d per lane, lanes refilled from the records: each
//                 cycle composes mu <- reduce(mu * G), walks baby steps to
//                 the first marked state x and one step beyond, and looks x
//                 up under its direct and mirror keys; the next cycle
//                 composes from state x + 1.  A d the search cannot finish
//                 (reduction or walk past its limits) goes to a fallback
//                 list that the plain persistent walk finishes.
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

__device__ __forceinline__ void store_entry(DEntry *e, float Q, float num, uint32_t S) {
    *reinterpret_cast<uint4 *>(e) = make_uint4(__float_as_uint(Q), __float_as_uint(num), S, 0u);
}

constexpr int kRecGroup = 10;  // steps per warp vote in the recording walk

// The recording baby walk.  Queue positions [q_lo, min(q_hi, n_surv)) are
// taken from the end of the survivor queue (largest d first), as in the
// plain persistent walk.
template <bool kFast>
__device__ __forceinline__ void walk_record_body(
    const Seg *__restrict__ segs, uint32_t nseg, const uint32_t *__restrict__ surv,
    const uint32_t *__restrict__ n_surv_ptr, uint32_t q_lo, uint32_t q_hi,
    uint32_t *__restrict__ next_ptr, uint32_t *__restrict__ flags, uint8_t *__restrict__ glog,
    unsigned long long *__restrict__ steps_acc, int *__restrict__ status, uint32_t step_limit,
    uint32_t nbaby, float tau, DRecord *__restrict__ recs, uint32_t *__restrict__ nrec,
    uint32_t rec_cap, unsigned char *__restrict__ pool) {
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
    uint32_t k = 0;          // entries recorded
    uint32_t jl = 0;         // position of the last marked state recorded
    bool rec_on = false;     // recording (and handing on) still possible for this d
    bool active = false;
    bool exhausted = q_lo >= q_end;  // warp-uniform
    uint32_t cand = 0;
    uint32_t done = 0;       // steps walked by the current d
    unsigned long long my_steps = 0;
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
                        // s = (C - 1)/2 (fast) or C/2, exactly; T = tau * s as bsgs_threshold
                        T = __fmul_rn(tau, __fmul_rn(kFast ? __fsub_rn(C, 1.0f) : C, 0.5f));
                        // entry 0: a_l = O_K again, (2, P_1), class 0
                        store_entry(tab, 2.0f, w.num, 0u);
                        k = 1;
                        jl = 0;
                        rec_on = true;
                        if (w.Q < T) {  // state 1 itself (S_1 = acc)
                            store_entry(tab + 1, w.Q, w.num, (uint32_t)w.acc);
                            k = 2;
                            jl = 1;
                        }
                    }
                }
            }
        }
        if (!__any_sync(kFull, active)) break;
        const uint32_t cap = (active && rec_on) ? min(nbaby, step_limit) : step_limit;
        uint32_t room = active ? cap - min(done, cap) : 0xffffffffu;
        for (int o = 16; o > 0; o >>= 1) room = min(room, __shfl_xor_sync(kFull, room, o));
        uint32_t n = 0, back = 0;
        bool hit = false, full = false;
        for (;;) {
            LeanState ws[kRecGroup];
            ws[0] = w;
            const bool c0 = lean_step<kFast>(ws[0], C);
            bool any = c0;
            bool mark = ws[0].Q < T;
#pragma unroll
            for (int i = 1; i < kRecGroup; ++i) {
                ws[i] = ws[i - 1];
                any |= lean_step<kFast>(ws[i], C);
                mark |= ws[i].Q < T;
            }
            const uint32_t n0 = n;  // steps of this invocation before the group
            n += kRecGroup;
            int sum = 0;
#pragma unroll
            for (int i = 0; i < kRecGroup; ++i) sum += ws[i].x;
            const int acc0 = w.acc;
            const int acc = w.acc + sum;
            w = ws[kRecGroup - 1];
            w.acc = acc;
            mark &= rec_on;
            if (__any_sync(kFull, mark)) {
                if (mark) {
                    // ws[i] is position done + n0 + i + 2 (state 1 had 0 steps);
                    // S = acc_i + steps_i (mod 3), reduced by the reader
                    int a = acc0;
                    const uint32_t st0 = done + n0 + 1;
#pragma unroll
                    for (int i = 0; i < kRecGroup; ++i) {
                        a += ws[i].x;
                        if (ws[i].Q < T && k < (uint32_t)kBsgsKmax) {
                            store_entry(tab + k, ws[i].Q, ws[i].num, (uint32_t)a + st0 + (uint32_t)i);
                            ++k;
                            jl = st0 + (uint32_t)i + 1;
                        }
                    }
                    full = k >= (uint32_t)kBsgsKmax;
                }
            }
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
}

}  // namespace

__global__ void __launch_bounds__(256, 3) k_walk_record(
    const Seg *__restrict__ segs, uint32_t nseg, const uint32_t *__restrict__ surv,
    const uint32_t *__restrict__ n_surv_ptr, uint32_t q_lo, uint32_t q_hi,
    uint32_t *__restrict__ next_ptr, uint32_t *__restrict__ flags, uint8_t *__restrict__ glog,
    unsigned long long *__restrict__ steps_acc, int *__restrict__ status, uint32_t step_limit,
    uint32_t nbaby, float tau, DRecord *__restrict__ recs, uint32_t *__restrict__ nrec,
    uint32_t rec_cap, unsigned char *__restrict__ pool, int fast) {
    if (fast)
        walk_record_body<true>(segs, nseg, surv, n_surv_ptr, q_lo, q_hi, next_ptr, flags, glog,
                               steps_acc, status, step_limit, nbaby, tau, recs, nrec, rec_cap, pool);
    else
        walk_record_body<false>(segs, nseg, surv, n_surv_ptr, q_lo, q_hi, next_ptr, flags, glog,
                                steps_acc, status, step_limit, nbaby, tau, recs, nrec, rec_cap,
                                pool);
}

// One warp per record: the open-addressing index of its table (the probing
// of bsgs_index; concurrent inserts claim empty slots by compare-and-swap
// on the slot's word in shared memory), stored after the entries; and G =
// entry k-1 with c_G added to the record.
__global__ void __launch_bounds__(256) k_bsgs_index(const Seg *__restrict__ segs, uint32_t nseg,
                                                    DRecord *__restrict__ recs,
                                                    const uint32_t *__restrict__ nrec,
                                                    uint32_t rec_cap, unsigned char *__restrict__ pool,
                                                    unsigned long long *__restrict__ handed) {
    __shared__ __align__(16) uint32_t sl_all[8][kBsgsSlots / 4];
    const uint32_t n = min(*nrec, rec_cap);
    if (blockIdx.x == 0 && threadIdx.x == 0 && handed) atomicAdd(handed, (unsigned long long)n);
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    uint32_t *sl32 = sl_all[wib];
    for (uint32_t r = blockIdx.x * 8 + wib; r < n; r += gridDim.x * 8) {
        const uint4 head = *reinterpret_cast<const uint4 *>(recs + r);  // cand, k, region, s
        const uint32_t k = head.y;
        unsigned char *base = pool + (size_t)head.z * kBsgsRegionBytes;
        const uint4 *e = reinterpret_cast<const uint4 *>(base);
        // every entry load of the table in flight at once (k <= 128)
        uint4 v[kBsgsKmax / 32];
#pragma unroll
        for (int t = 0; t < kBsgsKmax / 32; ++t) {
            const uint32_t i = lane + 32 * t;
            v[t] = i < k ? e[i] : make_uint4(0u, 0u, 0u, 0u);
        }
        for (int i = lane; i < kBsgsSlots / 4; i += 32) sl32[i] = 0xffffffffu;
        __syncwarp();
#pragma unroll
        for (int t = 0; t < kBsgsKmax / 32; ++t) {
            const uint32_t i = lane + 32 * t;
            if (i < k) {
                uint32_t p = bsgs_slot(v[t].x, v[t].y);
                for (;;) {
                    const uint32_t w = p >> 2, sh = 8 * (p & 3);
                    const uint32_t cur = sl32[w];
                    if (((cur >> sh) & 0xFFu) != 0xFFu) {
                        p = (p + 1) & (kBsgsSlots - 1);  // taken: next slot
                        continue;
                    }
                    const uint32_t nw = (cur & ~(0xFFu << sh)) | (i << sh);
                    if (atomicCAS(&sl32[w], cur, nw) == cur) break;  // else the word changed: retry
                }
            }
        }
        __syncwarp();
        uint2 *dst = reinterpret_cast<uint2 *>(base + kBsgsKmax * kBsgsEntryBytes);
        dst[lane] = make_uint2(sl32[2 * lane], sl32[2 * lane + 1]);
        // G = entry k-1, held by lane (k-1) % 32 in v[(k-1) / 32]
        const uint32_t src = (k - 1) & 31, tg = (k - 1) >> 5;
        uint32_t gx = 0, gy = 0, gz = 0;
#pragma unroll
        for (int t = 0; t < kBsgsKmax / 32; ++t) {
            if ((uint32_t)t == tg) {
                gx = v[t].x;
                gy = v[t].y;
                gz = v[t].z;
            }
        }
        gx = __shfl_sync(kFull, gx, src);
        gy = __shfl_sync(kFull, gy, src);
        gz = __shfl_sync(kFull, gz, src);
        if (lane == 0) {
            const int64_t s = (int64_t)head.w;
            Ideal G;
            G.a = (int64_t)__uint_as_float(gx) / 2;
            G.b = (int64_t)__uint_as_float(gy) - s;  // floor(P + s (+ 1/2)) - s = P
            G.g = (int)(gz % 3u);
            const int64_t d = (int64_t)cand_to_d(segs, nseg, head.x);
            DRecord &rc = recs[r];
            rc.k = k | ((uint32_t)G.g << 16);
            rc.ga = (uint32_t)G.a;
            rc.gb = (uint32_t)G.b;
            rc.cG = lean_cG(G, d);
        }
        __syncwarp();
    }
}

namespace {

// Steps per warp vote while the lanes walk to their marked states.
constexpr int kBsgsGroup = 4;

__device__ __forceinline__ void fallback(uint32_t *fb_list, uint32_t *fb_count, uint32_t fb_cap,
                                         uint32_t cand, int *status) {
    const uint32_t slot = atomicAdd(fb_count, 1u);
    if (slot < fb_cap)
        fb_list[slot] = cand;
    else
        atomicOr(status, kErrGiant);
}

template <bool kFast, int kCompose>
__device__ __forceinline__ void bsgs_body(
    const Seg *__restrict__ segs, uint32_t nseg, const DRecord *__restrict__ recs,
    const uint32_t *__restrict__ nrec, uint32_t rec_cap, uint32_t *__restrict__ next_ptr,
    const unsigned char *__restrict__ pool, uint32_t *__restrict__ flags, uint8_t *__restrict__ glog,
    unsigned long long *__restrict__ acc, int *__restrict__ status, uint32_t *__restrict__ fb_list,
    uint32_t *__restrict__ fb_count, uint32_t fb_cap, float tau, uint32_t max_cycles,
    uint32_t walk_cap) {
    const uint32_t n = min(*nrec, rec_cap);
    const int lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    bool active = false, exhausted = false;
    uint32_t cand = 0, cycles = 0;
    int64_t d = 0, s = 0, L = 0, cG = 0;
    float T = 0.0f, C = 0.0f;
    const DEntry *tab = nullptr;
    const uint8_t *slots = nullptr;
    Ideal G{1, 1, 0}, mu{1, 1, 0};
    unsigned long long my_cycles = 0, my_walk = 0;
    for (;;) {
        const unsigned need = __ballot_sync(kFull, !active);
        if (need && !exhausted) {
            const int leader = __ffs(need) - 1;
            uint32_t base = 0;
            if (lane == leader) base = atomicAdd(next_ptr, (uint32_t)__popc(need));
            base = __shfl_sync(kFull, base, leader);
            if ((uint64_t)base + __popc(need) >= n) exhausted = true;
            if (!active) {
                const uint32_t idx = base + __popc(need & lt);
                if (idx < n) {
                    const uint4 r0 = *reinterpret_cast<const uint4 *>(recs + idx);
                    const uint4 r1 = *(reinterpret_cast<const uint4 *>(recs + idx) + 1);
                    cand = r0.x;
                    d = (int64_t)cand_to_d(segs, nseg, cand);
                    s = (int64_t)r0.w;
                    if (kCompose == 1) L = (int64_t)isqrt44((uint64_t)s);
                    C = __uint2float_rn((uint32_t)(kFast ? 2 * s + 1 : 2 * s));
                    T = __fmul_rn(tau, __uint2float_rn((uint32_t)s));
                    tab = reinterpret_cast<const DEntry *>(pool + (size_t)r0.z * kBsgsRegionBytes);
                    slots = reinterpret_cast<const uint8_t *>(tab + kBsgsKmax);
                    G.a = (int64_t)r1.x;
                    G.b = (int64_t)r1.y;
                    G.g = (int)(r0.y >> 16);
                    cG = (int64_t)(((uint64_t)r1.w << 32) | r1.z);
                    mu = G;
                    cycles = 0;
                    active = true;
                }
            }
        }
        if (!__any_sync(kFull, active)) break;
        // ---- giant step: mu <- reduce(mu * G), with Q_{-1} of the result
        Ideal nx{1, 1, 0};
        int64_t Qm = 2;
        if (active) {
            const bool ok = bsgs_giant(kCompose, mu, G, cG, d, s, L, nx, Qm) && ++cycles <= max_cycles;
            if (!ok) {
                fallback(fb_list, fb_count, fb_cap, cand, status);
                my_cycles += cycles;
                active = false;
            }
        }
        // ---- walk to the first marked state x and one step beyond; a lane
        // stops there (at x + 1) while the others finish their walks
        LeanState w;
        float Cw = C;
        int gc = 0;
        if (active) {
            w.num = bsgs_num(nx.b, s, kFast);
            w.Q = __uint2float_rn((uint32_t)(2 * nx.a));
            w.Qp = __uint2float_rn((uint32_t)Qm);
            w.x = (int)((nx.b >> 1) & 1);
            w.acc = 0;
            gc = nx.g;
        } else {
            lean_park_idle(w, Cw);
        }
        bool walking = active, at_x = false;
        float numx = 0.0f;
        uint32_t walked = 0;
        while (__any_sync(kFull, walking)) {
#pragma unroll
            for (int i = 0; i < kBsgsGroup; ++i) {
                if (walking) {
                    lean_step<kFast>(w, Cw);
                    gc += 1 + w.x;
                    ++walked;
                    if (at_x) {
                        walking = false;  // at x + 1
                    } else if (w.Q < T) {
                        at_x = true;      // at x
                        numx = w.num;
                    }
                }
            }
            // a walk that meets no marked state within walk_cap steps gives
            // the d up to the fallback walk
            if (walking && walked >= walk_cap) {
                fallback(fb_list, fb_count, fb_cap, cand, status);
                my_cycles += cycles;
                active = false;
                walking = false;
            }
        }
        my_walk += walked;
        if (!active) continue;
        // ---- look x up: direct key (Q_x, P_x), then mirror key (Q_x, P_{x+1});
        // the lane stands at x + 1, so Q_x = w.Qp and g_x = gc - 1 - x_{x+1}
        const int gx = gc - 1 - w.x;
        int g = -1;
        int e = bsgs_find(tab, slots, __float_as_uint(w.Qp), __float_as_uint(numx));
        if (e >= 0) {
            g = (gx - (int)(tab[e].s % 3u) + 3 * 4) % 3;  // x = l + j
        } else {
            e = bsgs_find(tab, slots, __float_as_uint(w.Qp), __float_as_uint(w.num));
            if (e >= 0) g = (gx + (int)(tab[e].s % 3u)) % 3;  // x = l - j
        }
        if (g >= 0) {
            record_flag(flags, glog, cand, g);
            my_cycles += cycles;
            active = false;
        } else {
            mu.a = (int64_t)w.Q / 2;
            mu.b = (int64_t)w.num - s;
            mu.g = gc % 3;
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
    uint32_t *__restrict__ fb_count, uint32_t fb_cap, float tau, uint32_t max_cycles,
    uint32_t walk_cap) {
    bsgs_body<kFast, kCompose>(segs, nseg, recs, nrec, rec_cap, next_ptr, pool, flags, glog, acc,
                               status, fb_list, fb_count, fb_cap, tau, max_cycles, walk_cap);
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
                          uint32_t *fb_count, uint32_t fb_cap, float tau, uint32_t max_cycles,
                          uint32_t walk_cap) {
    void *args[] = {&segs, &nseg, &recs, &nrec, &rec_cap, &next_ptr, &pool, &flags, &glog,
                    &acc, &status, &fb_list, &fb_count, &fb_cap, &tau, &max_cycles, &walk_cap};
    return cudaLaunchKernel(k_bsgs_kernel(fast, compose), dim3(grid), dim3(128), args, 0, st);
}

}  // namespace eis
