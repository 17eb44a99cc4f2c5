// k_walk.cu -- the baby-step kernels (Appendix A walk, generator in Z/3).
//
//  k_walk_plain       one thread per candidate of a 2^24-wide block of d; the
//                     flags of a warp's 32 consecutive candidates are one
//                     ballot word.  A warp lasts as long as its longest walk.
//  k_walk_persistent  one resident grid; every lane walks one d at a time and,
//                     when its walk ends, takes the next square-free
//                     candidate from a global queue (warp-aggregated atomic),
//                     so lanes stay busy whatever the spread of periods.
//  k_sqfree_one       the square-free test of one d spread over a whole grid
//                     (single queries).
//  k_walk_single      one warp: the square-free answer of k_sqfree_one (or its
//                     own scan of the prime table), then the walk in lane 0.
// All three walkers run the lean step of eis_common.cuh (num = P + s state,
// class bit from the quotient's parity) and test for the centre once per
// group of steps.
#include "eis_common.cuh"
#include "eis_kernels.h"

namespace eis {

__device__ __forceinline__ void record_result(uint32_t *__restrict__ flags,
                                              uint8_t *__restrict__ glog, uint64_t cand, int g) {
    if (g == 0) atomicOr(&flags[cand >> 5], 1u << (cand & 31));
    if (glog) glog[cand] = (uint8_t)(1 + g);
}

__device__ __forceinline__ void add_steps(unsigned long long *acc, unsigned long long v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(acc, v);
}

// Steps per centre test in walk_one.
constexpr int kOneGroup = 8;

// One whole half-period walk by one thread, with the persistent walk's lean
// step: false past step_limit steps; otherwise g = log eps_d and n = steps
// after the first.  The centre is tested once per kOneGroup steps; a group
// that contains it is walked again from its first state, one step at a time.
template <bool kFast>
__device__ __forceinline__ bool walk_one(uint64_t d, uint32_t step_limit, int &g, uint32_t &n) {
    LeanState w;
    float C;
    n = 0;
    if (lean_init<kFast>(d, w, C, g)) return true;
    for (;;) {
        const LeanState w0 = w;
        bool any = false;
        int sum = 0;
#pragma unroll
        for (int i = 0; i < kOneGroup; ++i) {
            any |= lean_step<kFast>(w, C);
            sum += w.x;
        }
        if (any) {
            w = w0;
            for (int i = 0; i < kOneGroup; ++i) {
                const bool c = lean_step<kFast>(w, C);
                w.acc += w.x;
                ++n;
                if (c) break;
            }
            g = lean_finish(w, n);
            return true;
        }
        w.acc += sum;
        n += kOneGroup;
        if (n >= step_limit) return false;
    }
}

// K2.  Candidates [cand_first, cand_first + ncand) of one Seg, d of the first
// one = d_first.  cand_first is a multiple of 32, so each warp owns whole
// flag words and writes them without atomics.
__global__ void __launch_bounds__(256) k_walk_plain(uint64_t d_first, uint64_t cand_first,
                                                    uint32_t ncand,
                                                    const uint32_t *__restrict__ sqfree,
                                                    uint32_t *__restrict__ flags,
                                                    uint8_t *__restrict__ glog,
                                                    unsigned long long *__restrict__ steps_acc,
                                                    int *__restrict__ status, uint32_t step_limit) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t cand = cand_first + i;
    const bool valid = i < ncand;
    bool inE = false;
    unsigned long long steps = 0;
    if (valid && ((sqfree[cand >> 5] >> (cand & 31)) & 1u)) {
        const uint64_t d = d_first + 8ull * i;
        int g;
        uint32_t n = 0;
        steps = 1;
        const bool ok = (d < kFastDLimit) ? walk_one<true>(d, step_limit, g, n)
                                          : walk_one<false>(d, step_limit, g, n);
        steps += n;
        if (!ok) {
            atomicOr(status, kErrSteps);
            g = -1;
        }
        inE = (g == 0);
        if (glog && g >= 0) glog[cand] = (uint8_t)(1 + g);
    }
    const uint32_t word = __ballot_sync(kFull, inE);
    if ((threadIdx.x & 31) == 0 && valid) flags[cand >> 5] = word;
    add_steps(steps_acc, steps);
}

// Steps per warp vote in the persistent walk.
#ifndef EIS_WALK_GROUP
#define EIS_WALK_GROUP 10
#endif
constexpr int kWalkGroup = EIS_WALK_GROUP;

// K5.  The survivor queue surv[0, *n_surv) holds global candidate indices in
// increasing order; lanes take them from the end (largest d first within the
// Seg layout, which is sorted by d0) so that the cheapest walks run last.
// kDefer: walks longer than defer_after steps are handed to the giant-step
// kernel; the kernel without it carries none of that bookkeeping.
template <bool kDefer, bool kFast>
__device__ __forceinline__ void walk_persistent_body(
    const Seg *__restrict__ segs, uint32_t nseg, const uint32_t *__restrict__ surv,
    const uint32_t *__restrict__ n_surv_ptr, uint32_t *__restrict__ next_ptr,
    uint32_t *__restrict__ flags, uint8_t *__restrict__ glog,
    unsigned long long *__restrict__ steps_acc, int *__restrict__ status, uint32_t step_limit,
    uint32_t defer_after, uint32_t *__restrict__ defer_list, uint32_t *__restrict__ defer_count,
    uint32_t defer_cap) {
    const uint32_t n_surv = *n_surv_ptr;
    const int lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    // A walk longer than defer_after steps is handed to the giant-step kernel
    // (while the defer list has room).
    bool may_defer = kDefer;
    LeanState w;
    float C;  // 2s (+1): num' = C - remainder
    lean_park_idle(w, C);
    bool active = false;
    bool exhausted = false;  // warp-uniform
    uint32_t cand = 0;
    uint32_t done = 0;       // steps walked by the current d
    unsigned long long my_steps = 0;
    for (;;) {
        // Refill idle lanes; repeat while fresh d end at the first step.
        for (;;) {
            const unsigned need = __ballot_sync(kFull, !active);
            if (need == 0 || exhausted) break;
            const int leader = __ffs(need) - 1;
            uint32_t base = 0;
            if (lane == leader) base = atomicAdd(next_ptr, (uint32_t)__popc(need));
            base = __shfl_sync(kFull, base, leader);
            if ((uint64_t)base + __popc(need) >= n_surv) exhausted = true;
            if (!active) {
                const uint32_t idx = base + __popc(need & lt);
                if (idx < n_surv) {
                    cand = surv[n_surv - 1 - idx];
                    const uint64_t d = cand_to_d(segs, nseg, cand);
                    int g;
                    my_steps += 1;
                    if (lean_init<kFast>(d, w, C, g)) {
                        record_result(flags, glog, cand, g);
                        lean_park_idle(w, C);
                    } else {
                        active = true;
                        done = 0;
                        may_defer = kDefer;
                    }
                }
            }
        }
        if (!__any_sync(kFull, active)) break;
        // Walk until some lane reaches its centre (or the step limit),
        // kWalkGroup steps per warp vote: the intermediate states stay in
        // registers and a lane whose centre came early in the group takes
        // that state back (the steps past it are wasted, a few per d).  Idle
        // lanes hold NaN states whose centre test is false.
        const uint32_t cap = (kDefer && active && may_defer) ? min(defer_after, step_limit) : step_limit;
        uint32_t room = active ? cap - min(done, cap) : 0xffffffffu;
        for (int o = 16; o > 0; o >>= 1) room = min(room, __shfl_xor_sync(kFull, room, o));
        uint32_t n = 0, back = 0;
        bool hit = false;
        for (;;) {
            // The hot loop keeps two predicates (a centre at the group's first
            // step, and at any step); the exit path finds each lane's first
            // centre from the kept states, by bit equality (the values are
            // finite and non-zero on a lane with a centre, where it agrees
            // with the float test), and its acc by subtracting the class
            // bits of the steps after it.
            LeanState ws[kWalkGroup];
            ws[0] = w;
            const bool c0 = lean_step<kFast>(ws[0], C);
            bool any = c0;
#pragma unroll
            for (int i = 1; i < kWalkGroup; ++i) {
                ws[i] = ws[i - 1];
                any |= lean_step<kFast>(ws[i], C);
            }
            n += kWalkGroup;
            int sum = 0;
#pragma unroll
            for (int i = 0; i < kWalkGroup; ++i) sum += ws[i].x;
            const int acc = w.acc + sum;
            w = ws[kWalkGroup - 1];
            w.acc = acc;
            if (__any_sync(kFull, any)) {
                hit = any;
                int post = 0;  // class bits of the steps after step i
#pragma unroll
                for (int i = kWalkGroup - 1; i >= 0; --i) {
                    const bool c = i ? (any &&
                                        ((__float_as_int(ws[i].Q) == __float_as_int(ws[i - 1].Q)) |
                                         (__float_as_int(ws[i].num) == __float_as_int(ws[i - 1].num))))
                                     : c0;
                    if (c) {  // the last one written is the first centre
                        w = ws[i];
                        w.acc = acc - post;
                        back = (uint32_t)(kWalkGroup - 1 - i);
                    }
                    post += ws[i].x;
                }
                break;
            }
            if (n >= room) break;
        }
        if (active) {
            done += n - back;
            if (hit) {
                record_result(flags, glog, cand, lean_finish(w, done));
                my_steps += done;
                active = false;
                lean_park_idle(w, C);
            } else if (kDefer && may_defer && done >= defer_after && done < step_limit) {
                const uint32_t slot = atomicAdd(defer_count, 1u);
                if (slot < defer_cap) {
                    defer_list[slot] = cand;
                    my_steps += done;
                    active = false;
                    lean_park_idle(w, C);
                } else {
                    may_defer = false;  // list full: this walk goes on here
                }
            } else if (done >= step_limit) {
                atomicOr(status, kErrSteps);
                my_steps += done;
                active = false;
                lean_park_idle(w, C);
            }
        }
    }
    add_steps(steps_acc, my_steps);
}

__global__ void __launch_bounds__(256, 4) k_walk_persistent(
    const Seg *__restrict__ segs, uint32_t nseg, const uint32_t *__restrict__ surv,
    const uint32_t *__restrict__ n_surv_ptr, uint32_t *__restrict__ next_ptr,
    uint32_t *__restrict__ flags, uint8_t *__restrict__ glog,
    unsigned long long *__restrict__ steps_acc, int *__restrict__ status, uint32_t step_limit,
    uint32_t defer_after, uint32_t *__restrict__ defer_list, uint32_t *__restrict__ defer_count,
    uint32_t defer_cap, int fast) {
#define EIS_WALK_BODY(D, F)                                                                     \
    walk_persistent_body<D, F>(segs, nseg, surv, n_surv_ptr, next_ptr, flags, glog, steps_acc, \
                               status, step_limit, defer_after, defer_list, defer_count,        \
                               defer_cap)
    if (defer_after == 0) {
        if (fast) EIS_WALK_BODY(false, true); else EIS_WALK_BODY(false, false);
    } else {
        if (fast) EIS_WALK_BODY(true, true); else EIS_WALK_BODY(true, false);
    }
#undef EIS_WALK_BODY
}

// Square-free test of one d by a grid: *flag |= 1 when p^2 | d for one of
// the first nprimes odd primes of the table.  The caller passes the primes
// with p^2 <= d (no larger prime can divide d; d < 2^44 needs p < 2^22, the
// table's range) and sizes the grid to them.
__global__ void __launch_bounds__(256) k_sqfree_one(uint64_t d, const uint64_t *__restrict__ sqtab,
                                                    uint32_t nprimes, uint32_t *__restrict__ flag) {
    bool hit = false;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nprimes;
         i += gridDim.x * blockDim.x)
        hit |= d * sqtab[2 * i] <= sqtab[2 * i + 1];
    if (__any_sync(kFull, hit) && (threadIdx.x & 31) == 0) atomicOr(flag, 1u);
}

// Membership query for one d (one warp).  out[0] = 0 (d not in D) or
// 1 + log eps_d; out[1] = steps.  The square-free test covers every odd prime
// p with p^2 <= d from the table (d < 2^44 needs p < 2^22), or is read from
// sq_flag (k_sqfree_one) when given.
__global__ void __launch_bounds__(32) k_walk_single(uint64_t d, const uint32_t *__restrict__ primes,
                                                    const uint64_t *__restrict__ sqtab,
                                                    uint32_t nprimes, int *__restrict__ out,
                                                    int *__restrict__ status, uint32_t step_limit,
                                                    const uint32_t *__restrict__ sq_flag) {
    const bool sq = sq_flag ? (*sq_flag == 0) : warp_squarefree_fast(d, primes, sqtab, nprimes);
    if (threadIdx.x != 0) return;
    if (!sq || d % 8 != 5) {
        out[0] = 0;
        out[1] = 0;
        return;
    }
    int g;
    uint32_t k = 0;
    const bool ok = (d < kFastDLimit) ? walk_one<true>(d, step_limit, g, k)
                                      : walk_one<false>(d, step_limit, g, k);
    const uint32_t n = 1 + k;
    {
        if (!ok) {
            atomicOr(status, kErrSteps);
            g = -1;
        }
    }
    out[0] = 1 + g;
    out[1] = (int)n;
}

}  // namespace eis
