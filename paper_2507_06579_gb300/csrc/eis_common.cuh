// eis_common.cuh -- device-side building blocks shared by the kernels.
//
// The baby step (Appendix A of Breuer & Punch): on the reduced ideal
// [Q_j/2, (P_j + sqrt d)/2] of O_K, O_K = Z[(1+sqrt d)/2],
//     q_j = floor((P_j + sqrt d)/Q_j),  P_{j+1} = q_j Q_j - P_j,
//     Q_{j+1} = (d - P_{j+1}^2)/Q_j,
//     theta_{j+2} = (P_{j+1} + sqrt d)/Q_j * theta_{j+1}.
// The generator is kept in (O_K/2O_K)* = F_4* = Z/3 (Appendix A): the factor
// (P_{j+1}+sqrt d)/Q_j = [(P_{j+1}-1)/2 + omega] * [Q_j/2]^(-1) with Q_j/2 odd
// is omega (log 1) when P_{j+1} == 1 (mod 4) and omega + 1 = omega^2 (log 2)
// when P_{j+1} == 3 (mod 4).  eps_d == 1 (mod 2O_K) iff the logs over one
// period sum to 0 mod 3.
//
// Arithmetic: for d < 2^44 every quantity of a reduced state (P, Q, P + s with
// s = floor(sqrt d), q Q, Q_{j+1} - Q_{j-1}) is an integer below 2^23, so the
// walk runs in fp32 registers with every operation exact:
//   * q from a hardware reciprocal estimate: 2^23 + floor(num * rcp(Q) - 1/2)
//     by one FMA rounded toward -inf.  rcp.approx has at most 1 ulp error, so
//     |num*rcp(Q) - num/Q| < num/Q * 2^-23 < 1/2 and the estimate is q or q-1;
//     one compare of the remainder against Q corrects it.
//   * Q_{j+1} by the recurrence Q_{j+1} = Q_{j-1} + q_j (P_j - P_{j+1}),
//     which follows from Q_j Q_{j+1} = d - P_{j+1}^2 and Q_{j-1} Q_j = d - P_j^2
//     (no division, no 64-bit product).
//   * P is carried as P + 2^23, so the float's low mantissa bits are P itself
//     and P mod 4 is one AND on the bit pattern.
//
// Fast quotient (d < kFastDLimit): the walk carries num' = P + s + 1/2, so
// num'/Q = q + (r + 1/2)/Q lies at least 1/(2Q) from every integer.  With
// |rcp(Q) - 1/Q| <= 2^-23 / Q the product num' * rcp(Q) errs by less than
// num' 2^-23 / Q < 1/(2Q) while num' < 2^22, so one FMA rounded toward -inf
// onto 2^23 gives 2^23 + q exactly and no correction is needed.  The
// remainder comes out as r + 1/2, and P' + 2^23 = (s + 2^23) - (r + 1/2)
// rounded up (the exact value is the half-integer P' + 2^23 - 1/2).
//
// Half period: the P's and Q's of one period are palindromic,
// Q_j = Q_{l-j} and P_j = P_{l+1-j}; the walk stops at the centre, which is
// the first j with Q_{j+1} = Q_j (l = 2j+1) or P_{j+1} = P_j (l = 2j), the
// test of Algorithm 1.  With S_j = sum_{i<=j} log(P_i):
//   l = 2j+1: log eps = 2 S_j + log(P_{j+1});   l = 2j: log eps = 2 S_j.
#pragma once

#include <cmath>
#include <cstdint>
#include <cstring>
#include <cuda_runtime.h>

namespace eis {

constexpr int kTileCands = 1 << 16;          // candidates per sieve tile
constexpr int kTileWords = kTileCands / 32;  // bitmap words per tile
constexpr int kPlainBlockCands = 1 << 21;    // 2^24-wide block of d = 2^21 candidates
constexpr float kMagic = 8388608.0f;         // 2^23
constexpr unsigned kFull = 0xffffffffu;

// One interval of a plan, in the plan's candidate layout.
struct Seg {
    uint64_t d0;     // first candidate d (== 5 mod 8)
    uint64_t ncand;  // number of candidates
    uint64_t cand0;  // global index of candidate 0 (multiple of 32)
};

// A sieve / count tile: up to kTileCands consecutive candidates of one Seg.
struct Tile {
    uint64_t cand0;  // global candidate index of the first candidate (multiple of 32)
    uint32_t seg;    // index into the Seg table
    uint32_t ncand;  // candidates in this tile
};

// d below this use the fast quotient: 2 sqrt(d) + 1/2 < 2^22 for every
// d <= (2^21 - 1)^2 = 4398042316801.
constexpr uint64_t kFastDLimit = 4390000000000ull;

// Error codes written by kernels into the plan's status word.
constexpr int kErrSteps = 1;  // a baby walk ran past its step limit
constexpr int kErrGiant = 2;  // a giant-step search failed (table full, no hit)

// Exact small integer <-> float by the 2^23 bit pattern (no conversion
// unit): for 0 <= v < 2^23, the float with bits 0x4B000000 | v is 2^23 + v.
__host__ __device__ __forceinline__ float u23_to_float(uint32_t v) {
    uint32_t b = 0x4B000000u | v;
    float f;
    memcpy(&f, &b, 4);
    return f - 8388608.0f;
}

// floor(sqrt(d)) for d < 2^44 in fp32 and 64-bit integers, without the FP64
// unit.  float(d) is formed exactly rounded from two 22-bit halves (one
// rounding, in the FMA); sqrt(float(d)) differs from sqrt(d) by less than
// sqrt(d) 2^-25 <= 1/8 plus the IEEE square root's rounding (a quarter ulp
// at most 1/8 here), so its floor is floor(sqrt d) or one off, and one
// integer correction each way makes it exact.
__host__ __device__ __forceinline__ uint64_t isqrt44(uint64_t d) {
    const float hi = u23_to_float((uint32_t)(d >> 22));
    const float lo = u23_to_float((uint32_t)(d & 0x3FFFFFu));
#ifdef __CUDA_ARCH__
    const float fd = __fmaf_rn(hi, 4194304.0f, lo);
    const float r = __fsqrt_rn(fd);
    const float fl = __fadd_rd(r, 8388608.0f);  // 2^23 + floor(r), r < 2^22
#else
    const float fd = std::fma(hi, 4194304.0f, lo);
    const float r = std::sqrt(fd);
    float fl;
    {
        const float t = std::floor(r);
        fl = t + 8388608.0f;  // exact: t < 2^22
    }
#endif
    uint32_t bits;
    memcpy(&bits, &fl, 4);
    uint64_t s = bits & 0x7FFFFFu;
    if (s * s > d) --s;
    if ((s + 1) * (s + 1) <= d) ++s;
    return s;
}

// Square-free test of one d (d == 5 mod 8, d < 2^44) by one warp, without
// division: for odd m, m | d iff d * m^(-1) mod 2^64 <= floor((2^64-1)/m)
// (Granlund & Montgomery, "Division by invariant integers using
// multiplication", PLDI 1994, section 9).  sqtab[2i] = (p_i^2)^(-1) mod 2^64,
// sqtab[2i+1] = floor((2^64-1)/p_i^2) for the odd primes p_i (ascending);
// the primes with p^2 <= d are found by binary search.
__device__ __forceinline__ bool warp_squarefree_fast(uint64_t d, const uint32_t *__restrict__ primes,
                                                     const uint64_t *__restrict__ sqtab,
                                                     uint32_t nprimes) {
    uint32_t lo = 0, hi = nprimes;  // count of primes with p^2 <= d
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        const uint64_t p = primes[mid];
        if (p * p <= d) lo = mid + 1; else hi = mid;
    }
    bool hit = false;
    for (uint32_t i = threadIdx.x & 31; i < lo; i += 32) {
        const uint64_t inv = sqtab[2 * i], lim = sqtab[2 * i + 1];
        hit |= d * inv <= lim;
    }
    return !__any_sync(0xffffffffu, hit);
}

__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

struct WalkState {
    float Pm;    // P_j + 2^23
    float Q;     // Q_j
    float Qp;    // Q_{j-1}
    float soff;  // s - 2^23
    float sm;    // s + 2^23
    int acc2;    // 2 S_j (sum of 2*log over the states walked), not reduced
};

// An idle state for lanes without a d: every quantity is NaN, so both centre
// tests of walk_step compare false and the lane never reports a centre.
__device__ __forceinline__ void walk_park_idle(WalkState &w) {
    const float nan = __int_as_float(0x7fffffff);
    w.Pm = nan;
    w.Q = nan;
    w.Qp = nan;
    w.soff = nan;
    w.sm = nan;
    w.acc2 = 0;
}

// First step from (P_0, Q_0) = (1, 2) in 64-bit integers: q_0 = floor((1+s)/2),
// P_1 = 2 q_0 - 1, Q_1 = (d - P_1^2)/2.  Returns true when the period is 1
// (Q_1 = Q_0 = 2), with *g = log eps_d; otherwise leaves the state at j = 1.
template <bool kFast>
__device__ __forceinline__ bool walk_init(uint64_t d, WalkState &w, int &g) {
    const uint64_t s = isqrt44(d);
    const uint64_t a0 = (1 + s) >> 1;
    const uint64_t P1 = 2 * a0 - 1;
    const uint64_t Q1 = (d - P1 * P1) >> 1;
    const int c1 = 1 + (int)((P1 >> 1) & 1);  // log of (P_1 + sqrt d)/2 mod 2
    if (Q1 == 2) {
        g = c1;
        return true;
    }
    w.Pm = __fadd_rn(__uint2float_rn((uint32_t)P1), kMagic);
    w.Q = __uint2float_rn((uint32_t)Q1);
    w.Qp = 2.0f;
    const float sf = __uint2float_rn((uint32_t)s);
    w.soff = kFast ? __fsub_rn(__fadd_rn(sf, 0.5f), kMagic)   // s + 1/2 - 2^23
                   : __fsub_rn(sf, kMagic);                    // s - 2^23
    w.sm = __fadd_rn(sf, kMagic);
    w.acc2 = 2 * c1;
    return false;
}

// One baby step j -> j+1.  Always advances the state and adds
// 2 log(P_{j+1}) = 2 + 2[P_{j+1} == 3 mod 4] to acc2; returns true when the
// new state is the centre of the period (Q_{j+1} = Q_j or P_{j+1} = P_j).
template <bool kFast>
__device__ __forceinline__ bool walk_step(WalkState &w) {
    float qf, Pn;
    if (kFast) {
        const float num = __fadd_rn(w.Pm, w.soff);            // P_j + s + 1/2
        const float rq = rcp_approx(w.Q);
        const float qm = __fmaf_rd(num, rq, kMagic);          // 2^23 + q exactly
        qf = __fsub_rn(qm, kMagic);
        const float r = __fmaf_rn(-qf, w.Q, num);             // r + 1/2
        Pn = __fsub_ru(w.sm, r);                              // P_{j+1} + 2^23
    } else {
        const float num = __fadd_rn(w.Pm, w.soff);            // P_j + s
        const float rq = rcp_approx(w.Q);
        const float qm = __fmaf_rd(num, rq, kMagic - 0.5f);   // 2^23 + (q or q-1)
        qf = __fsub_rn(qm, kMagic);
        float r = __fmaf_rn(-qf, w.Q, num);                   // remainder, in [0, 2Q)
        if (r >= w.Q) {
            r = __fsub_rn(r, w.Q);
            qf = __fadd_rn(qf, 1.0f);                         // q_j
        }
        Pn = __fsub_rn(w.sm, r);                              // P_{j+1} + 2^23 = s - r + 2^23
    }
    const float dP = __fsub_rn(w.Pm, Pn);                     // P_j - P_{j+1}
    const float Qn = __fmaf_rn(qf, dP, w.Qp);                 // Q_{j+1}
    w.acc2 += 2 + (__float_as_int(Pn) & 2);
    const bool centre = (Qn == w.Q) | (dP == 0.0f);
    w.Qp = w.Q;
    w.Q = Qn;
    w.Pm = Pn;
    return centre;
}

// log eps_d (mod 3, in 0..2) once walk_step has returned true.  The centre
// is of odd type (l = 2j+1) iff the last two Q are equal, else of even type.
__device__ __forceinline__ int walk_finish(const WalkState &w) {
    const int t = __float_as_int(w.Pm) & 2;
    const int g = (w.Q == w.Qp) ? (w.acc2 - 1 - (t >> 1)) : (w.acc2 - 2 - t);
    return g % 3;
}

// ---------------------------------------------------------------- lean walk
// The persistent walk's state.  P_j is carried only inside num = P_j + s
// (+ 1/2 on the fast path): the next num is C - r with C = 2s (+1) and r the
// remainder (+ 1/2), and num - num' = P_j - P_{j+1}.  The class bit
// x_j = [P_j == 3 mod 4] follows from P_{j+1} = q_j Q_j - P_j with
// Q_j == 2 (mod 4): x_{j+1} = 1 xor (q_j mod 2) xor x_j, where q_j mod 2 is
// the low bit of the quotient in 2^23 + q form.  Six FMA-pipe instructions,
// one MUFU.RCP, two compares and one LOP3 per step.
struct LeanState {
    float num;  // P_j + s (+ 1/2 when kFast)
    float Q;    // Q_j
    float Qp;   // Q_{j-1}
    int x;      // [P_j == 3 mod 4]
    int acc;    // 1 + x_1 + sum of x over the steps taken (the 1 per step apart)
};

// Idle lanes: NaN everywhere, so both centre tests compare false.
__device__ __forceinline__ void lean_park_idle(LeanState &w, float &C) {
    const float nan = __int_as_float(0x7fffffff);
    w.num = nan;
    w.Q = nan;
    w.Qp = nan;
    w.x = 0;
    w.acc = 0;
    C = nan;
}

// First step from (P_0, Q_0) = (1, 2) in 64-bit integers, as walk_init.
// Returns true when the period is 1, with *g = log eps_d.
template <bool kFast>
__device__ __forceinline__ bool lean_init(uint64_t d, LeanState &w, float &C, int &g) {
    const uint64_t s = isqrt44(d);
    const uint64_t a0 = (1 + s) >> 1;
    const uint64_t P1 = 2 * a0 - 1;
    const uint64_t Q1 = (d - P1 * P1) >> 1;
    const int x1 = (int)((P1 >> 1) & 1);
    if (Q1 == 2) {
        g = 1 + x1;
        return true;
    }
    const uint32_t s2 = 2 * (uint32_t)s;
    w.num = kFast ? __fadd_rn(__uint2float_rn((uint32_t)(P1 + s)), 0.5f)
                  : __uint2float_rn((uint32_t)(P1 + s));
    w.Q = __uint2float_rn((uint32_t)Q1);
    w.Qp = 2.0f;
    w.x = x1;
    w.acc = 1 + x1;
    C = __uint2float_rn(kFast ? s2 + 1 : s2);
    return false;
}

// One step j -> j+1 (acc is left to the caller).  Returns true when the new
// state is the centre of the period (Q_{j+1} = Q_j or P_{j+1} = P_j).
template <bool kFast>
__device__ __forceinline__ bool lean_step(LeanState &w, float C) {
    const float rq = rcp_approx(w.Q);
    float qm, qf, r;
    if (kFast) {
        qm = __fmaf_rd(w.num, rq, kMagic);        // 2^23 + q exactly
        qf = __fsub_rn(qm, kMagic);
        r = __fmaf_rn(-qf, w.Q, w.num);           // remainder + 1/2
    } else {
        qm = __fmaf_rd(w.num, rq, kMagic - 0.5f); // 2^23 + (q or q-1)
        qf = __fsub_rn(qm, kMagic);
        r = __fmaf_rn(-qf, w.Q, w.num);           // remainder, in [0, 2Q)
        if (r >= w.Q) {
            r = __fsub_rn(r, w.Q);
            qf = __fadd_rn(qf, 1.0f);
            qm = __fadd_rn(qm, 1.0f);
        }
    }
    const float numn = __fsub_rn(C, r);           // P_{j+1} + s (+ 1/2)
    const float dP = __fsub_rn(w.num, numn);      // P_j - P_{j+1}
    const float Qn = __fmaf_rn(qf, dP, w.Qp);     // Q_{j+1}
    w.x = ~(w.x ^ __float_as_int(qm)) & 1;
    const bool centre = (Qn == w.Q) | (dP == 0.0f);
    w.Qp = w.Q;
    w.Q = Qn;
    w.num = numn;
    return centre;
}

// log eps_d (mod 3) at a centre reached after `steps` steps from state 1:
// S_j = acc + steps, and the odd / even centre rules of walk_finish.
__device__ __forceinline__ int lean_finish(const LeanState &w, uint32_t steps) {
    const int S = w.acc + (int)(steps % 3);
    const int g = (w.Q == w.Qp) ? (2 * S - 1 - w.x) : (2 * S - 2 - 2 * w.x);
    return g % 3;
}

// Candidate index -> d by binary search over Segs sorted by cand0.
__device__ __forceinline__ uint64_t cand_to_d(const Seg *__restrict__ segs, uint32_t nseg,
                                              uint64_t cand) {
    uint32_t lo = 0, hi = nseg;  // find the last seg with cand0 <= cand
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (segs[mid].cand0 <= cand) lo = mid; else hi = mid;
    }
    return segs[lo].d0 + 8 * (cand - segs[lo].cand0);
}

// Block-wide sum of one value per thread (valid in thread 0).
__device__ __forceinline__ uint32_t block_sum(uint32_t v, uint32_t *red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    uint32_t s = 0;
    if (threadIdx.x < 32) {
        s = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
    }
    return s;  // valid in thread 0
}

// Exclusive block scan of one value per thread; returns the prefix and
// writes the block total to *total (all threads).
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *red, uint32_t *total) {
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    uint32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, x, o);
        if (l >= o) x += y;
    }
    __syncthreads();
    if (l == 31) red[w] = x;
    __syncthreads();
    if (w == 0) {
        uint32_t s = (l < nw) ? red[l] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, s, o);
            if (l >= o) s += y;
        }
        if (l < nw) red[l] = s;  // inclusive scan of warp totals
    }
    __syncthreads();
    const uint32_t warp_prefix = (w > 0) ? red[w - 1] : 0;
    *total = red[nw - 1];
    return warp_prefix + x - v;
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

}  // namespace eis
