// eis_bsgs.cuh -- the lane-per-d infrastructure search of the batch path
// (Algorithm 1 with a sparse baby table), shared by the kernels and the host
// model of the tests.
//
// Marked states.  A state (P_j, Q_j) of the principal cycle is marked when
// Q_j < T, T = tau * floor(sqrt d) in fp32 (about 1 state in 1.39/tau: the
// reduced Q / sqrt(d) are close to uniform near 0).  The mark depends on Q
// alone, and Q_j = Q_{l-j} (the cycle is palindromic), so the mirror of a
// marked state is marked.
//
// Baby table.  The baby walk a_1 .. a_N records every marked state j as
// (Q_j, P_j, S_j), S_j the generator class of a_j in Z/3 (Appendix A), plus
// entry 0 = (2, P_1, 0), which is a_l = O_K again (Q_l = Q_0 = 2,
// P_l = P_1).  jl is the last marked state recorded.
//
// Giant steps.  G = a_jl.  mu starts at G; every cycle sets
// mu <- reduce(mu * G) (textbook composition or NUCOMP, eis_infra.cuh) and
// then walks baby steps from mu, looking up every marked state x it passes
// under two keys:
//   direct  (Q_x, P_x)     = entry j  ->  x = l + j, log eps = g_x - S_j;
//   mirror  (Q_x, P_{x+1}) = entry j  ->  x = l - j, log eps = g_x + S_j
// ((Q_x, P_{x+1}) is state l - x, because P_i = P_{l+1-i}).  A cycle's walk
// lasts at least until it has passed one marked state and looked it up under
// both keys; the next composition starts from wherever the walk stopped.
//
// Why the first hit is in the first period.  Every marked state at position
// l - jl .. l + jl is in the table (directly or as a mirror).  A walk that
// starts inside that window meets a marked state before leaving it (l and
// l + jl are marked); a walk that starts before it and reaches it passes the
// marked position l - jl.  Between the end of one walk and the next landing
// lies one composition with G, a distance delta_jl + kappa, kappa the
// reduction's offset (|kappa| below about log(2 sqrt d)), which is shorter
// than the window's width 2 delta_jl - (one step) once delta_jl exceeds a
// few dozen, so no gap can hold the whole window.  Walks only move forward
// from position jl on, so a direct key cannot match a baby position
// (j <= jl) in the first period.  Hence the first hit is at l - j or l + j.
#pragma once

#include <cstdint>
#include <cstring>

#include "eis_infra.cuh"

namespace eis {

constexpr int kBsgsKmax = 128;            // table entries per d, entry 0 included
constexpr int kBsgsSlots = 256;           // hash slots per d (u8 entry index, 0xFF = empty)
constexpr int kBsgsMinJl = 256;           // a d is searched only if its last marked state
                                          // is at least this far in (window margin)
constexpr uint32_t kBsgsEntryBytes = 16;
constexpr uint32_t kBsgsRegionBytes = kBsgsKmax * kBsgsEntryBytes + kBsgsSlots;  // 2304

// One baby-table entry: the fp32 bit patterns of Q_j and of num_j = P_j + s
// (+ 1/2 on the fast path, as the walk carries it), and S_j (reduced mod 3
// by the reader).
struct DEntry {
    uint32_t q;
    uint32_t num;
    uint32_t s;
    uint32_t pad;
};

// A deferred d handed from the baby walk to the giant-step kernel.
struct DRecord {
    uint32_t cand;    // candidate index in the plan layout
    uint32_t k;       // entries in the table (entry k-1 is G = a_jl)
    uint32_t region;  // table region index in the pool
    uint32_t pad;
};

EIS_HD uint32_t float_bits(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    return u;
}

EIS_HD float bits_float(uint32_t u) {
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

// The marking threshold T = tau * s in fp32, rounded to nearest (the same
// single product on the host and the device).
EIS_HD float bsgs_threshold(float tau, uint64_t s) { return tau * (float)(uint32_t)s; }

// num as the walk carries it: P + s + 1/2 (fast quotient) or P + s.
EIS_HD float bsgs_num(int64_t P, int64_t s, bool fast) {
    const float v = (float)(uint32_t)(P + s);
    return fast ? v + 0.5f : v;
}

EIS_HD uint32_t bsgs_slot(uint32_t q, uint32_t num) {
    uint32_t h = q * 0x9E3779B1u ^ num * 0x85EBCA6Bu;
    h ^= h >> 15;
    return (h * 0x2C1B3C6Du) >> 24;
}

// Open-addressing index of the k entries (linear probing; k < kBsgsSlots).
EIS_HD void bsgs_index(const DEntry *e, int k, uint8_t *slots) {
    for (int i = 0; i < kBsgsSlots; ++i) slots[i] = 0xFF;
    for (int i = 0; i < k; ++i) {
        uint32_t p = bsgs_slot(e[i].q, e[i].num);
        while (slots[p] != 0xFF) p = (p + 1) & (kBsgsSlots - 1);
        slots[p] = (uint8_t)i;
    }
}

// Entry index of the key (q, num), or -1.
EIS_HD int bsgs_find(const DEntry *e, const uint8_t *slots, uint32_t q, uint32_t num) {
    uint32_t p = bsgs_slot(q, num);
    for (int n = 0; n < kBsgsSlots; ++n) {
        const uint32_t i = slots[p];
        if (i == 0xFF) return -1;
        if (e[i].q == q && e[i].num == num) return (int)i;
        p = (p + 1) & (kBsgsSlots - 1);
    }
    return -1;
}

// mu * G reduced, with Q_{-1} = (d - P^2)/Q of the result (the state before
// it on the cycle), by the textbook composition (compose = 0) or NUCOMP (1).
EIS_HD bool bsgs_giant(int compose, const Ideal &mu, const Ideal &G, int64_t d, int64_t s,
                       int64_t L, Ideal &out, int64_t &Qm) {
    const bool ok = compose ? ideal_mul_nucomp(mu, G, d, s, L, out) : ideal_mul(mu, G, d, s, out);
    if (!ok) return false;
    Qm = exact_quot(d, out.b, 2 * out.a);
    return true;
}

}  // namespace eis
