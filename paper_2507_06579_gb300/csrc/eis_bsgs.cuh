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

#include <cmath>
#include <cstdint>
#include <cstring>

#include "eis_infra.cuh"

namespace eis {

constexpr int kBsgsKmax = 128;            // table entries per d, entry 0 included
constexpr int kBsgsSlots = 256;           // hash slots per d
constexpr int kBsgsMinJl = 256;           // a d is searched only if its last marked state
                                          // is at least this far in (window margin)
constexpr int kBsgsWideGap = 64;          // the wide stride a_jl * a_j' takes the last
                                          // table state j' <= jl - kBsgsWideGap
constexpr uint32_t kBsgsEntryBytes = 16;
constexpr uint32_t kBsgsRegionBytes = kBsgsKmax * kBsgsEntryBytes;  // 2048: the entries

// Per-decade settings of the search, looked up per d: row r covers
// d < d_hi[r] (the last row every larger d as well).  nbaby = 0 walks the d
// to its centre without a table.
constexpr int kTuneRows = 8;
struct TuneTab {
    uint64_t d_hi[kTuneRows];
    uint32_t nbaby[kTuneRows];
    float tau[kTuneRows];  // marking threshold factor: T = tau * floor(sqrt d)
    uint32_t n;
};

EIS_HD int tune_row(const TuneTab &t, uint64_t d) {
    int r = 0;
    while (r + 1 < (int)t.n && d >= t.d_hi[r]) ++r;
    return r;
}

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
    uint32_t s;       // floor(sqrt d)
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


// ------------------------------------------------------------ lean product
// reduce(mu * G) for the search, with every operand of a reduced ideal below
// 2^23 (d < 2^44): the composition of forms (Cohen, "A Course in Computational
// Algebraic Number Theory", Algorithm 5.4.7, with f1 = mu and f2 = G fixed, so
// that c2 = c_G = (b_G^2 - d) / (4 a_G) is computed once per d), its two
// extended Euclid steps in fp32 (every remainder, quotient and cofactor is an
// integer below 2^23, so each operation is exact; quotients come from a
// reciprocal estimate with one correction each way), and the residues mod
// v1 < 2^22 by a float quotient estimate with integer corrections.

// floor(x / y) for integers 0 <= x < 2^23, 0 < y < 2^23 held in floats, and
// the remainder.
EIS_HD float fdivmod(float x, float y, float &rem) {
#ifdef __CUDA_ARCH__
    const float e = __fmaf_rd(x, rcp_approx(y), 8388608.0f) - 8388608.0f;
#else
    const float e = std::floor(x * (1.0f / y));
#endif
    // x rcp(y) lies within (x/y) 2^-22 <= 2 of x/y: at most two corrections
    float q = e;
    float r = x - q * y;  // exact: |q y| <= x + 2y < 2^24
    while (r < 0.0f) {
        q -= 1.0f;
        r += y;
    }
    while (r >= y) {
        q += 1.0f;
        r -= y;
    }
    rem = r;
    return q;
}

// floor(x / y) and the remainder for quotients below 2^22, where the estimate
// is within one of the quotient: one select-based correction each way.
EIS_HD float fdivmod1(float x, float y, float &rem) {
#ifdef __CUDA_ARCH__
    float q = __fmaf_rd(x, rcp_approx(y), 8388608.0f) - 8388608.0f;
#else
    float q = std::floor(x * (1.0f / y));
#endif
    float r = x - q * y;
    const bool lo = r < 0.0f;
    q = lo ? q - 1.0f : q;
    r = lo ? r + y : r;
    const bool hi = r >= y;
    q = hi ? q + 1.0f : q;
    rem = hi ? r - y : r;
    return q;
}

// Extended Euclid on 0 <= A < 2^22, 0 <= B < 2^22 in fp32: returns g = gcd(A, B)
// with xa A + xb B = g.  Unrolled by two so that the pairs (r0, r1),
// (a0, a1), (b0, b1) take turns as dividend and divisor in place; every
// remainder, quotient and cofactor is an integer below 2^22, so each
// operation is exact.  Invariant: a0 A + b0 B = r0, a1 A + b1 B = r1.
EIS_HD float fegcd(float A, float B, float &xa, float &xb) {
    float r0 = A, r1 = B, a0 = 1.0f, a1 = 0.0f, b0 = 0.0f, b1 = 1.0f;
    for (;;) {
        if (r1 == 0.0f) {
            xa = a0;
            xb = b0;
            return r0;
        }
        float rem;
        float q = fdivmod1(r0, r1, rem);
        r0 = rem;
        a0 -= q * a1;  // |q a1| <= B: exact
        b0 -= q * b1;
        if (r0 == 0.0f) {
            xa = a1;
            xb = b1;
            return r1;
        }
        q = fdivmod1(r1, r0, rem);
        r1 = rem;
        a1 -= q * a0;
        b1 -= q * b0;
    }
}

// x mod m in [0, m) for |x| < 2^23, 0 < m < 2^23.
EIS_HD int32_t fmodp(int32_t x, int32_t m) {
    float rem;
    const float ax = (float)(x < 0 ? -x : x);
    fdivmod(ax, (float)m, rem);
    const int32_t r = (int32_t)rem;
    return (x < 0 && r != 0) ? m - r : r;
}

// a b mod m for 0 <= a, b < m < 2^22.
EIS_HD int32_t mulmod22(int32_t a, int32_t b, int32_t m) {
    const int64_t p = (int64_t)a * b;  // < 2^44
#ifdef __CUDA_ARCH__
    const float e = __fmul_rn(__fmul_rn((float)a, (float)b), rcp_approx((float)m));
#else
    const float e = ((float)a * (float)b) * (1.0f / (float)m);
#endif
    // e is within 0.1 + p/m 2^-22 < 1.1 of p/m: the remainder needs at most two
    // corrections each way
    int64_t r = p - (int64_t)e * m;
    while (r < 0) r += m;
    while (r >= m) r -= m;
    return (int32_t)r;
}

// Per-d constant of the lean product: c_G = (b_G^2 - d) / (4 a_G).
EIS_HD int64_t lean_cG(const Ideal &G, int64_t d) { return (G.b * G.b - d) / (4 * G.a); }

// rho steps from (P, Q) with Q_{-1} = Qm until reduced, as ideal_reduce;
// class gained, or -1 past max_steps.
EIS_HD int lean_rho(int64_t &P, int64_t &Q, int64_t &Qm, int64_t s, int max_steps) {
    int g = 0;
    for (int it = 0; !ideal_is_reduced(P, Q, s); ++it) {
        if (it >= max_steps) return -1;
        const int64_t q = Q > 0 ? floor_div_fast(P + s, Q) : floor_div_fast(P + s + 1, Q);
        const int64_t Pn = q * Q - P;
        const int64_t Qn = Qm + q * (P - Pn);
        g += 1 + (int)((Pn >> 1) & 1);
        Qm = Q;
        P = Pn;
        Q = Qn;
    }
    return g;
}

// rho steps until reduced, as ideal_reduce, also returning Q_{-1} of the
// result; class gained, or -1 past max_steps.
EIS_HD int lean_reduce(int64_t &P, int64_t &Q, int64_t &Qm, int64_t d, int64_t s, int max_steps) {
    Qm = exact_quot(d, P, Q);
    return lean_rho(P, Q, Qm, s, max_steps);
}

// reduce(mu * G) and Q_{-1} of the result; false if the reduction ran away.
EIS_HD bool lean_mul(const Ideal &mu, const Ideal &G, int64_t cG, int64_t d, int64_t s, Ideal &out,
                     int64_t &Qm) {
    const int32_t a1 = (int32_t)mu.a, a2 = (int32_t)G.a;
    const int32_t b1 = (int32_t)mu.b, b2 = (int32_t)G.b;
    const int32_t sh = (b1 + b2) / 2, n = b2 - sh;
    float fu, fv;
    const int32_t dd = (int32_t)fegcd((float)a2, (float)a1, fu, fv);  // u a2 + v a1 = dd
    const int32_t y1 = (int32_t)fu;
    int32_t x2 = 0, y2 = -1, d1 = dd;
    if (dd > 1) {
        const int32_t sm = fmodp(sh, dd);
        if (sm != 0) {
            float xs, xd;
            d1 = (int32_t)fegcd((float)sm, (float)dd, xs, xd);  // xs (sh mod dd) + xd dd = d1
            // with sh = (sh mod dd) + k dd: xs sh + (xd - xs k) dd = d1
            x2 = (int32_t)xs;
            y2 = -((int32_t)xd - (int32_t)xs * ((sh - sm) / dd));
        }
    }
    const int32_t v1 = a1 / d1, v2 = a2 / d1;
    int32_t r = 0;
    if (v1 > 1) {
        const int32_t t1 = mulmod22(mulmod22(fmodp(y1, v1), fmodp(y2, v1), v1), fmodp(n, v1), v1);
        int32_t t2 = 0;
        if (x2 != 0) {
            int64_t cm = cG % v1;
            if (cm < 0) cm += v1;
            t2 = mulmod22(fmodp(x2, v1), (int32_t)cm, v1);
        }
        r = t1 - t2;
        if (r < 0) r += v1;
    }
    int64_t P = (int64_t)b2 + 2 * (int64_t)v2 * r;  // in [0, Q + 2^22)
    int64_t Q = 2 * (int64_t)v1 * v2;
    while (P > s) P -= Q;  // the representative in (s - Q, s]: a reduced
                           // product is recognised as it is
    const int gr = lean_reduce(P, Q, Qm, d, s, 256);
    if (gr < 0) return false;
    out.a = Q / 2;
    out.b = P;
    out.g = (mu.g + G.g + gr) % 3;
    return true;
}

// ------------------------------------------------------------ lean NUCOMP
// NUCOMP (Algorithm 2, as ideal_mul_nucomp in eis_infra.cuh) specialised to
// two reduced ideals of a discriminant d < 2^44.  Every coefficient u, v, w
// of a reduced form is below sqrt(d) < 2^22 in magnitude (u |w| = (d - P^2)/4
// with both factors reduced Q's over 2), so both Euclid runs (the gcd of the
// u's and the partial Euclid that stops below L) work on integers below 2^22
// in fp32, exactly, with reciprocal quotient estimates and one select-based
// correction each way.  The closing formulas multiply those small numbers
// into 64-bit values and divide exactly by a small divisor, each quotient
// taken from a float estimate rounded to the nearest integer.  The result is
// near-reduced: about one rho step finishes it, against about six for the
// textbook product.  The third coefficients are passed in: w = -Q_{-1}/2 of
// each ideal, which the walk carries.

// float |v| < 2^22 to the nearest int32, and 0 <= v < 2^23 to float, with no
// conversion instruction
EIS_HD int32_t fl_to_i(float v) { return (int32_t)(float_bits(v + 12582912.0f) - 0x4B400000u); }
EIS_HD float i_to_fl(int32_t v) { return u23_to_float((uint32_t)v); }

// n / dv for dv | n, 0 < |dv| < 2^23: the estimate n rcp(dv) has relative
// error below 2^-22, so while |n / dv| < 2^21 it lies within 1/2 of the
// quotient and rounds to it; one correction each way guards the bound.
// Larger quotients take the 64-bit division.
EIS_HD int64_t exact_div_small(int64_t n, int32_t dv) {
#ifdef __CUDA_ARCH__
    const float e = __fmul_rn((float)n, rcp_approx((float)dv));
#else
    const float e = (float)n * (1.0f / (float)dv);
#endif
    if (!(fabsf(e) < 2097152.0f)) return n / dv;
    int64_t q = (int64_t)fl_to_i(e);  // nearest integer
    const int64_t r = n - q * dv;
    if (r != 0) q += ((r > 0) == (dv > 0)) ? 1 : -1;
    return q;
}

// x mod m in [0, m) for |x| < 2^45, 0 < m < 2^22: x = hi 2^23 + lo, and
// 2^23 mod m = 2 (2^22 mod m) folded once.
EIS_HD int32_t mod_small(int64_t x, int32_t m) {
    const int32_t hi = (int32_t)(x >> 23), lo = (int32_t)(x & 0x7FFFFF);
    int32_t p23 = 2 * fmodp(1 << 22, m);
    p23 = p23 >= m ? p23 - m : p23;
    const int32_t r = mulmod22(fmodp(hi, m), p23, m) + fmodp(lo, m);
    return r >= m ? r - m : r;
}

// log_omega of gamma mod 2O_K from A, B, C mod 2^32 (gamma_class of
// eis_infra.cuh in 32-bit words: C = 2 u3 with |u3| < 2^25 has at most 25
// trailing zeros, so the low 32 bits decide every case alike).
EIS_HD int gamma_class32(uint32_t A, uint32_t B, uint32_t C, bool &ok) {
    const uint32_t a = A - B, b = 2u * B;
#ifdef __CUDA_ARCH__
    const int ka = a ? __ffs((int)a) - 1 : 32, kb = b ? __ffs((int)b) - 1 : 32;
    const int kc = C ? __ffs((int)C) - 1 : 32;
#else
    const int ka = a ? __builtin_ctz(a) : 32, kb = b ? __builtin_ctz(b) : 32;
    const int kc = C ? __builtin_ctz(C) : 32;
#endif
    const int k = ka < kb ? ka : kb;
    if (k != kc || k >= 31) {
        ok = false;
        return 0;
    }
    return f4_log((int)((a >> k) & 1u), (int)((b >> k) & 1u));
}

// reduce(X * Y) by NUCOMP, with Q_{-1} of the result; wX, wY are the forms'
// third coefficients (b^2 - d) / (4a) and L = floor(sqrt(floor(sqrt d))).
// Ideals with a tiny norm, and squares, take the lean textbook product.
EIS_HD bool lean_nucomp(const Ideal &X, int64_t wX, const Ideal &Y, int64_t wY, int64_t d, int64_t s,
                        int64_t L, Ideal &out, int64_t &Qm) {
    int32_t u1 = (int32_t)X.a, v1 = -(int32_t)X.b, w1 = (int32_t)wX;
    int32_t u2 = (int32_t)Y.a, v2 = -(int32_t)Y.b, w2 = (int32_t)wY;
    if (u1 <= 50 || u2 <= 50 || (u1 == u2 && v1 == v2)) return lean_mul(X, Y, wY, d, s, out, Qm);
    if (w1 < w2) {
        int32_t t = u1; u1 = u2; u2 = t;
        t = v1; v1 = v2; v2 = t;
        t = w1; w1 = w2; w2 = t;
    }
    const int32_t sp = (v1 + v2) / 2, m = v2 - sp;  // v1 + v2 is even
    float fb, fc;
    const int32_t F = fl_to_i(fegcd(i_to_fl(u2), i_to_fl(u1), fb, fc));  // b u2 + c u1 = F
    const int32_t b = fl_to_i(fb);
    int32_t G = F, By = u1, Cy = u2, Dy = sp, bx;
    if (F == 1) {
        bx = mulmod22(fmodp(m, By), fmodp(b, By), By);  // Bx = m b mod By
    } else {
        const int32_t spF = fmodp(sp, F);
        if (spF != 0) {
            float xx, yy;
            G = fl_to_i(fegcd(i_to_fl(F), i_to_fl(spF), xx, yy));  // xx F + yy sp == G (mod F)
            const int32_t H = F / G, c = fl_to_i(fc);
            By = u1 / G;
            Cy = u2 / G;
            Dy = sp / G;
            // l = yy (b (w1 mod H) + c (w2 mod H)) mod H; Bx = (b m + l By) / H
            int32_t t = mulmod22(fmodp(b, H), fmodp(w1, H), H) + mulmod22(fmodp(c, H), fmodp(w2, H), H);
            t = t >= H ? t - H : t;
            const int32_t l = mulmod22(fmodp(fl_to_i(yy), H), t, H);
            const int64_t Bx = exact_div_small((int64_t)b * m + (int64_t)l * By, H);
            bx = mod_small(Bx, By);
        } else {
            By = u1 / F;
            Cy = u2 / F;
            Dy = sp / F;
            bx = mulmod22(fmodp(m, By), fmodp(b, By), By);
        }
    }
    // partial Euclid on (By, bx) down to L, cofactors (x, y), z steps
    int32_t by, x, y, z = 0;
    {
        float fby = i_to_fl(By), fbx = i_to_fl(bx), fx = 1.0f, fy = 0.0f;
        const float fL = i_to_fl((int32_t)L);
        while (fby > fL && fbx != 0.0f) {
            float r;
            const float q = fdivmod1(fby, fbx, r);
            fby = fbx;
            fbx = r;
            const float t = fy - q * fx;  // |q x| <= By: exact
            fy = fx;
            fx = t;
            ++z;
        }
        by = fl_to_i(fby);
        bx = fl_to_i(fbx);
        x = fl_to_i(fx);
        y = fl_to_i(fy);
    }
    if (z & 1) {
        by = -by;
        y = -y;
    }
    int64_t u3, v3, w3;
    if (z != 0) {
        const int64_t cx = exact_div_small((int64_t)Cy * bx - (int64_t)m * x, By);
        const int64_t Q1 = (int64_t)by * cx, Q2 = Q1 + m;
        const int64_t dx = exact_div_small((int64_t)Dy * bx - (int64_t)w2 * x, By);
        const int64_t Q3 = (int64_t)y * dx, Q4 = Q3 + Dy;
        const int64_t dy = exact_div_small(Q4, x);
        if (bx == 0 && dx == 0) return false;  // (not expected)
        const int64_t cy = bx != 0 ? exact_div_small(Q2, bx) : (cx * dy - w1) / dx;
        u3 = (int64_t)by * cy - (int64_t)G * y * dy;
        w3 = (int64_t)bx * cx - (int64_t)G * x * dx;
        v3 = (int64_t)G * (Q3 + Q4) - Q1 - Q2;
    } else {
        const int64_t Q1 = (int64_t)Cy * bx;
        const int64_t cx = exact_div_small(Q1 - m, By), dx = exact_div_small((int64_t)bx * Dy - w2, By);
        u3 = (int64_t)by * Cy;
        w3 = (int64_t)bx * cx - (int64_t)G * dx;
        v3 = v2 - 2 * Q1;
    }
    // gamma mod 2O_K from A = G (2 u3 x + v3 y), B = G y, C = 2 u3
    bool ok = true;
    const uint32_t C2 = 2u * (uint32_t)u3;
    const int lg = gamma_class32((uint32_t)G * (C2 * (uint32_t)x + (uint32_t)v3 * (uint32_t)y),
                                 (uint32_t)G * (uint32_t)y, C2, ok);
    if (!ok || u3 == 0) return false;
    // the ideal [|u3|, (-v3 + sqrt d)/2]: P0 = -v3 with Q_{-1} = -2 w3 sign(u3),
    // moved into (s - Q, s] by k Q, which changes Q_{-1} by -k (P0 + P)
    int64_t Q = 2 * (u3 < 0 ? -u3 : u3);
    const int64_t P0 = -v3;
    const int64_t k = floor_div_fast(s - P0, Q);
    int64_t P = P0 + k * Q;
    Qm = (u3 > 0 ? -2 * w3 : 2 * w3) - k * (P0 + P);
    const int gr = lean_rho(P, Q, Qm, s, 256);
    if (gr < 0) return false;
    out.a = Q / 2;
    out.b = P;
    out.g = (X.g + Y.g + 3 - lg + gr) % 3;
    return true;
}

// mu * G reduced, with Q_{-1} = (d - P^2)/Q of the result (the state before
// it on the cycle): the lean textbook product (compose = 0), the lean NUCOMP
// (1), the general textbook code of eis_infra.cuh (2) or its general NUCOMP
// (3), the last two the references the tests compare with.  wmu and wG are
// the forms' third coefficients (b^2 - d)/(4a) (lean_cG), L = floor(sqrt s).
EIS_HD bool bsgs_giant(int compose, const Ideal &mu, int64_t wmu, const Ideal &G, int64_t wG, int64_t d,
                       int64_t s, int64_t L, Ideal &out, int64_t &Qm) {
    if (compose == 0) return lean_mul(mu, G, wG, d, s, out, Qm);
    if (compose == 1) return lean_nucomp(mu, wmu, G, wG, d, s, L, out, Qm);
    const bool ok = compose == 3 ? ideal_mul_nucomp(mu, G, d, s, L, out) : ideal_mul(mu, G, d, s, out);
    if (!ok) return false;
    Qm = exact_quot(d, out.b, 2 * out.a);
    return true;
}

}  // namespace eis
