// eis_infra.cuh -- infrastructure giant steps (Algorithm 1) with the
// generator kept in (O_K/2O_K)* = Z/3 (Appendix A).
//
// An ideal is [a, (b + sqrt d)/2] with a = Q/2 > 0 odd and b odd, plus the
// class g in Z/3 of the generator it was reached with.
//
// Composition: the product of two primitive ideals is e [a3, (b3+sqrt d)/2]
// with e odd (it divides a1), so the primitive part's generator class is
// g1 + g2.  (a3, b3) follow the textbook form-composition algorithm; every
// product is reduced modulo v1 = a1/e first, so all values stay in int64 for
// d < 2^44.
//
// Reduction applies rho (Appendix A) until the ideal is reduced:
// q = floor((P + sqrt d)/Q) = floor((P + s)/Q) for Q > 0 and
// floor((P + s + 1)/Q) for Q < 0 (s = floor(sqrt d)), P' = qQ - P,
// Q' = (d - P'^2)/Q, and the class gains log((P'-1)/2 + omega) mod 2, which
// is 1 when P' == 1 (mod 4) and 2 when P' == 3 (mod 4) (Q/2 odd, sign +-1
// == 1 mod 2).  Q_{-1} = (d - P^2)/Q is found once, by exact division: P^2
// can exceed 2^64, but the quotient is below 2^62, so with Q = 2a,
// ((d - P^2) mod 2^64) >> 1 = a Q_{-1} (mod 2^63), times the inverse of a
// modulo 2^64 (Newton iteration x <- x(2 - a x)).  Every step after that
// uses Q' = Q_{-1} + q (P - P') (from Q_{-1} Q = d - P^2 and P + P' = qQ),
// with no division; q(P - P') = Q' - Q_{-1} stays below 2^47.
//
// Reduced: Q > 0, 0 < P <= s and s - P < Q <= s + P (sqrt d irrational).
#pragma once

#include <cstdint>

#include "eis_common.cuh"

namespace eis {

// The ideal arithmetic below is plain integer code that also compiles for
// the host, where tests run it against an exact walk of the cycle.
#define EIS_HD __host__ __device__ __forceinline__

struct Ideal {
    int64_t a;  // Q/2
    int64_t b;  // P
    int g;      // generator class in Z/3
};

// Extended Euclid in 32-bit arithmetic for 0 <= a, b < 2^31 (the ideal norms
// and their half-sums are below 2^23): returns gcd with x a + y b = gcd.
EIS_HD int64_t egcd32(int32_t a, int32_t b, int64_t &x, int64_t &y) {
    int32_t x0 = 1, y0 = 0, x1 = 0, y1 = 1;
    while (b != 0) {
        const int32_t q = a / b;
        int32_t t = a - q * b;
        a = b;
        b = t;
        t = x0 - q * x1;
        x0 = x1;
        x1 = t;
        t = y0 - q * y1;
        y0 = y1;
        y1 = t;
    }
    x = x0;
    y = y0;
    return a;
}

// Extended Euclid: returns gcd(a, b) >= 0 with x a + y b = gcd.  Operands
// below 2^31 in magnitude take the 32-bit loop on |a|, |b| (the cofactors'
// signs follow the operands'); the forms' middle coefficients are negative.
EIS_HD int64_t egcd64(int64_t a, int64_t b, int64_t &x, int64_t &y) {
    const int64_t aa = a < 0 ? -a : a, ab = b < 0 ? -b : b;
    if (aa < 0x7fffffff && ab < 0x7fffffff) {
        const int64_t g = egcd32((int32_t)aa, (int32_t)ab, x, y);
        if (a < 0) x = -x;
        if (b < 0) y = -y;
        return g;
    }
    int64_t x0 = 1, y0 = 0, x1 = 0, y1 = 1;
    while (b != 0) {
        const int64_t q = a / b;
        int64_t t = a - q * b;
        a = b;
        b = t;
        t = x0 - q * x1;
        x0 = x1;
        x1 = t;
        t = y0 - q * y1;
        y0 = y1;
        y1 = t;
    }
    if (a < 0) {
        a = -a;
        x0 = -x0;
        y0 = -y0;
    }
    x = x0;
    y = y0;
    return a;
}

EIS_HD int64_t mod_pos(int64_t x, int64_t m) {
    int64_t r = x % m;
    return r < 0 ? r + m : r;
}

EIS_HD int64_t floor_div(int64_t x, int64_t y) {
    int64_t q = x / y;
    if ((x % y != 0) && ((x < 0) != (y < 0))) --q;
    return q;
}

// floor(x / y) for |x|, |y| < 2^47, y != 0.  The fp32 estimate
// x * rcp(y) has relative error below 2^-21.4 (two conversions, rcp.approx
// and the product), so while it is below 2^20 in magnitude it lies within
// 0.4 of x/y and its floor is q - 1, q or q + 1; one integer correction each
// way fixes it.  Larger quotients take the 64-bit division.
EIS_HD int64_t floor_div_fast(int64_t x, int64_t y) {
#ifdef __CUDA_ARCH__
    const float e = floorf(__fmul_rn((float)x, rcp_approx((float)y)));
#else
    const float e = floorf((float)x * (1.0f / (float)y));  // within the same bound
#endif
    if (fabsf(e) >= 1048576.0f) return floor_div(x, y);
    int64_t q = (int64_t)(int32_t)e;
    const int64_t r = x - q * y;  // floor wants 0 <= r < y (y > 0), y < r <= 0 (y < 0)
    if (y > 0) {
        if (r < 0) --q; else if (r >= y) ++q;
    } else {
        if (r > 0) --q; else if (r <= y) ++q;
    }
    return q;
}

// Inverse of an odd a modulo 2^64.
EIS_HD uint64_t inv_odd_u64(uint64_t a) {
    uint64_t x = a;  // a * a == 1 (mod 8): 3 correct bits
    for (int i = 0; i < 5; ++i) x *= 2 - a * x;
    return x;
}

// Primitive part (a3, b3) of the product of [a1,(b1+sqrt d)/2] and
// [a2,(b2+sqrt d)/2] (both primitive, b odd, 4a | b^2 - d, a < 2^22).
EIS_HD void ideal_compose(int64_t a1, int64_t b1, int64_t a2, int64_t b2,
                          int64_t d, int64_t &a3, int64_t &b3) {
    if (a1 > a2) {
        int64_t t = a1; a1 = a2; a2 = t;
        t = b1; b1 = b2; b2 = t;
    }
    const int64_t s = (b1 + b2) / 2;
    const int64_t n = b2 - s;
    const int64_t c2 = (b2 * b2 - d) / (4 * a2);
    int64_t y1, dd;
    if (a2 % a1 == 0) {
        y1 = 0;
        dd = a1;
    } else {
        int64_t u, v;
        dd = egcd64(a2, a1, u, v);  // u a2 + v a1 = dd
        y1 = u;
    }
    int64_t x2, y2, d1;
    if (s % dd == 0) {
        y2 = -1;
        x2 = 0;
        d1 = dd;
    } else {
        int64_t u, v;
        d1 = egcd64(s, dd, u, v);   // u s + v dd = d1
        x2 = u;
        y2 = -v;
    }
    const int64_t v1 = a1 / d1, v2 = a2 / d1;
    int64_t r = 0;
    if (v1 > 1) {
        const int64_t t1 = mod_pos(mod_pos(y1, v1) * mod_pos(y2, v1), v1) * mod_pos(n, v1);
        const int64_t t2 = mod_pos(x2, v1) * mod_pos(c2, v1);
        r = mod_pos(mod_pos(t1, v1) - mod_pos(t2, v1), v1);
    }
    b3 = b2 + 2 * v2 * r;
    a3 = v1 * v2;
}

EIS_HD bool ideal_is_reduced(int64_t P, int64_t Q, int64_t s) {
    return Q > 0 && P > 0 && P <= s && s - P < Q && Q <= s + P;
}

// (d - P^2) / Q exactly, for Q == 2 (mod 4) dividing d - P^2 and a quotient
// below 2^62 in magnitude.
EIS_HD int64_t exact_quot(int64_t d, int64_t P, int64_t Q) {
    const uint64_t X = (uint64_t)d - (uint64_t)P * (uint64_t)P;  // d - P^2 mod 2^64
    const int64_t ha = Q > 0 ? Q / 2 : -(Q / 2);                   // |Q|/2, odd
    const uint64_t m = ((X >> 1) * inv_odd_u64((uint64_t)ha)) & 0x7fffffffffffffffull;
    const int64_t v = (m & 0x4000000000000000ull) ? (int64_t)(m | 0x8000000000000000ull) : (int64_t)m;
    return Q < 0 ? -v : v;
}

// rho until reduced; returns the class gained, or -1 past max_steps.  P must
// lie within about |Q| + 2^23 of 0 on entry (true of every composition here),
// which keeps Q_{-1} and every later value below 2^47.
EIS_HD int ideal_reduce(int64_t &P, int64_t &Q, int64_t d, int64_t s,
                        int max_steps) {
    if (ideal_is_reduced(P, Q, s)) return 0;
    int g = 0;
    int64_t Qm = exact_quot(d, P, Q);  // Q_{-1}
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

// reduce(X * Y) with classes; returns false if the reduction ran away.
EIS_HD bool ideal_mul(const Ideal &X, const Ideal &Y, int64_t d, int64_t s,
                      Ideal &out) {
    int64_t a3, b3;
    ideal_compose(X.a, X.b, Y.a, Y.b, d, a3, b3);
    int64_t P = b3, Q = 2 * a3;
    const int gr = ideal_reduce(P, Q, d, s, 256);
    if (gr < 0) return false;
    out.a = Q / 2;
    out.b = P;
    out.g = (X.g + Y.g + gr) % 3;
    return true;
}

// ---------------------------------------------------------------- NUCOMP
// Algorithms 2-4 (NUCOMP, NUDUPL, NUCOMPchoose) on forms (u, v, w) with
// v^2 - 4uw = d; the ideal [Q/2, (P+sqrt d)/2] is the form (Q/2, -P, w),
// w = (P^2 - d)/(2Q).  The output ideal I = (1/gamma) I1 I2 is near-reduced,
// so one or two rho steps finish the reduction.  Its generator class is
// g1 + g2 - log(gamma mod 2O_K): gamma = (A + B sqrt d)/C is a unit at 2
// (Appendix A: 1/gamma = theta/(theta' theta'') with all three outside 2O_K);
// gamma C = (A - B) + 2B omega, and after dividing both coordinates by their
// common power of two (which equals the power of two in C) the parities give
// gamma mod 2O_K.  Only those low bits are needed, so A, B, C are formed in
// wrapping 64-bit arithmetic.

// Trailing zero bits of x != 0.
EIS_HD int ctz64(uint64_t x) {
#ifdef __CUDA_ARCH__
    return __ffsll((long long)x) - 1;
#else
    return __builtin_ctzll(x);
#endif
}

// log_omega of (x + y omega) for (x, y) != (0, 0) mod 2.
EIS_HD int f4_log(int x, int y) { return y ? (x ? 2 : 1) : 0; }
                  
                  EIS_HD int gamma_class(uint64_t A, uint64_t B, uint64_t C, bool &ok) {
    const uint64_t a = A - B, b = 2 * B;
    const int ka = a ? ctz64(a) : 64;
    const int kb = b ? ctz64(b) : 64;
    const int k = ka < kb ? ka : kb;
    const int kc = C ? ctz64(C) : 64;
    if (k != kc || k >= 63) {
        ok = false;
        return 0;
    }
    return f4_log((int)((a >> k) & 1), (int)((b >> k) & 1));
}

// Partial Euclid of NUCOMP/NUDUPL: stops once |by| <= L or bx = 0.  Here
// 0 <= bx < by < 2^31 (by is a norm over a gcd), so the loop runs in 32-bit
// arithmetic; the cofactors x, y stay below by in magnitude.
EIS_HD void nu_partial(int64_t &bx, int64_t &by, int64_t &x, int64_t &y,
                       int &z, int64_t L) {
    x = 1;
    y = 0;
    z = 0;
    if (bx >= 0 && by >= 0 && by < 0x7fffffff) {
        int32_t bx32 = (int32_t)bx, by32 = (int32_t)by, x32 = 1, y32 = 0;
        while (by32 > L && bx32 != 0) {
            const int32_t q = by32 / bx32, t = by32 - q * bx32;
            by32 = bx32;
            bx32 = t;
            const int32_t u = y32 - q * x32;
            y32 = x32;
            x32 = u;
            ++z;
        }
        bx = bx32;
        by = by32;
        x = x32;
        y = y32;
        if (z & 1) {
            by = -by;
            y = -y;
        }
        return;
    }
    while ((by < 0 ? -by : by) > L && bx != 0) {
        const int64_t q = by / bx, t = by - q * bx;  // bx, by >= 0 here
        by = bx;
        bx = t;
        const int64_t u = y - q * x;
        y = x;
        x = u;
        ++z;
    }
    if (z & 1) {
        by = -by;
        y = -y;
    }
}

// NUCOMP (Algorithm 2).  Returns false if a division that must be exact is
// not (never expected).
EIS_HD bool nucomp(int64_t u1, int64_t v1, int64_t w1, int64_t u2, int64_t v2,
                   int64_t w2, int64_t L, int64_t &u3, int64_t &v3,
                   int64_t &w3, uint64_t &A, uint64_t &B, uint64_t &C) {
    if (w1 < w2) {
        int64_t t = u1; u1 = u2; u2 = t;
        t = v1; v1 = v2; v2 = t;
        t = w1; w1 = w2; w2 = t;
    }
    const int64_t s = (v1 + v2) / 2, m = v2 - s;
    int64_t b, c;
    const int64_t F = egcd64(u2, u1, b, c);  // b u2 + c u1 = F
    int64_t G, Bx, By, Cy, Dy;
    if (s % F == 0) {
        G = F;
        Bx = m * b;
        By = u1 / G;
        Cy = u2 / G;
        Dy = s / G;
    } else {
        int64_t xx, yy;
        G = egcd64(F, s, xx, yy);  // xx F + yy s = G
        const int64_t H = F / G;
        By = u1 / G;
        Cy = u2 / G;
        Dy = s / G;
        const int64_t l = mod_pos(mod_pos(yy, H) * mod_pos(mod_pos(b, H) * mod_pos(w1, H) +
                                                        mod_pos(c, H) * mod_pos(w2, H), H), H);
        const int64_t num = b * m + l * By;
        if (num % H) return false;
        Bx = num / H;
    }
    int64_t bx = mod_pos(Bx, By), by = By, x, y;
    int z;
    nu_partial(bx, by, x, y, z, L);
    const int64_t ax = G * x, ay = G * y;
    if (z != 0) {
        const int64_t n1 = Cy * bx - m * x;
        if (n1 % By) return false;
        const int64_t cx = n1 / By;
        const int64_t Q1 = by * cx, Q2 = Q1 + m;
        const int64_t n2 = Dy * bx - w2 * x;
        if (n2 % By) return false;
        const int64_t dx = n2 / By;
        const int64_t Q3 = y * dx, Q4 = Q3 + Dy;
        if (Q4 % x) return false;
        const int64_t dy = Q4 / x;
        int64_t cy;
        if (bx != 0) {
            if (Q2 % bx) return false;
            cy = Q2 / bx;
        } else {
            const int64_t n3 = cx * dy - w1;
            if (n3 % dx) return false;
            cy = n3 / dx;
        }
        u3 = by * cy - ay * dy;
        w3 = bx * cx - ax * dx;
        v3 = G * (Q3 + Q4) - Q1 - Q2;
    } else {
        const int64_t Q1 = Cy * bx;
        if ((Q1 - m) % By || (bx * Dy - w2) % By) return false;
        const int64_t cx = (Q1 - m) / By, dx = (bx * Dy - w2) / By;
        u3 = by * Cy;
        w3 = bx * cx - G * dx;
        v3 = v2 - 2 * Q1;
    }
    const uint64_t t = 2 * (uint64_t)u3;
    A = (uint64_t)G * ((uint64_t)x * t + (uint64_t)y * (uint64_t)v3);
    B = (uint64_t)G * (uint64_t)y;
    C = t;
    return true;
}

// NUDUPL (Algorithm 3).
EIS_HD bool nudupl(int64_t u, int64_t v, int64_t w, int64_t L, int64_t &u3,
                   int64_t &v3, int64_t &w3, uint64_t &A, uint64_t &B,
                   uint64_t &C) {
    int64_t xx, yy;
    const int64_t G = egcd64(u, v, xx, yy);  // xx u + yy v = G
    const int64_t By = u / G, Dy = v / G;
    int64_t bx = mod_pos(mod_pos(yy, By) * mod_pos(w, By), By), by = By, x, y;
    int z;
    nu_partial(bx, by, x, y, z, L);
    const int64_t ax = G * x, ay = G * y;
    if (z == 0) {
        const int64_t n = bx * Dy - w;
        if (n % By) return false;
        const int64_t dx = n / By;
        u3 = by * by;
        w3 = bx * bx;
        v3 = v - (bx + by) * (bx + by) + u3 + w3;
        w3 = w3 - G * dx;
    } else {
        const int64_t n = bx * Dy - w * x;
        if (n % By) return false;
        const int64_t dx = n / By;
        const int64_t Q1 = dx * y;
        int64_t dy = Q1 + Dy;
        v3 = G * (dy + Q1);
        if (dy % x) return false;
        dy = dy / x;
        u3 = by * by;
        w3 = bx * bx;
        v3 = v3 - (bx + by) * (bx + by) + u3 + w3;
        u3 = u3 - ay * dy;
        w3 = w3 - ax * dx;
    }
    const uint64_t t = 2 * (uint64_t)u3;
    A = (uint64_t)G * ((uint64_t)x * t + (uint64_t)y * (uint64_t)v3);
    B = (uint64_t)G * (uint64_t)y;
    C = t;
    return true;
}

// NUCOMPchoose (Algorithm 4) + reduction: reduce(X * Y) with classes.
EIS_HD bool ideal_mul_nucomp(const Ideal &X, const Ideal &Y, int64_t d,
                             int64_t s, int64_t L, Ideal &out) {
    int64_t u1 = 2 * X.a, u2 = 2 * Y.a;  // Q (positive for reduced ideals)
    int64_t v1 = mod_pos(X.b, u1), v2 = mod_pos(Y.b, u2);
    int64_t P, Q;
    int lg = 0;
    if (u1 <= 50 || u2 <= 50) {
        int64_t a3, b3;
        ideal_compose(X.a, X.b, Y.a, Y.b, d, a3, b3);  // gamma = content, odd
        P = b3;
        Q = 2 * a3;
    } else {
        const int64_t w1 = (v1 * v1 - d) / (2 * u1);
        int64_t u3, v3, w3;
        uint64_t A, B, C;
        bool ok;
        if (u1 == u2 && v1 == v2) {
            ok = nudupl(u1 / 2, -v1, w1, L, u3, v3, w3, A, B, C);
        } else {
            const int64_t w2 = (v2 * v2 - d) / (2 * u2);
            ok = nucomp(u1 / 2, -v1, w1, u2 / 2, -v2, w2, L, u3, v3, w3, A, B, C);
        }
        if (!ok) return false;
        bool okg = true;
        lg = gamma_class(A, B, C, okg);
        if (!okg) return false;
        Q = 2 * (u3 < 0 ? -u3 : u3);
        P = mod_pos(-v3, Q);
    }
    const int gr = ideal_reduce(P, Q, d, s, 256);
    if (gr < 0) return false;
    out.a = Q / 2;
    out.b = P;
    out.g = (X.g + Y.g + 3 - lg + gr) % 3;
    return true;
}

// ---------------------------------------------------------------- baby table
// Open-addressing hash in shared memory, one per warp, written by lane 0 only.
// Entry: key (Q << 24 | P) << 3 | type << 2 | class, 0 = empty.
constexpr uint64_t kMirror = 1;

__device__ __forceinline__ uint64_t infra_key(int64_t Q, int64_t P) {
    return ((uint64_t)Q << 24) | (uint64_t)P;
}

__device__ __forceinline__ uint32_t infra_hash(uint64_t key, int log2n) {
    return (uint32_t)((key * 0x9E3779B97F4A7C15ull) >> (64 - log2n));
}

__device__ __forceinline__ bool infra_insert(uint64_t *tab, int log2n, uint64_t key, uint64_t type,
                                             int cls) {
    const uint32_t mask = (1u << log2n) - 1;
    uint32_t h = infra_hash(key, log2n);
    for (uint32_t i = 0; i <= mask; ++i, h = (h + 1) & mask) {
        const uint64_t e = tab[h];
        if (e == 0) {
            tab[h] = (key << 3) | (type << 2) | (uint64_t)cls;
            return true;
        }
        if ((e >> 3) == key) return true;  // already present (same ideal)
    }
    return false;
}

// The same insert for several lanes of a warp at once (compare-and-swap on
// the slot, so two lanes never claim one empty slot).
__device__ __forceinline__ bool infra_insert_cas(uint64_t *tab, int log2n, uint64_t key,
                                                 uint64_t type, int cls) {
    const uint32_t mask = (1u << log2n) - 1;
    const unsigned long long val = (key << 3) | (type << 2) | (uint64_t)cls;
    uint32_t h = infra_hash(key, log2n);
    for (uint32_t i = 0; i <= mask; ++i, h = (h + 1) & mask) {
        const unsigned long long e =
            atomicCAS(reinterpret_cast<unsigned long long *>(tab + h), 0ull, val);
        if (e == 0) return true;
        if ((e >> 3) == key) return true;
    }
    return false;
}

// Returns the entry for key, or 0.
__device__ __forceinline__ uint64_t infra_find(const uint64_t *tab, int log2n, uint64_t key) {
    const uint32_t mask = (1u << log2n) - 1;
    uint32_t h = infra_hash(key, log2n);
    for (uint32_t i = 0; i <= mask; ++i, h = (h + 1) & mask) {
        const uint64_t e = tab[h];
        if (e == 0) return 0;
        if ((e >> 3) == key) return e;
    }
    return 0;
}

}  // namespace eis
