/*
 * oracle.c -- CPU oracle for Eisenstein discriminants (Breuer & Punch,
 * "Quadratic units and cubic fields").
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).  Plain C99 + POSIX threads,
 * integers only.  Each function cites the passage of the paper it writes
 * out:
 *
 *   Section 1       D = { d > 0 : d == 5 mod 8, d square-free },
 *                   E = { d in D : eps_d == 1 mod 2O_K },
 *                   pi_E(x) = #{ d in E : d <= x },
 *                   O_K = Z[omega], omega = (1+sqrt d)/2,
 *                   eps_d = (x0 + y0 sqrt d)/2, 2 inert in K.
 *   Lemma 1.1       (i) eps == 1 mod 2O_K  <=> (ii) no odd solution of
 *                   x^2 - d y^2 = 4  <=> (iv) #Cl(Z[sqrt d]) = 3 #Cl(O_K).
 *   Appendix A      the baby step rho on [Q_j/2, (P_j+sqrt d)/2]:
 *                   q_j = floor((P_j+sqrt d)/Q_j), P_{j+1} = q_j Q_j - P_j,
 *                   Q_{j+1} = (d - P_{j+1}^2)/Q_j,
 *                   theta_{j+2} = (P_{j+1}+sqrt d)/Q_j * theta_{j+1},
 *                   starting from (Q_0,P_0) = (2,1), theta_1 = 1; generators
 *                   reduced modulo 2O_K (Theorem A.1: never 0 mod 2O_K);
 *                   theta_j = (G_{j-2} + B_{j-2} sqrt d)/2 with G = 2A - B.
 *
 * Nothing here uses the half-period shortcut, the Z/3 logarithm, the
 * recurrence form of Q or any floating point: those are the CUDA path's
 * choices, and the oracle deliberately avoids them.
 */
#define _GNU_SOURCE
#include "oracle.h"

#include <pthread.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

typedef unsigned __int128 u128;

/* ------------------------------------------------------------------ */
/* Integer helpers                                                      */
/* ------------------------------------------------------------------ */

uint64_t orc_isqrt(uint64_t n) {
    /* Integer Newton iteration x <- (x + n/x)/2 from above; stops at
     * floor(sqrt(n)). */
    if (n < 2) return n;
    uint64_t x = n, y;
    for (;;) {
        uint64_t q = n / x;
        y = (x >> 1) + (q >> 1) + (x & q & 1); /* floor((x + q)/2), no overflow */
        if (y >= x) return x;
        x = y;
    }
}

int orc_is_squarefree(uint64_t n) {
    /* Definition: no square k^2 > 1 divides n.  Trying every k (not only
     * primes) keeps the test obviously equal to the definition. */
    if (n == 0) return 0;
    for (uint64_t k = 2; k <= n / k; k++) {
        if (n % k == 0 && (n / k) % k == 0) return 0;
    }
    return 1;
}

int orc_is_prime(uint64_t n) {
    /* Definition: n >= 2 with no divisor k, 2 <= k <= sqrt(n). */
    if (n < 2) return 0;
    for (uint64_t k = 2; k <= n / k; k++)
        if (n % k == 0) return 0;
    return 1;
}

int orc_in_D(uint64_t d) {
    /* Section 1: d > 0, d == 5 (mod 8), square-free. */
    return d > 0 && d % 8 == 5 && orc_is_squarefree(d);
}

uint64_t orc_num_candidates(uint64_t lo, uint64_t hi, uint64_t *d0_out) {
    uint64_t d0 = lo + ((13 - lo % 8) % 8); /* least d >= lo, d == 5 mod 8 */
    if (d0_out) *d0_out = d0;
    if (hi <= d0) return 0;
    return (hi - d0 + 7) / 8;
}

/* ------------------------------------------------------------------ */
/* O_K / 2O_K = F_2[omega] arithmetic                                    */
/* ------------------------------------------------------------------ */

/* An element x + y*omega of O_K/2O_K is coded as x + 2y.  The minimal
 * polynomial of omega = (1+sqrt d)/2 is t^2 - t - (d-1)/4, so
 * omega^2 = omega + (d-1)/4 and modulo 2: omega^2 = omega + c with
 * c = ((d-1)/4) mod 2. */
static int f2w_mul(int a, int b, int c) {
    int x1 = a & 1, y1 = a >> 1, x2 = b & 1, y2 = b >> 1;
    int yy = y1 & y2;                        /* coefficient of omega^2 */
    int x = (x1 & x2) ^ (yy & c);            /* omega^2 -> omega + c */
    int y = (x1 & y2) ^ (x2 & y1) ^ yy;
    return x | (y << 1);
}

/* ------------------------------------------------------------------ */
/* Oracle-B: the Appendix A walk with theta reduced mod 2O_K            */
/* ------------------------------------------------------------------ */

#define ORC_MAX_STEPS (((uint64_t)1) << 40)

int orc_walk_mod2(uint64_t d, int *theta_out, uint64_t *period_out) {
    if (!orc_in_D(d)) return ORC_ENOTD;
    const int64_t D = (int64_t)d;
    const int64_t s = (int64_t)orc_isqrt(d);
    const int c = (int)(((d - 1) / 4) & 1);
    int64_t P = 1, Q = 2; /* (P_0, Q_0): O_K = [2/2, (1+sqrt d)/2] */
    int theta = 1;        /* theta_1 = 1 */
    uint64_t n = 0;
    do {
        /* Invariants of a primitive ideal [Q/2, (P+sqrt d)/2] of O_K:
         * Q > 0, Q/2 odd (its norm; 2 is inert), P odd, Q | d - P^2. */
        if (Q <= 0 || (Q / 2) % 2 != 1 || (P & 1) == 0) return ORC_EINVARIANT;
        /* q_j = floor((P_j + sqrt d)/Q_j); for Q_j > 0 and P_j + s >= 0 this
         * is floor((P_j + s)/Q_j) with s = floor(sqrt d). */
        if (P + s < 0) return ORC_EINVARIANT;
        int64_t q = (P + s) / Q;
        int64_t Pn = q * Q - P;          /* P_{j+1} = q_j Q_j - P_j */
        int64_t num = D - Pn * Pn;       /* d - P_{j+1}^2 */
        if (num % Q != 0) return ORC_EINVARIANT;
        int64_t Qn = num / Q;            /* Q_{j+1} = (d - P_{j+1}^2)/Q_j */
        /* theta_{j+2} = (P_{j+1}+sqrt d)/Q_j * theta_{j+1}.  Modulo 2O_K:
         * (P_{j+1}+sqrt d)/Q_j = [(P_{j+1}+sqrt d)/2] * [Q_j/2]^(-1) with
         * Q_j/2 odd, so [Q_j/2]^(-1) == 1, and
         * (P_{j+1}+sqrt d)/2 = (P_{j+1}-1)/2 + omega. */
        if ((Pn & 1) == 0) return ORC_EINVARIANT;
        int fx = (int)(((Pn - 1) / 2) & 1);
        int factor = fx | (1 << 1);
        theta = f2w_mul(theta, factor, c);
        if (theta == 0) return ORC_EINVARIANT; /* Theorem A.1 */
        P = Pn;
        Q = Qn;
        n++;
        if (n > ORC_MAX_STEPS) return ORC_EINVARIANT;
    } while (Q != 2); /* the first n >= 1 with norm Q_n/2 = 1: back at O_K */
    if (theta_out) *theta_out = theta;
    if (period_out) *period_out = n;
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Minimal non-negative multi-precision integers (64-bit limbs)          */
/* ------------------------------------------------------------------ */

typedef struct {
    uint64_t *w;
    size_t n;   /* used limbs; 0 means the value 0 */
    size_t cap;
} bn;

static int bn_reserve(bn *a, size_t cap) {
    if (cap <= a->cap) return 0;
    size_t nc = a->cap ? a->cap : 4;
    while (nc < cap) nc *= 2;
    uint64_t *w = (uint64_t *)realloc(a->w, nc * sizeof(uint64_t));
    if (!w) return -1;
    a->w = w;
    a->cap = nc;
    return 0;
}
static void bn_trim(bn *a) {
    while (a->n && a->w[a->n - 1] == 0) a->n--;
}
static int bn_set_u64(bn *a, uint64_t v) {
    if (bn_reserve(a, 1)) return -1;
    a->w[0] = v;
    a->n = v ? 1 : 0;
    return 0;
}
static void bn_free(bn *a) {
    free(a->w);
    a->w = NULL;
    a->n = a->cap = 0;
}
static int bn_cmp(const bn *a, const bn *b) {
    if (a->n != b->n) return a->n < b->n ? -1 : 1;
    for (size_t i = a->n; i-- > 0;) {
        if (a->w[i] != b->w[i]) return a->w[i] < b->w[i] ? -1 : 1;
    }
    return 0;
}
/* r = a*m + b*k (r may not alias a or b). */
static int bn_lincomb(bn *r, const bn *a, uint64_t m, const bn *b, uint64_t k) {
    size_t n = (a->n > b->n ? a->n : b->n) + 2;
    if (bn_reserve(r, n)) return -1;
    u128 carry = 0; /* stays below 2^66 */
    for (size_t i = 0; i < n; i++) {
        u128 pa = (i < a->n) ? (u128)a->w[i] * m : 0;
        u128 pb = (i < b->n) ? (u128)b->w[i] * k : 0;
        u128 lo = (u128)(uint64_t)pa + (uint64_t)pb + (uint64_t)carry;
        u128 hi = (pa >> 64) + (pb >> 64) + (carry >> 64) + (lo >> 64);
        r->w[i] = (uint64_t)lo;
        carry = hi;
    }
    r->n = n;
    bn_trim(r);
    return carry ? -1 : 0;
}
/* a = a / q exactly; returns the remainder (must be 0 for exactness). */
static uint64_t bn_div_small(bn *a, uint64_t q) {
    u128 rem = 0;
    for (size_t i = a->n; i-- > 0;) {
        u128 cur = (rem << 64) | a->w[i];
        a->w[i] = (uint64_t)(cur / q);
        rem = cur % q;
    }
    bn_trim(a);
    return (uint64_t)rem;
}
/* r = a * b (schoolbook). */
static int bn_mul(bn *r, const bn *a, const bn *b) {
    size_t n = a->n + b->n;
    if (bn_reserve(r, n + 1)) return -1;
    memset(r->w, 0, (n + 1) * sizeof(uint64_t));
    for (size_t i = 0; i < a->n; i++) {
        u128 carry = 0;
        for (size_t j = 0; j < b->n; j++) {
            u128 t = (u128)a->w[i] * b->w[j] + r->w[i + j] + carry;
            r->w[i + j] = (uint64_t)t;
            carry = t >> 64;
        }
        size_t k = i + b->n;
        while (carry) {
            u128 t = (u128)r->w[k] + carry;
            r->w[k] = (uint64_t)t;
            carry = t >> 64;
            k++;
        }
    }
    r->n = n;
    bn_trim(r);
    return 0;
}
/* r = a - b, requires a >= b. */
static int bn_sub(bn *r, const bn *a, const bn *b) {
    if (bn_reserve(r, a->n)) return -1;
    uint64_t borrow = 0;
    for (size_t i = 0; i < a->n; i++) {
        uint64_t bi = i < b->n ? b->w[i] : 0;
        uint64_t t = a->w[i] - bi - borrow;
        borrow = (a->w[i] < bi) || (a->w[i] - bi < borrow);
        r->w[i] = t;
    }
    r->n = a->n;
    bn_trim(r);
    return borrow ? -1 : 0;
}
static uint64_t bn_bits(const bn *a) {
    if (!a->n) return 0;
    uint64_t top = a->w[a->n - 1];
    return 64 * (a->n - 1) + (64 - (uint64_t)__builtin_clzll(top));
}

/* ------------------------------------------------------------------ */
/* Oracle-A: the exact fundamental unit                                 */
/* ------------------------------------------------------------------ */

int orc_unit_exact(uint64_t d, orc_unit *out) {
    if (!orc_in_D(d)) return ORC_ENOTD;
    const int64_t D = (int64_t)d;
    const int64_t s = (int64_t)orc_isqrt(d);
    int rc = ORC_OK;
    /* theta = (X + Y sqrt d)/2; theta_1 = 1 -> X = 2, Y = 0.
     * Convergents of omega: A_{-2}=0, A_{-1}=1, B_{-2}=1, B_{-1}=0. */
    bn X = {0}, Y = {0}, Xn = {0}, Yn = {0};
    bn A1 = {0}, A2 = {0}, B1 = {0}, B2 = {0}, An = {0}, Bn = {0}, t = {0};
    bn zero = {0};
    if (bn_set_u64(&X, 2) || bn_set_u64(&Y, 0) || bn_set_u64(&A1, 1) ||
        bn_set_u64(&A2, 0) || bn_set_u64(&B1, 0) || bn_set_u64(&B2, 1) ||
        bn_set_u64(&zero, 0)) {
        rc = ORC_ENOMEM;
        goto done;
    }
    int64_t P = 1, Q = 2;
    uint64_t n = 0;
    do {
        if (Q <= 0 || (Q / 2) % 2 != 1 || (P & 1) == 0 || P + s < 0) {
            rc = ORC_EINVARIANT;
            goto done;
        }
        int64_t q = (P + s) / Q;
        int64_t Pn = q * Q - P;
        int64_t num = D - Pn * Pn;
        if (num % Q != 0 || Pn <= 0) {
            rc = ORC_EINVARIANT;
            goto done;
        }
        int64_t Qn = num / Q;
        /* theta_{j+2} = (P_{j+1} + sqrt d)/Q_j * theta_{j+1}:
         * X' = (X P_{j+1} + Y d)/Q_j,  Y' = (X + Y P_{j+1})/Q_j,
         * both divisions exact because theta_{j+2} lies in O_K. */
        if (bn_lincomb(&Xn, &X, (uint64_t)Pn, &Y, d) ||
            bn_lincomb(&Yn, &X, 1, &Y, (uint64_t)Pn)) {
            rc = ORC_ENOMEM;
            goto done;
        }
        if (bn_div_small(&Xn, (uint64_t)Q) != 0 || bn_div_small(&Yn, (uint64_t)Q) != 0) {
            rc = ORC_EINVARIANT;
            goto done;
        }
        /* Convergents: A_j = q_j A_{j-1} + A_{j-2}, same for B. */
        if (bn_lincomb(&An, &A1, (uint64_t)q, &A2, 1) ||
            bn_lincomb(&Bn, &B1, (uint64_t)q, &B2, 1)) {
            rc = ORC_ENOMEM;
            goto done;
        }
        /* Appendix A: theta_{j+2} = (G_j + B_j sqrt d)/2 with G_j = 2A_j - B_j,
         * i.e. Y' = B_j and X' + B_j = 2 A_j. */
        if (bn_lincomb(&t, &Xn, 1, &Bn, 1)) {
            rc = ORC_ENOMEM;
            goto done;
        }
        {
            bn twoA = {0};
            if (bn_lincomb(&twoA, &An, 2, &zero, 0)) {
                bn_free(&twoA);
                rc = ORC_ENOMEM;
                goto done;
            }
            int okG = bn_cmp(&t, &twoA) == 0;
            bn_free(&twoA);
            if (!okG || bn_cmp(&Yn, &Bn) != 0) {
                rc = ORC_EINVARIANT;
                goto done;
            }
        }
        /* shift */
        { bn tmp = X; X = Xn; Xn = tmp; }
        { bn tmp = Y; Y = Yn; Yn = tmp; }
        { bn tmp = A2; A2 = A1; A1 = An; An = tmp; }
        { bn tmp = B2; B2 = B1; B1 = Bn; Bn = tmp; }
        P = Pn;
        Q = Qn;
        n++;
        if (n > ORC_MAX_STEPS) {
            rc = ORC_EINVARIANT;
            goto done;
        }
    } while (Q != 2);

    /* epsilon_d = theta_{n+1} = (x0 + y0 sqrt d)/2 with x0 = X, y0 = Y.
     * Unit check: x0^2 - d y0^2 = +-4. */
    {
        bn X2 = {0}, Y2 = {0}, dY2 = {0}, diff = {0};
        int norm = 0;
        if (bn_mul(&X2, &X, &X) || bn_mul(&Y2, &Y, &Y) ||
            bn_lincomb(&dY2, &Y2, d, &zero, 0)) {
            rc = ORC_ENOMEM;
        } else {
            int cmp = bn_cmp(&X2, &dY2);
            if (cmp > 0) {
                bn_sub(&diff, &X2, &dY2);
                if (diff.n == 1 && diff.w[0] == 4) norm = +1;
            } else if (cmp < 0) {
                bn_sub(&diff, &dY2, &X2);
                if (diff.n == 1 && diff.w[0] == 4) norm = -1;
            }
            if (norm == 0) rc = ORC_ENORM;
        }
        bn_free(&X2);
        bn_free(&Y2);
        bn_free(&dY2);
        bn_free(&diff);
        if (rc != ORC_OK) goto done;
        /* O_K coordinates: epsilon = u + v omega with v = y0, u = (x0-y0)/2.
         * epsilon == 1 (mod 2O_K) iff u odd and v even. */
        int x_par = X.n ? (int)(X.w[0] & 1) : 0;
        int y_par = Y.n ? (int)(Y.w[0] & 1) : 0;
        if (x_par != y_par) {
            rc = ORC_EINVARIANT; /* x0 == y0 (mod 2) for elements of O_K */
            goto done;
        }
        bn u = {0};
        if (bn_cmp(&X, &Y) < 0) { /* x0 > y0 for eps > 1 with y0 > 0 */
            rc = ORC_EINVARIANT;
            goto done;
        }
        bn_sub(&u, &X, &Y);
        bn_div_small(&u, 2);
        int u_par = u.n ? (int)(u.w[0] & 1) : 0;
        bn_free(&u);
        if (out) {
            out->period = n;
            out->norm = norm;
            out->theta = u_par | (y_par << 1);
            out->flag = (u_par == 1 && y_par == 0);
            out->x0_lo = X.n ? X.w[0] : 0;
            out->y0_lo = Y.n ? Y.w[0] : 0;
            out->x0_fits = X.n <= 1;
            out->y0_fits = Y.n <= 1;
            out->y0_bits = bn_bits(&Y);
        }
    }
done:
    bn_free(&X); bn_free(&Y); bn_free(&Xn); bn_free(&Yn);
    bn_free(&A1); bn_free(&A2); bn_free(&B1); bn_free(&B2);
    bn_free(&An); bn_free(&Bn); bn_free(&t); bn_free(&zero);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Lemma 1.1(ii): brute-force search for x^2 - d y^2 = +-4              */
/* ------------------------------------------------------------------ */

uint64_t orc_pell_smallest(uint64_t d, uint64_t ymax, uint64_t *x_out, int *sign_out) {
    for (uint64_t y = 1; y <= ymax; y++) {
        uint64_t dy2 = d * y * y;
        /* for equal y the norm -1 solution has the smaller x, hence is the
         * smaller unit (x + y sqrt d)/2: try it first */
        uint64_t cand[2] = {dy2 >= 4 ? dy2 - 4 : 0, dy2 + 4};
        int sgn[2] = {-1, +1};
        for (int i = 0; i < 2; i++) {
            if (cand[i] == 0) continue;
            uint64_t x = orc_isqrt(cand[i]);
            if (x * x == cand[i]) {
                if (x_out) *x_out = x;
                if (sign_out) *sign_out = sgn[i];
                return y;
            }
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Lemma 1.1(iv): narrow class numbers by cycles of reduced forms        */
/* ------------------------------------------------------------------ */

typedef struct {
    int64_t a, b, c;
} form3;

static int64_t gcd_i64(int64_t a, int64_t b) {
    if (a < 0) a = -a;
    if (b < 0) b = -b;
    while (b) {
        int64_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}
static int64_t abs_i64(int64_t a) { return a < 0 ? -a : a; }

/* (a,b,c) of discriminant Dl = b^2 - 4ac > 0, Dl not a square, is reduced
 * iff |sqrt(Dl) - 2|a|| < b < sqrt(Dl).  With r = floor(sqrt(Dl)) and sqrt(Dl)
 * irrational: b < sqrt(Dl) <=> b <= r; sqrt(Dl) - 2|a| < b <=> (2|a|+b)^2 > Dl;
 * 2|a| - sqrt(Dl) < b <=> 2|a| - b <= 0 or (2|a|-b)^2 < Dl. */
static int form_reduced(int64_t a, int64_t b, int64_t Dl, int64_t r) {
    int64_t A2 = 2 * abs_i64(a);
    if (b <= 0 || b > r) return 0;
    if ((A2 + b) * (A2 + b) <= Dl) return 0;
    if (A2 - b > 0 && (A2 - b) * (A2 - b) >= Dl) return 0;
    return 1;
}

static int cmp_form(const void *x, const void *y) {
    const form3 *p = (const form3 *)x, *q = (const form3 *)y;
    if (p->a != q->a) return p->a < q->a ? -1 : 1;
    if (p->b != q->b) return p->b < q->b ? -1 : 1;
    return 0;
}

int64_t orc_narrow_classno(uint64_t Du) {
    const int64_t Dl = (int64_t)Du;
    const int64_t r = (int64_t)orc_isqrt(Du);
    if (r * r == Dl || Dl <= 0 || Dl % 4 == 2 || Dl % 4 == 3) return -1;
    size_t cap = 1024, nf = 0;
    form3 *fs = (form3 *)malloc(cap * sizeof(form3));
    if (!fs) return -1;
    /* Enumerate reduced primitive forms: 0 < b <= r, b == Dl (mod 2),
     * a*c = -(Dl - b^2)/4 with a, c of opposite signs. */
    for (int64_t b = (Dl & 1) ? 1 : 2; b <= r; b += 2) {
        int64_t N = (Dl - b * b) / 4; /* = -ac > 0 */
        for (int64_t m = 1; m <= N; m++) {
            if (N % m) continue;
            for (int sg = -1; sg <= 1; sg += 2) {
                int64_t a = sg * m, c = -N / a;
                if (!form_reduced(a, b, Dl, r)) continue;
                if (gcd_i64(gcd_i64(a, b), c) != 1) continue;
                if (nf == cap) {
                    cap *= 2;
                    form3 *t = (form3 *)realloc(fs, cap * sizeof(form3));
                    if (!t) { free(fs); return -1; }
                    fs = t;
                }
                fs[nf].a = a;
                fs[nf].b = b;
                fs[nf].c = c;
                nf++;
            }
        }
    }
    qsort(fs, nf, sizeof(form3), cmp_form);
    unsigned char *seen = (unsigned char *)calloc(nf ? nf : 1, 1);
    if (!seen) { free(fs); return -1; }
    int64_t cycles = 0;
    for (size_t i = 0; i < nf; i++) {
        if (seen[i]) continue;
        cycles++;
        size_t cur = i;
        while (!seen[cur]) {
            seen[cur] = 1;
            /* rho(a,b,c) = (c, b', (b'^2 - Dl)/(4c)) with b' == -b (mod 2|c|)
             * and sqrt(Dl) - 2|c| < b' < sqrt(Dl). */
            int64_t c = fs[cur].c, b = fs[cur].b;
            int64_t m = 2 * abs_i64(c);
            int64_t bp = r - (((r + b) % m) + m) % m;
            int64_t num = bp * bp - Dl;
            if (num % (4 * c) != 0) { free(fs); free(seen); return -1; }
            form3 key = {c, bp, num / (4 * c)};
            form3 *hit = (form3 *)bsearch(&key, fs, nf, sizeof(form3), cmp_form);
            if (!hit || hit->c != key.c) { free(fs); free(seen); return -1; }
            cur = (size_t)(hit - fs);
        }
        /* the orbit must close on its first element */
        if (cur != i) { free(fs); free(seen); return -1; }
    }
    free(fs);
    free(seen);
    return cycles;
}

/* ------------------------------------------------------------------ */
/* Range drivers (POSIX threads over blocks of candidates)              */
/* ------------------------------------------------------------------ */

int orc_default_threads(void) {
    long n = sysconf(_SC_NPROCESSORS_ONLN);
    return n > 0 ? (int)n : 1;
}

typedef struct {
    uint64_t d0, n;
    uint8_t *codes;
    uint32_t *periods;
    uint8_t *thetas;
    uint64_t next;           /* next block of candidates (atomic) */
    uint64_t cnt[3];         /* #D, #E, steps (atomic adds) */
    int err;                 /* first error (atomic) */
    int sieve_only;          /* 1: codes = 1 for d in D, no walk */
    int primes;              /* 1: only prime d (prime subsequence, Section 3.2) */
} range_job;

#define ORC_BLOCK 4096

static void *range_worker(void *arg) {
    range_job *J = (range_job *)arg;
    uint64_t loc[3] = {0, 0, 0};
    unsigned char *notsf = (unsigned char *)malloc(ORC_BLOCK);
    if (!notsf) {
        int zero = 0;
        __atomic_compare_exchange_n(&J->err, &zero, ORC_ENOMEM, 0, __ATOMIC_RELAXED,
                                    __ATOMIC_RELAXED);
        return NULL;
    }
    for (;;) {
        uint64_t b = __atomic_fetch_add(&J->next, ORC_BLOCK, __ATOMIC_RELAXED);
        if (b >= J->n) break;
        uint64_t e = b + ORC_BLOCK < J->n ? b + ORC_BLOCK : J->n;
        /* Square-freeness of every candidate of the block, by the definition
         * applied in bulk: for every k >= 2 with k^2 <= max d, mark each
         * multiple of k^2 that is a candidate (== 5 mod 8) of the block. */
        uint64_t dlo = J->d0 + 8 * b, dhi = J->d0 + 8 * (e - 1); /* inclusive */
        memset(notsf, 0, (size_t)(e - b));
        for (uint64_t k = 2; k <= dhi / k; k++) {
            if (J->primes) {
                /* composite: a multiple k*j with j >= k (so k*j != k) */
                uint64_t x = (dlo + k - 1) / k * k;
                if (x < k * k) x = k * k;
                for (; x <= dhi; x += k) {
                    if (x % 8 == 5) notsf[(x - dlo) / 8] = 1;
                }
            } else {
                uint64_t k2 = k * k;
                uint64_t x = (dlo + k2 - 1) / k2 * k2; /* least multiple >= dlo */
                for (; x <= dhi; x += k2) {
                    if (x % 8 == 5) notsf[(x - dlo) / 8] = 1;
                }
            }
        }
        for (uint64_t kk = b; kk < e; kk++) {
            uint64_t d = J->d0 + 8 * kk;
            uint8_t code = 0, th = 0;
            uint32_t per = 0;
            if (!notsf[kk - b] && J->sieve_only) {
                code = 1;
                loc[0]++;
            } else if (!notsf[kk - b]) {
                int theta = 0;
                uint64_t n = 0;
                int rc = orc_walk_mod2(d, &theta, &n);
                if (rc != ORC_OK) {
                    int zero = 0;
                    __atomic_compare_exchange_n(&J->err, &zero, rc, 0, __ATOMIC_RELAXED,
                                                __ATOMIC_RELAXED);
                    continue;
                }
                code = theta == 1 ? 2 : 1;
                th = (uint8_t)theta;
                per = n > UINT32_MAX ? UINT32_MAX : (uint32_t)n;
                loc[0]++;
                loc[1] += code == 2;
                loc[2] += n;
            }
            if (J->codes) J->codes[kk] = code;
            if (J->periods) J->periods[kk] = per;
            if (J->thetas) J->thetas[kk] = th;
        }
    }
    free(notsf);
    for (int i = 0; i < 3; i++) __atomic_fetch_add(&J->cnt[i], loc[i], __ATOMIC_RELAXED);
    return NULL;
}

static int run_range(uint64_t lo, uint64_t hi, int nthreads, uint8_t *codes,
                     uint32_t *periods, uint8_t *thetas, uint64_t out[3],
                     int sieve_only, int primes) {
    if (hi < lo) return ORC_EINVAL;
    range_job J;
    memset(&J, 0, sizeof(J));
    J.sieve_only = sieve_only;
    J.primes = primes;
    J.n = orc_num_candidates(lo, hi, &J.d0);
    J.codes = codes;
    J.periods = periods;
    J.thetas = thetas;
    if (nthreads <= 0) nthreads = orc_default_threads();
    if ((uint64_t)nthreads > J.n / ORC_BLOCK + 1) nthreads = (int)(J.n / ORC_BLOCK + 1);
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    if (!th) return ORC_ENOMEM;
    int started = 0;
    for (int i = 0; i < nthreads; i++) {
        if (pthread_create(&th[i], NULL, range_worker, &J) != 0) break;
        started++;
    }
    if (started == 0) range_worker(&J);
    for (int i = 0; i < started; i++) pthread_join(th[i], NULL);
    free(th);
    if (out) memcpy(out, J.cnt, sizeof(J.cnt));
    return J.err;
}

int orc_classify_range(uint64_t lo, uint64_t hi, int nthreads, uint8_t *codes,
                       uint32_t *periods, uint8_t *thetas) {
    return run_range(lo, hi, nthreads, codes, periods, thetas, NULL, 0, 0);
}

int orc_classify_range_primes(uint64_t lo, uint64_t hi, int nthreads, uint8_t *codes,
                              uint8_t *thetas) {
    return run_range(lo, hi, nthreads, codes, NULL, thetas, NULL, 0, 1);
}

int orc_count_range_primes(uint64_t lo, uint64_t hi, int nthreads, uint64_t out[3]) {
    return run_range(lo, hi, nthreads, NULL, NULL, NULL, out, 0, 1);
}

int orc_count_range(uint64_t lo, uint64_t hi, int nthreads, uint64_t out[3]) {
    return run_range(lo, hi, nthreads, NULL, NULL, NULL, out, 0, 0);
}

int orc_sqfree_range(uint64_t lo, uint64_t hi, int nthreads, uint8_t *in_D_out,
                     uint64_t *count_out) {
    uint64_t cnt[3] = {0, 0, 0};
    int rc = run_range(lo, hi, nthreads, in_D_out, NULL, NULL, cnt, 1, 0);
    if (count_out) *count_out = cnt[0];
    return rc;
}
