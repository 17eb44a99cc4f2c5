/*
 * oracle.h -- CPU oracle for Eisenstein discriminants (Breuer & Punch,
 * "Quadratic units and cubic fields").
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline / reference leg of bench.py may load this library.  It shares
 * no code with the CUDA library under paper_2507_06579_gb300/ and neither
 * side includes the other.
 *
 * Every function is plain, single-purpose and slow on purpose: it writes out
 * the definition or the algorithm step of the paper it cites, in 64-bit or
 * exact multi-precision integers.  No floating point is used anywhere.
 *
 * Candidate indexing used by the range functions: for a half-open range
 * [lo, hi) the candidates are the d = d0 + 8k (k = 0 .. n-1) with d == 5
 * (mod 8), where d0 is the least such d >= lo.
 */
#ifndef EIS_ORACLE_H
#define EIS_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes (negative = an invariant of the paper was violated). */
#define ORC_OK 0
#define ORC_ENOTD -1      /* d is not in D (d != 5 mod 8 or not squarefree) */
#define ORC_EINVARIANT -2 /* an identity the paper guarantees failed */
#define ORC_ENORM -3      /* the unit found does not have norm +-1 */
#define ORC_ENOMEM -4
#define ORC_EINVAL -5

/* floor(sqrt(n)) by integer Newton iteration. */
uint64_t orc_isqrt(uint64_t n);

/* 1 iff no k >= 2 has k^2 | n (trial division by every k with k^2 <= n).
 * Definition of "square-free" in the set D, Section 1. */
int orc_is_squarefree(uint64_t n);

/* 1 iff n is prime (trial division by every k with k^2 <= n).  For the
 * prime subsequence E cap P of Section 3.2. */
int orc_is_prime(uint64_t n);

/* 1 iff d is in D = { d > 0 : d == 5 (mod 8), d square-free }, Section 1. */
int orc_in_D(uint64_t d);

/* Oracle-B: epsilon_d mod 2O_K by the infrastructure baby step rho of
 * Appendix A, carrying theta reduced modulo 2O_K as an element x + y*omega
 * of O_K/2O_K (x, y in {0,1}).  Walks the whole period: from
 * (P_0,Q_0) = (1,2), theta_1 = 1 until the first n >= 1 with Q_n = 2.
 *   theta_out  : x + 2y for theta_{n+1} = epsilon_d (mod 2O_K)
 *   period_out : n (the period length of the cycle of reduced ideals)
 * Returns ORC_OK, ORC_ENOTD or ORC_EINVARIANT. */
int orc_walk_mod2(uint64_t d, int *theta_out, uint64_t *period_out);

/* Oracle-A: the fundamental unit epsilon_d = (x0 + y0 sqrt d)/2 computed
 * exactly (multi-precision) as theta_{n+1} of the same walk, with the
 * generator recurrence theta_{j+2} = (P_{j+1}+sqrt d)/Q_j * theta_{j+1}
 * carried exactly, cross-checked against the continued-fraction convergents
 * (theta_j = (G_{j-2} + B_{j-2} sqrt d)/2 with G = 2A - B) and verified to
 * satisfy x0^2 - d y0^2 = +-4.  flag = [epsilon_d == 1 (mod 2O_K)] read off
 * the O_K-coordinates epsilon = u + v*omega, u = (x0-y0)/2, v = y0. */
typedef struct {
    uint64_t period; /* n = period of the ideal cycle */
    int norm;        /* +1 or -1: x0^2 - d y0^2 = 4 * norm */
    int flag;        /* 1 iff epsilon_d == 1 (mod 2O_K) */
    int theta;       /* u + 2v mod 2 (same coding as orc_walk_mod2) */
    uint64_t x0_lo;  /* x0 mod 2^64 */
    uint64_t y0_lo;  /* y0 mod 2^64 */
    int y0_fits;     /* 1 iff y0 < 2^64 (then y0_lo == y0) */
    int x0_fits;     /* 1 iff x0 < 2^64 */
    uint64_t y0_bits;/* bit length of y0 */
} orc_unit;
int orc_unit_exact(uint64_t d, orc_unit *out);

/* Smallest y in [1, ymax] such that d*y^2 + 4 or d*y^2 - 4 is a perfect
 * square x^2 (Lemma 1.1(ii): solutions of x^2 - d y^2 = +-4).  Returns y and
 * writes x and the sign (+1 for x^2 - dy^2 = 4, -1 for -4); returns 0 if no
 * y <= ymax works.  Requires d * ymax^2 < 2^63. */
uint64_t orc_pell_smallest(uint64_t d, uint64_t ymax, uint64_t *x_out, int *sign_out);

/* Narrow class number h+(D) of discriminant D > 0 (D not a square), counted
 * as the number of rho-cycles of reduced primitive indefinite binary
 * quadratic forms (a,b,c), b^2 - 4ac = D.  Used with Lemma 1.1(iv):
 * for d in D, h+(4d) = 3 h+(d) iff d is an Eisenstein discriminant.
 * Returns -1 on an internal inconsistency or allocation failure. */
int64_t orc_narrow_classno(uint64_t D);

/* Per candidate d = d0 + 8k in [lo, hi): codes[k] = 0 (d not in D),
 * 1 (d in D but not in E), 2 (d in E), by Oracle-B.  periods (nullable)
 * receives the period n for d in D, 0 otherwise; thetas (nullable) receives
 * x + 2y of epsilon_d mod 2O_K, 0 for d not in D.  Runs on nthreads POSIX
 * threads (nthreads <= 0: one per online CPU).  Returns ORC_OK or the first
 * error met. */
int orc_classify_range(uint64_t lo, uint64_t hi, int nthreads, uint8_t *codes,
                       uint32_t *periods, uint8_t *thetas);

/* Counts over [lo, hi) by Oracle-B: out[0] = #D, out[1] = #E, out[2] = total
 * rho steps walked (sum of periods).  Returns ORC_OK or an error. */
int orc_count_range(uint64_t lo, uint64_t hi, int nthreads, uint64_t out[3]);

/* Membership in D only (no walk): in_D_out[k] (nullable) = 1 iff d0 + 8k is
 * square-free; *count_out = #D in [lo, hi).  Square-freeness by marking the
 * multiples of k^2 for every k >= 2 (the definition applied to a block). */
int orc_sqfree_range(uint64_t lo, uint64_t hi, int nthreads, uint8_t *in_D_out,
                     uint64_t *count_out);

/* The same for the prime candidates only (Section 3.2, E cap P): codes[k] =
 * 0 (d not prime), 1 (prime, not in E), 2 (prime in E); primality by marking,
 * for every k >= 2, the multiples k*j with j >= k. */
int orc_classify_range_primes(uint64_t lo, uint64_t hi, int nthreads, uint8_t *codes,
                              uint8_t *thetas);
/* out[0] = #primes == 5 (mod 8), out[1] = #(E cap P), out[2] = rho steps. */
int orc_count_range_primes(uint64_t lo, uint64_t hi, int nthreads, uint64_t out[3]);

/* Number of candidates d == 5 (mod 8) in [lo, hi) and the first one. */
uint64_t orc_num_candidates(uint64_t lo, uint64_t hi, uint64_t *d0_out);

/* Threads orc_classify_range/orc_count_range use for nthreads <= 0. */
int orc_default_threads(void);

#ifdef __cplusplus
}
#endif
#endif
