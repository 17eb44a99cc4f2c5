"""Identities the GPU walk and giant steps rest on, checked on the CPU.

These are the facts behind the kernels' arithmetic, not part of the oracle
(which walks the plain definition).  Each is checked in exact integers (and
exact rationals for the fp32 claims, with rcp.approx allowed one ulp either
side of the correctly rounded reciprocal):

* rho from O_K keeps Q == 2 (mod 4) and P odd (d == 5 mod 8), and
  Q_{j+1} = Q_{j-1} + q_j (P_j - P_{j+1}) (no division);
* [P_{j+1} == 3 mod 4] = 1 xor (q_j mod 2) xor [P_j == 3 mod 4] (the lean
  walk's class bit);
* the half-period rule (Algorithm 1's symmetry test, Appendix A classes):
  at the first j with Q_{j+1} = Q_j, log eps = 2 S_j + c(P_{j+1}); at the
  first j with P_{j+1} = P_j, log eps = 2 S_j -- against the oracle's
  full-period walk;
* the fast quotient: num = P + s + 1/2 lies at least 1/(2Q) from every
  multiple of Q, so floor(num * rcp(Q)) = q for d below the fast limit;
* the giant-step reduction's quotient estimate with one correction, and its
  exact division by the 2-adic inverse.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

FAST_D_LIMIT = 4_390_000_000_000  # the walk kernels' fast-quotient bound
D_LIMIT = 1 << 44


def _c(P):
    """log of (P-1)/2 + omega mod 2 in Z/3: 1 if P == 1 (mod 4), else 2."""
    return 1 + ((P >> 1) & 1)


def _nonsquare_5mod8(rng, lo, hi, k):
    out = []
    while len(out) < k:
        d = int(rng.integers(lo // 8, hi // 8)) * 8 + 5
        if math.isqrt(d) ** 2 != d:
            out.append(d)
    return out


def _rho(d, steps):
    """(P_j, Q_j, q_j, P_{j+1}, Q_{j+1}) for j = 0..steps-1 from (1, 2)."""
    s = math.isqrt(d)
    P, Q = 1, 2
    out = []
    for _ in range(steps):
        q = (P + s) // Q
        Pn = q * Q - P
        Qn = (d - Pn * Pn) // Q
        assert Qn * Q == d - Pn * Pn
        out.append((P, Q, q, Pn, Qn))
        P, Q = Pn, Qn
    return out


@pytest.mark.parametrize("lo,hi", [(10**3, 10**6), (10**9, 10**11), (10**12, D_LIMIT)])
def test_rho_recurrence_parity_and_class_bit(lo, hi):
    rng = np.random.default_rng(lo % 97 + 1)
    for d in _nonsquare_5mod8(rng, lo, hi, 12):
        Qprev = None
        for P, Q, q, Pn, Qn in _rho(d, 400):
            assert Q % 4 == 2 and P % 2 == 1
            if Qprev is not None:
                assert Qn == Qprev + q * (P - Pn)
            assert ((Pn >> 1) & 1) == 1 ^ (q & 1) ^ ((P >> 1) & 1)
            Qprev = Q


def _half_period_log(d):
    """log eps_d in Z/3 by the half-period rule, S_j = c(P_1) + ... + c(P_j)."""
    s = math.isqrt(d)
    P = 2 * ((1 + s) // 2) - 1  # P_1
    Q = (d - P * P) // 2       # Q_1
    if Q == 2:
        return _c(P) % 3       # period 1
    S = _c(P)
    while True:
        q = (P + s) // Q
        Pn = q * Q - P
        Qn = (d - Pn * Pn) // Q
        if Qn == Q:
            return (2 * S + _c(Pn)) % 3
        if Pn == P:
            return (2 * S) % 3
        S += _c(Pn)
        P, Q = Pn, Qn


def test_half_period_rule_matches_oracle(orc):
    lo, hi = 5, 40_005
    ref = orc.classify_range(lo, hi, thetas=True)
    d0 = ref["d0"]
    n = 0
    for k, th in enumerate(ref["thetas"]):
        if th == 0:
            continue  # not in D
        d = d0 + 8 * k
        assert _half_period_log(d) == th - 1, d
        n += 1
    assert n > 3000


def _f32_rcp_candidates(Q):
    r = np.float32(1.0) / np.float32(Q)
    return [np.nextafter(r, np.float32(0)), r, np.nextafter(r, np.float32(np.inf))]


@pytest.mark.parametrize("top", [10**9, 10**11, FAST_D_LIMIT - 1])
def test_fast_quotient_is_exact_below_the_limit(top):
    rng = np.random.default_rng(top % 89 + 3)
    for d in _nonsquare_5mod8(rng, top - 10**8, top, 6):
        s = math.isqrt(d)
        for P, Q, q, _, _ in _rho(d, 300)[1:]:
            num = Fraction(2 * (P + s) + 1, 2)  # P + s + 1/2, exact in fp32
            assert float(num) == float(np.float32(float(num)))
            # at least 1/(2Q) from every integer: the numerator 2(P+s)+1 is odd
            frac = num / Q - math.floor(num / Q)
            assert frac >= Fraction(1, 2 * Q) and 1 - frac >= Fraction(1, 2 * Q)
            for r in _f32_rcp_candidates(Q):
                assert math.floor(num * Fraction(float(r))) == q, (d, P, Q)


def _floor_div_fast(x, y, r):
    """The giant-step reduction's quotient: fp32 estimate, one correction."""
    fx = np.float32(x)
    e = math.floor(float(np.float32(fx * r)))
    if abs(e) >= 1 << 20:
        return x // y
    q = e
    rem = x - q * y
    if y > 0:
        if rem < 0:
            q -= 1
        elif rem >= y:
            q += 1
    else:
        if rem > 0:
            q -= 1
        elif rem <= y:
            q += 1
    return q


def test_floor_div_fast_with_one_correction():
    rng = np.random.default_rng(11)
    for _ in range(20000):
        y = int(rng.integers(1, 1 << 46)) * (1 if rng.random() < 0.5 else -1)
        qmax = min(1 << 21, (1 << 47) // abs(y))
        x = y * int(rng.integers(-qmax, qmax + 1)) + int(rng.integers(-abs(y) + 1, abs(y)))
        if abs(x) >= 1 << 47:
            continue
        ry = np.float32(1.0) / np.float32(y)
        for r in (np.nextafter(ry, np.float32(-np.inf)), ry, np.nextafter(ry, np.float32(np.inf))):
            assert _floor_div_fast(x, y, r) == x // y, (x, y)


def _exact_quot(d, P, Q):
    """(d - P^2)/Q from d - P^2 mod 2^64 and the inverse of |Q|/2 mod 2^64."""
    M = (1 << 64) - 1
    X = (d - P * P) & M
    ha = abs(Q) // 2
    inv = ha
    for _ in range(5):
        inv = (inv * (2 - ha * inv)) & M
    m = ((X >> 1) * inv) & ((1 << 63) - 1)
    v = m - (1 << 63) if m & (1 << 62) else m
    return -v if Q < 0 else v


def test_exact_division_by_the_2adic_inverse():
    rng = np.random.default_rng(12)
    for d in _nonsquare_5mod8(rng, 10**12, D_LIMIT, 40):
        for P, Q, q, Pn, Qn in _rho(d, 50):
            # P moved by multiples of Q, up to P^2 ~ 2^80 > 2^64 (the quotient
            # stays below 2^62, as after a composition)
            for k in (1, 3, 17, 1 << 18, (1 << 18) + 7):
                Pk = Pn + k * Q
                if (d - Pk * Pk) % Q == 0:
                    assert _exact_quot(d, Pk, Q) == (d - Pk * Pk) // Q
                    assert _exact_quot(d, Pk, -Q) == (d - Pk * Pk) // -Q


@pytest.mark.parametrize("top", [FAST_D_LIMIT + 10**9, 10**13, D_LIMIT - 1])
def test_corrected_quotient_up_to_2_44(top):
    """Above the fast limit the walk floors num * rcp(Q) onto 2^23 - 1/2 with
    num = P + s: the result is q or q - 1, the remainder num - q' Q lies in
    [0, 2Q), and one compare with Q gives q."""
    rng = np.random.default_rng(top % 83 + 9)
    M = 1 << 23
    for d in _nonsquare_5mod8(rng, top - 10**9, top, 6):
        s = math.isqrt(d)
        for P, Q, q, _, _ in _rho(d, 300)[1:]:
            num = P + s
            assert num < M  # exact in fp32, as is every product below
            for r in _f32_rcp_candidates(Q):
                # fma rounded toward -inf onto the integer grid of [2^23, 2^24)
                qm = math.floor(Fraction(num) * Fraction(float(r)) + M - Fraction(1, 2))
                qe = qm - M
                assert qe in (q, q - 1), (d, P, Q)
                rem = num - qe * Q
                assert 0 <= rem < 2 * Q
                if rem >= Q:
                    qe += 1
                assert qe == q
