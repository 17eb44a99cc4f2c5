"""The giant-step ideal arithmetic (textbook composition + rho reduction, and
NUCOMP/NUDUPL/NUCOMPchoose with the gamma class, eis_infra.cuh) run on the
host against an exact walk of the principal cycle.

State j of the cycle is the reduced ideal [Q_j/2, (P_j + sqrt d)/2] with
generator class S_j = c(P_1) + ... + c(P_j) in Z/3 (c(P) = 1 if P == 1 mod 4,
else 2; Appendix A).  The reduced product of states i and k must be a state
m of the cycle, at about the sum of their distances, and carry the class
S_m -- as long as the sum stays inside the first half period, where no unit
is crossed.  The host build compiles the same source as the kernels."""
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def infra_host(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("infra") / "infra_host")
    r = subprocess.run([nvcc, "-std=c++17", "-O2", "-gencode", "arch=compute_103a,code=sm_103a",
                        "-I", os.path.join(ROOT, "include"),
                        "-I", os.path.join(ROOT, "paper_2507_06579_gb300", "csrc"),
                        os.path.join(ROOT, "tests", "infra_host.cu"), "-o", exe],
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    return exe


def _c(P):
    return 1 + ((P >> 1) & 1)


def _half_cycle(d):
    """States 1..j* of the cycle up to the first centre: (Q_j, P_j, S_j mod 3,
    delta_j), delta_j = log theta_j the distance from O_K."""
    s = math.isqrt(d)
    rd = math.sqrt(d)
    P = 2 * ((1 + s) // 2) - 1
    Q = (d - P * P) // 2
    delta = math.log((P + rd) / 2)
    states = [(Q, P, _c(P) % 3, delta)]
    S = _c(P)
    while Q != 2:
        q = (P + s) // Q
        Pn = q * Q - P
        Qn = (d - Pn * Pn) // Q
        if Qn == Q or Pn == P:
            break  # centre: the second half mirrors the first
        S += _c(Pn)
        delta += math.log((Pn + rd) / Q)
        P, Q = Pn, Qn
        states.append((Q, P, S % 3, delta))
    return states


def _pick_d(orc, rng, lo, hi, min_states, k):
    out = []
    while len(out) < k:
        d = int(rng.integers(lo // 8, hi // 8)) * 8 + 5
        if orc.in_D(d) and len(_half_cycle(d)) >= min_states:
            out.append(d)
    return out


@pytest.mark.parametrize("lo,hi", [(10**5, 10**7), (10**8, 10**10), (10**11, 10**12)])
def test_products_land_on_the_cycle_with_their_class(infra_host, orc, lo, hi):
    rng = np.random.default_rng(lo % 101 + 5)
    lines, expect = [], []
    for d in _pick_d(orc, rng, lo, hi, 120, 6):
        st = _half_cycle(d)
        index = {(Q, P): (j, S, dl) for j, (Q, P, S, dl) in enumerate(st)}
        m = len(st)
        pairs = [(i, k) for i in range(0, m // 4, max(1, m // 40)) for k in (i, m // 4 - i)]
        pairs += [(0, 1), (1, 1), (2, 3)]  # small norms: NUCOMPchoose's textbook branch
        for i, k in pairs:
            (Qi, Pi, Si, di), (Qk, Pk, Sk, dk) = st[i], st[k]
            lines.append("%d %d %d %d %d %d %d" % (d, Qi // 2, Pi, Si, Qk // 2, Pk, Sk))
            expect.append((d, i, k, index, di + dk))
    r = subprocess.run([infra_host], input="\n".join(lines) + "\n", capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    rows = r.stdout.split("\n")
    n_small = 0
    for (d, i, k, index, dsum), row in zip(expect, rows):
        okT, aT, bT, gT, okN, aN, bN, gN, okL, aL, bL, gL, okM, aM, bM, gM = map(int, row.split())
        assert okT == 1 and okN == 1 and okL == 1 and okM == 1, (d, i, k)
        for a, b, g in ((aT, bT, gT), (aN, bN, gN), (aL, bL, gL), (aM, bM, gM)):
            assert (2 * a, b) in index, (d, i, k, a, b)  # a reduced state of the cycle
            j, S, dj = index[(2 * a, b)]
            assert g == S, (d, i, k, j)                  # with that state's class
            # near the sum of the two distances (a reduction ends within about
            # log d of it)
            assert abs(dj - dsum) <= math.log(d), (d, i, k, j, dj, dsum)
        n_small += min(i, k) < 3
    assert len(rows) - 1 == len(expect) and n_small > 0


class _Composer:
    """reduce(X * Y) through the host driver, one product per line."""

    def __init__(self, exe):
        self.p = subprocess.Popen([exe], stdin=subprocess.PIPE, stdout=subprocess.PIPE, text=True,
                                  bufsize=1)

    def mul(self, d, X, Y, nucomp):
        self.p.stdin.write("%d %d %d %d %d %d %d\n" % ((d,) + X + Y))
        self.p.stdin.flush()
        okT, aT, bT, gT, okN, aN, bN, gN = map(int, self.p.stdout.readline().split()[:8])
        ok, out = (okN, (aN, bN, gN)) if nucomp else (okT, (aT, bT, gT))
        assert ok == 1
        return out

    def close(self):
        self.p.stdin.close()
        self.p.wait(timeout=60)


def _search_log(comp, d, N, nucomp):
    """Algorithm 1 as the giant-step kernel runs it: baby states 1..N in a
    table under direct keys (Q_j, P_j) and mirror keys (Q_j, P_{j+1}), O_K as
    (2, P_1); G = state N+1; lane t starts at G^(t+2) and strides by G^32;
    the first hit in (round, lane) order gives log eps = g(mu) + S_j (mirror)
    or g(mu) - S_j (direct).  None when the centre comes within N steps."""
    s = math.isqrt(d)
    P = 2 * ((1 + s) // 2) - 1
    Q = (d - P * P) // 2
    table = {(2, P): ("d", 0)}
    S = _c(P)
    for _ in range(N):
        q = (P + s) // Q
        Pn = q * Q - P
        Qn = (d - Pn * Pn) // Q
        if Qn == Q or Pn == P:
            return None
        table.setdefault((Q, P), ("d", S % 3))
        table.setdefault((Q, Pn), ("m", S % 3))
        S += _c(Pn)
        P, Q = Pn, Qn
    G = (Q // 2, P, S % 3)
    mu = [comp.mul(d, G, G, nucomp)]
    for _ in range(31):
        mu.append(comp.mul(d, mu[-1], G, nucomp))
    stride = comp.mul(d, mu[29], G, nucomp)  # G^32 = G^31 * G
    for _ in range(100000):
        for a, b, g in mu:
            hit = table.get((2 * a, b))
            if hit:
                kind, Sj = hit
                return (g + Sj) % 3 if kind == "m" else (g - Sj) % 3
        mu = [comp.mul(d, m, stride, nucomp) for m in mu]
    raise AssertionError("no hit")


@pytest.mark.parametrize("nucomp", [False, True], ids=["textbook", "nucomp"])
def test_giant_step_search_model_matches_oracle(infra_host, orc, nucomp):
    rng = np.random.default_rng(31 + nucomp)
    comp = _Composer(infra_host)
    try:
        n = 0
        while n < 12:
            d = int(rng.integers(10**9 // 8, 10**11 // 8)) * 8 + 5
            if not orc.in_D(d):
                continue
            got = _search_log(comp, d, 64, nucomp)
            if got is None:
                continue  # short period: the baby phase ends it
            rc, theta, _ = orc.walk_mod2(d)
            assert rc == 0 and got == theta - 1, (d, got, theta)
            n += 1
    finally:
        comp.close()


def _first_states(d, k):
    """The first k states (Q_j, P_j, S_j mod 3, delta_j) of the cycle from a_1."""
    s = math.isqrt(d)
    rd = math.sqrt(d)
    P = 2 * ((1 + s) // 2) - 1
    Q = (d - P * P) // 2
    S = _c(P)
    delta = math.log((P + rd) / 2)
    out = [(Q, P, S % 3, delta)]
    Qp = 2
    while len(out) < k:
        q = (P + s) // Q
        Pn = q * Q - P
        Qn = Qp + q * (P - Pn)
        S += _c(Pn)
        delta += math.log((Pn + rd) / Q)
        Qp, P, Q = Q, Pn, Qn
        out.append((Q, P, S % 3, delta))
    return out


@pytest.mark.parametrize("lo,hi", [(10**6, 10**8), (10**10, 10**11), (10**12, 2 * 10**12),
                                   (2**44 - 10**10, 2**44)])
def test_lean_product_lands_on_the_cycle_with_its_class(infra_host, orc, lo, hi):
    """The search's two lean products -- the textbook one (fp32 Euclid, c of
    the second ideal precomputed, residues by float estimates) and the lean
    NUCOMP (fp32 Euclid and partial Euclid, exact divisions by float
    estimates, the gamma class in 32-bit words) -- on random pairs of early
    cycle states, equal states (squares) and pairs whose norms share a factor
    included: a reduced state of the cycle, with that state's class, within
    log d of the sum of the two distances, and Q_{-1} = (d - P^2)/Q.  Most
    lean textbook products equal the general textbook code's term for term
    (the two can differ by where the reduction stops on an already reduced
    product).  The lean NUCOMP starts from the forms (a, -P, w) with w small,
    where the general code takes -(P mod 2a): equivalent forms, whose
    near-reduced products may reduce to different states near the same
    distance."""
    rng = np.random.default_rng(lo % 97 + 7)
    lines, expect = [], []
    common = 0
    for d in _pick_d_fast(orc, rng, lo, hi, 8):
        st = _first_states(d, 1400)  # all inside the first period (_pick_d_fast)
        index = {(Q, P): (j, S, dl) for j, (Q, P, S, dl) in enumerate(st)}
        pairs = [tuple(int(x) for x in rng.integers(0, 500, size=2)) for _ in range(150)]
        pairs += [(5, 5), (40, 40), (0, 0)]
        for i, k in pairs:
            (Qi, Pi, Si, di), (Qk, Pk, Sk, dk) = st[i], st[k]
            common += math.gcd(Qi // 2, Qk // 2) > 1
            lines.append("%d %d %d %d %d %d %d" % (d, Qi // 2, Pi, Si, Qk // 2, Pk, Sk))
            expect.append((d, index, di + dk))
    r = subprocess.run([infra_host], input="\n".join(lines) + "\n", capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    rows = [row for row in r.stdout.split("\n") if row.strip()]
    assert len(rows) == len(lines)
    same_t = 0
    for line, (d, index, dsum), row in zip(lines, expect, rows):
        okT, aT, bT, gT, okN, aN, bN, gN, okL, aL, bL, gL, okM, aM, bM, gM = map(int, row.split())
        assert okT == 1 and okN == 1 and okL == 1 and okM == 1, line
        for a, b, g in ((aL, bL, gL), (aM, bM, gM)):
            assert (2 * a, b) in index, line
            j, S, dj = index[(2 * a, b)]
            assert g == S, line
            assert abs(dj - dsum) <= math.log(d), line
        same_t += (aL, bL, gL) == (aT, bT, gT)
    assert common > 10
    assert same_t > 0.9 * len(rows)


def _pick_d_fast(orc, rng, lo, hi, k, min_period=1500):
    """k d in D from [lo, hi) whose period exceeds min_period states."""
    out = []
    while len(out) < k:
        d = int(rng.integers(lo // 8, hi // 8)) * 8 + 5
        if orc.in_D(d) and orc.walk_mod2(d)[2] > min_period:
            out.append(d)
    return out
