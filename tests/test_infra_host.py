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
        okT, aT, bT, gT, okN, aN, bN, gN = map(int, row.split())
        assert okT == 1 and okN == 1, (d, i, k)
        for a, b, g in ((aT, bT, gT), (aN, bN, gN)):
            assert (2 * a, b) in index, (d, i, k, a, b)  # a reduced state of the cycle
            j, S, dj = index[(2 * a, b)]
            assert g == S, (d, i, k, j)                  # with that state's class
            # near the sum of the two distances (a reduction ends within about
            # log d of it)
            assert abs(dj - dsum) <= math.log(d), (d, i, k, j, dj, dsum)
        n_small += min(i, k) < 3
    assert len(rows) - 1 == len(expect) and n_small > 0
