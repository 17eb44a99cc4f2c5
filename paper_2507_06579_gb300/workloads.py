"""Seeded synthetic workloads (inputs only; none of the method's arithmetic).

Both the CUDA path and the CPU oracle take their inputs from here, so the two
sides see the same intervals.  Every generator is a pure function of its seed
(NumPy PCG64).  The shapes follow the workloads of the paper's computation
(Section 3.1: pi_E(x) for x <= 10^11, Table 1's length-10^8 intervals) and
the benchmark configurations:

* ``CFG_SMALL``     every candidate in [5, 10^6]
* ``CFG_1E9``       every candidate in [5, 10^9]
* ``CFG_TOP``       the window [10^11 - 10^9, 10^11]
* ``batched_intervals``  4096 intervals [a, a+L), a log-uniform in
  [10^6, 10^12], L log-uniform in [10^3, 10^7]
* ``parity_windows``     short windows at log-uniform positions for
  element-by-element comparison with the oracle
* ``serving_stream``     Poisson arrivals of range-count and membership
  requests
"""
from __future__ import annotations

import numpy as np

# Half-open [lo, hi) forms of the closed intervals of the configurations.
CFG_SMALL = (5, 10**6 + 1)
CFG_1E9 = (5, 10**9 + 1)
CFG_TOP = (10**11 - 10**9, 10**11 + 1)

# Table 1 intervals (closed in the paper; their endpoints are multiples of 8,
# never == 5 mod 8, so open and closed agree).
TABLE1 = [(0, 10**8), (9 * 10**8, 10**9), (99 * 10**8, 10**10), (999 * 10**8, 10**11)]


def log_uniform_int(rng: np.random.Generator, lo: float, hi: float, size=None):
    return np.floor(np.exp(rng.uniform(np.log(lo), np.log(hi), size=size))).astype(np.int64)


def batched_intervals(n: int = 4096, seed: int = 4, a_range=(1e6, 1e12), len_range=(1e3, 1e7)):
    """n intervals [a, a+L): a log-uniform in a_range, L log-uniform in len_range."""
    rng = np.random.Generator(np.random.PCG64(seed))
    a = log_uniform_int(rng, *a_range, size=n)
    L = log_uniform_int(rng, *len_range, size=n)
    lo = a.astype(np.uint64)
    hi = (a + L).astype(np.uint64)
    return lo, hi


def parity_windows(n: int = 24, seed: int = 3, pos_range=(1e6, 1e12), work: float = 1e8):
    """n windows [lo, lo + w) at log-uniform positions.  The width shrinks as
    sqrt(lo) grows so that a full-period CPU walk of every candidate costs
    about `work` steps: near x a period averages ~0.14 sqrt(x) steps and ~81%
    of the candidates are square-free, so w ~ 8 work / (0.11 sqrt(x))."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pos = log_uniform_int(rng, *pos_range, size=n)
    out = []
    for p in pos:
        p = int(p)
        w = int(np.clip(73.0 * work / np.sqrt(p), 2000, 2e5))
        out.append((p, p + w))
    return out


def sample_candidates(lo: int, hi: int, k: int, seed: int = 7):
    """k distinct candidate indices of [lo, hi) (d == 5 mod 8), sorted."""
    d0 = lo + ((13 - lo % 8) % 8)
    n = (hi - d0 + 7) // 8 if hi > d0 else 0
    rng = np.random.Generator(np.random.PCG64(seed))
    k = min(k, n)
    idx = rng.choice(n, size=k, replace=False) if k else np.zeros(0, dtype=np.int64)
    return np.sort(idx.astype(np.int64)), d0


def serving_stream(n: int, rate: float, seed: int = 5, frac_member: float = 0.1,
                   a_range=(1e6, 1e12), len_range=(1e2, 1e6), d_max: float = 1e12):
    """Poisson arrivals at `rate` req/s.  Returns a list of
    (t_arrival_s, kind, lo, hi) with kind 'count' ([lo, hi) range count) or
    'member' (single d = lo, hi = lo + 1; d == 5 mod 8, random below d_max; the
    caller filters square-free d)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate, size=n)
    t = np.cumsum(gaps)
    kinds = rng.uniform(size=n) < frac_member
    a = log_uniform_int(rng, *a_range, size=n)
    L = log_uniform_int(rng, *len_range, size=n)
    dm = rng.integers(0, int(d_max) // 8, size=n) * 8 + 5
    out = []
    for i in range(n):
        if kinds[i]:
            out.append((float(t[i]), "member", int(dm[i]), int(dm[i]) + 1))
        else:
            out.append((float(t[i]), "count", int(a[i]), int(a[i] + L[i])))
    return out
