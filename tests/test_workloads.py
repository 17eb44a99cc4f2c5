"""The seeded synthetic inputs: reproducible, and with the shapes the design
states (interval and length distributions, arrival process, candidate
sampling)."""
import numpy as np

from paper_2507_06579_gb300 import workloads as W


def test_batched_intervals_match_the_stated_recipe():
    lo, hi = W.batched_intervals(n=4096, seed=4)
    lo2, hi2 = W.batched_intervals(n=4096, seed=4)
    assert np.array_equal(lo, lo2) and np.array_equal(hi, hi2)
    a = lo.astype(np.float64)
    L = (hi - lo).astype(np.float64)
    assert a.min() >= 1e6 and a.max() < 1e12
    assert L.min() >= 1e3 and L.max() < 1e7
    # log-uniform: log10 spread evenly over 6 and 4 decades
    assert abs(np.log10(a).mean() - 9.0) < 0.1
    assert abs(np.log10(L).mean() - 5.0) < 0.1
    # about 4.45e9 of total width, i.e. about 4.5e8 discriminants
    assert 4.0e9 < L.sum() < 4.9e9


def test_serving_stream_is_poisson_with_a_tenth_membership():
    reqs = W.serving_stream(20000, 1000.0, seed=5)
    t = np.array([r[0] for r in reqs])
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(t)
    assert abs(gaps.mean() - 1e-3) < 5e-5          # rate 1000 / s
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.05  # exponential gaps
    kinds = [r[1] for r in reqs]
    frac = kinds.count("member") / len(kinds)
    assert abs(frac - 0.1) < 0.01
    for _, kind, lo, hi in reqs[:2000]:
        if kind == "member":
            assert lo % 8 == 5 and hi == lo + 1 and lo < 1e12
        else:
            assert 1e6 <= lo < 1e12 and 1e2 <= hi - lo < 1e6
    assert W.serving_stream(50, 10.0, seed=5) == W.serving_stream(50, 10.0, seed=5)


def test_parity_windows_and_candidate_samples():
    wins = W.parity_windows(n=64, seed=3)
    assert wins == W.parity_windows(n=64, seed=3)
    for lo, hi in wins:
        assert 1e6 <= lo < 1e12 and 2000 <= hi - lo <= 2e5
    lo, hi = W.CFG_TOP
    idx, d0 = W.sample_candidates(lo, hi, 1000, seed=7)
    assert d0 % 8 == 5 and lo <= d0 < lo + 8
    n = (hi - d0 + 7) // 8
    assert len(idx) == 1000 and len(set(idx.tolist())) == 1000
    assert idx.min() >= 0 and idx.max() < n and np.all(np.diff(idx) > 0)
    assert d0 + 8 * int(idx.max()) < hi
