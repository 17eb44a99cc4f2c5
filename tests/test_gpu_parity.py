"""GPU parity: the CUDA path against the CPU oracle, bit-exact.

Every comparison is on integers (per-candidate codes, logs, flags, counts):
the bar is exact equality.  Small sizes are compared element by element
(spanning several sieve tiles and ragged tails); the full benchmark window
[10^11 - 10^9, 10^11] is compared on sampled candidates walked one by one by
the oracle, plus the paper's Table 1 total inside it and a Moebius count of D.
"""
import concurrent.futures as cf

import math

import numpy as np
import pytest

import paper_2507_06579_gb300 as E
from paper_2507_06579_gb300 import workloads as W
from test_oracle import count_D_mobius, paper

pytestmark = pytest.mark.gpu

MODES = [E.EIS_MODE_PERSISTENT, E.EIS_MODE_PLAIN]
MODE_IDS = ["persistent", "plain"]


@pytest.fixture(scope="module")
def ctx():
    E.build()
    c = E.Context(0)
    c.set_option(E.EIS_OPT_STEP_LIMIT, 1 << 25)
    yield c
    c.close()


@pytest.fixture
def in_mode(ctx, request):
    ctx.set_option(E.EIS_OPT_MODE, request.param)
    yield request.param
    ctx.set_option(E.EIS_OPT_MODE, E.EIS_MODE_PERSISTENT)


def unpack(words, n):
    bits = np.unpackbits(np.asarray(words, dtype=np.uint32).view(np.uint8), bitorder="little")
    return bits[:n]


# ---------------------------------------------------------------- points

def test_known_points(ctx):
    for d in (5, 13, 21, 29, 53, 61):
        assert ctx.is_eisenstein(d) is False
    for d in [37, 101] + paper()["examples_in_E"]["d"]:
        assert ctx.is_eisenstein(d) is True
    for d in (45, 8, 9, 125, 5 * 9 * 49):
        with pytest.raises(E.EisError) as ei:
            ctx.is_eisenstein(d)
        assert ei.value.code == E.EIS_ENOTD
    with pytest.raises(E.EisError) as ei:
        ctx.is_eisenstein(E.EIS_D_LIMIT + 5)
    assert ei.value.code == E.EIS_ERANGE


def test_membership_square_factor_at_the_scan_bound(ctx, orc):
    """A single query scans only the odd primes p with p^2 <= d: d = 5 p^2 with
    p the largest prime below a bound (the last prime the scan needs, at
    several sizes, up to 2^44) is refused as not square-free; d = 5 p^2 + 8,
    square-free or not, matches the oracle."""
    def prevprime(n):
        n -= 1
        while any(n % q == 0 for q in range(2, math.isqrt(n) + 1)):
            n -= 1
        return n

    for bound in (7, 1000, 10**5, math.isqrt(E.EIS_D_LIMIT // 5)):
        p = prevprime(bound)
        d = 5 * p * p
        assert d % 8 == 5 and d < E.EIS_D_LIMIT
        with pytest.raises(E.EisError) as ei:
            ctx.is_eisenstein(d)
        assert ei.value.code == E.EIS_ENOTD, d
        d2 = d + 8
        rc, theta, _ = orc.walk_mod2(d2)
        if rc == orc.ORC_ENOTD:
            with pytest.raises(E.EisError):
                ctx.is_eisenstein(d2)
        else:
            assert ctx.is_eisenstein(d2) == (theta == 1), d2


def test_is_eisenstein_matches_oracle(ctx, orc):
    rng = np.random.default_rng(11)
    ds = [int(x) * 8 + 5 for x in rng.integers(1, 10**11 // 8, size=40)]
    ds += [int(x) * 8 + 5 for x in rng.integers(10**11 // 8, 10**12 // 8, size=10)]
    for d in ds:
        rc, theta, _ = orc.walk_mod2(d)
        if rc == orc.ORC_ENOTD:
            with pytest.raises(E.EisError):
                ctx.is_eisenstein(d)
        else:
            assert rc == 0
            assert ctx.is_eisenstein(d) == (theta == 1), d


# ---------------------------------------------------------------- small configuration

@pytest.mark.parametrize("in_mode", MODES, ids=MODE_IDS, indirect=True)
def test_small_config_codes(ctx, orc, in_mode):
    lo, hi = W.CFG_SMALL
    ref = orc.classify_range(lo, hi)["codes"]
    codes, cnt = ctx.classify_range_u8(lo, hi)
    assert codes.shape == ref.shape
    assert np.array_equal(codes, ref)
    assert cnt == int((ref == 2).sum())
    assert ctx.count_range(lo, hi) == cnt


def test_small_config_log_matches_theta(ctx, orc):
    lo, hi = W.CFG_SMALL
    ref = orc.classify_range(lo, hi, thetas=True)
    g = ctx.classify_range_log(lo, hi)
    # log byte 1 + log_omega(eps mod 2) and theta code x + 2y coincide:
    # 1 <-> 1, omega <-> 2, omega^2 = 1 + omega <-> 3; 0 = not in D.
    assert np.array_equal(g, ref["thetas"])


@pytest.mark.parametrize("in_mode", MODES, ids=MODE_IDS, indirect=True)
@pytest.mark.parametrize("lo,hi", [
    (10, 10), (0, 5), (5, 6), (0, 6), (13, 14), (6, 13), (0, 0),
    (100, 100 + 8 * 37 + 3),                       # ragged, under one word
    (10**6, 10**6 + 8 * (2 * 65536 + 37)),         # three tiles, ragged tail
    (10**9 + 3, 10**9 + 8 * 65536 + 11),           # exactly one tile + 1
    (E.EIS_D_LIMIT - 2000, E.EIS_D_LIMIT),         # top of the supported range
    (4389999990000, 4390000000000),                # fast quotient just below its limit
    (4390000000000 - 800, 4390000000000 + 800),    # a plan straddling that limit
])
def test_edge_ranges(ctx, orc, in_mode, lo, hi):
    ref = orc.classify_range(lo, hi)["codes"]
    codes, cnt = ctx.classify_range_u8(lo, hi)
    assert np.array_equal(codes, ref), (lo, hi)
    f, s, c2 = ctx.classify_range(lo, hi)
    n = len(ref)
    assert np.array_equal(unpack(f, n), (ref == 2).astype(np.uint8))
    assert np.array_equal(unpack(s, n), (ref > 0).astype(np.uint8))
    if n % 32:
        # bits above the last candidate are zero
        assert int(f[-1]) >> (n % 32) == 0 and int(s[-1]) >> (n % 32) == 0
    assert cnt == c2 == int((ref == 2).sum())


def test_range_errors(ctx):
    with pytest.raises(E.EisError) as ei:
        ctx.count_range(10, 5)
    assert ei.value.code == E.EIS_EINVAL
    with pytest.raises(E.EisError) as ei:
        ctx.count_range(0, E.EIS_D_LIMIT + 1)
    assert ei.value.code == E.EIS_ERANGE


@pytest.mark.parametrize("in_mode", MODES, ids=MODE_IDS, indirect=True)
def test_parity_windows(ctx, orc, in_mode):
    for lo, hi in W.parity_windows(n=16):
        ref = orc.classify_range(lo, hi)["codes"]
        codes, _ = ctx.classify_range_u8(lo, hi)
        assert np.array_equal(codes, ref), (lo, hi)


# ---------------------------------------------------------------- paper values

def test_table1_totals(ctx):
    ivs = paper()["table1_totals"]["intervals"]
    los = [iv["lo"] for iv in ivs]
    his = [iv["hi"] for iv in ivs]
    got = ctx.count_batch(los, his)
    assert [int(x) for x in got] == [iv["total"] for iv in ivs]
    for iv in ivs[:2]:
        assert ctx.count_range(iv["lo"], iv["hi"]) == iv["total"]


def test_count_batch_matches_single_ranges(ctx, orc):
    lo, hi = W.batched_intervals(n=48, seed=9, a_range=(1e6, 1e10), len_range=(1e2, 3e4))
    got = ctx.count_batch(lo, hi)
    for i in range(len(lo)):
        assert int(got[i]) == ctx.count_range(int(lo[i]), int(hi[i]))
        assert int(got[i]) == orc.count_range(int(lo[i]), int(hi[i]))[1]


# ---------------------------------------------------------------- plans

def test_plan_relaunch_and_modes_agree(ctx):
    lo, hi = W.batched_intervals(n=64, seed=12, a_range=(1e6, 1e11), len_range=(1e3, 1e5))
    lo = list(lo) + [0, 5]
    hi = list(hi) + [0, 6]
    res = []
    for mode in MODES:
        plan = ctx.plan_create(lo, hi, mode)
        plan.launch()
        c1 = plan.counts()
        st = plan.stats()
        plan.launch()
        c2 = plan.counts()
        assert np.array_equal(c1, c2)
        assert st["baby_steps"] > 0 and st["in_E"] == int(c1.sum())
        fptr, sptr, off, tot = plan.bitmaps()
        assert fptr and sptr and tot > 0 and len(off) == len(lo)
        plan.destroy()
        res.append(c1)
    assert np.array_equal(res[0], res[1])


def test_device_outputs_and_stream(ctx):
    torch = pytest.importorskip("torch")
    lo, hi = 10**7, 10**7 + 8 * 100_003
    n, _ = E.num_candidates(lo, hi)
    nw = (n + 31) // 32
    f_h, s_h, c_h = ctx.classify_range(lo, hi)
    stream = torch.cuda.Stream()
    f_d = torch.zeros(nw, dtype=torch.int32, device="cuda")
    s_d = torch.zeros(nw, dtype=torch.int32, device="cuda")
    _, _, c_d = ctx.classify_range(lo, hi, flags_out=f_d, sqfree_out=s_d, stream=stream)
    torch.cuda.synchronize()
    assert c_d == c_h
    assert np.array_equal(f_d.cpu().numpy().view(np.uint32), f_h)
    assert np.array_equal(s_d.cpu().numpy().view(np.uint32), s_h)
    codes_d = torch.zeros(n, dtype=torch.uint8, device="cuda")
    ctx.classify_range_u8(lo, hi, codes_out=codes_d)
    codes_h, _ = ctx.classify_range_u8(lo, hi)
    assert np.array_equal(codes_d.cpu().numpy(), codes_h)


def test_step_limit_reports_error(ctx):
    ctx.set_option(E.EIS_OPT_STEP_LIMIT, 50)
    try:
        for mode in MODES:
            ctx.set_option(E.EIS_OPT_MODE, mode)
            with pytest.raises(E.EisError) as ei:
                ctx.count_range(10**10, 10**10 + 8000)
            assert ei.value.code == E.EIS_ESTEPS
    finally:
        ctx.set_option(E.EIS_OPT_STEP_LIMIT, 1 << 25)
        ctx.set_option(E.EIS_OPT_MODE, E.EIS_MODE_PERSISTENT)
    assert ctx.count_range(5, 10**6 + 1) > 0  # the context is still usable


# ---------------------------------------------------------------- full sizes

def _sampled_parity(orc, lo, hi, f, s, k, seed):
    idx, d0 = W.sample_candidates(lo, hi, k, seed=seed)
    fb = unpack(f, int(idx.max()) + 1 if len(idx) else 0)
    sb = unpack(s, int(idx.max()) + 1 if len(idx) else 0)
    ds = [d0 + 8 * int(i) for i in idx]
    with cf.ThreadPoolExecutor(max_workers=orc.default_threads()) as ex:
        res = list(ex.map(orc.walk_mod2, ds))
    for i, d, (rc, theta, _) in zip(idx, ds, res):
        if rc == orc.ORC_ENOTD:
            assert sb[i] == 0 and fb[i] == 0, d
        else:
            assert rc == 0
            assert sb[i] == 1 and fb[i] == (theta == 1), d


def _count_bits(words, a, b):
    """Set bits among candidates [a, b) of a bitmap."""
    bits = unpack(words, b)
    return int(bits[a:b].sum())


def test_full_top_window_persistent(ctx, orc):
    """The benchmark workload, in the benchmark's configuration."""
    lo, hi = W.CFG_TOP
    f, s, cnt = ctx.classify_range(lo, hi)
    n, d0 = E.num_candidates(lo, hi)
    assert len(f) == (n + 31) // 32
    _sampled_parity(orc, lo, hi, f, s, k=600, seed=21)
    # Table 1: #E cap [10^11 - 10^8, 10^11] = 3 345 503
    iv = paper()["table1_totals"]["intervals"][3]
    a = (iv["lo"] - d0 + 7) // 8
    assert _count_bits(f, a, n) == iv["total"]
    # #D over the window by inclusion-exclusion
    assert _count_bits(s, 0, n) == count_D_mobius(lo, hi)
    assert cnt == _count_bits(f, 0, n)


def test_full_top_window_plain_equals_persistent(ctx):
    lo, hi = W.CFG_TOP
    f1, s1, c1 = ctx.classify_range(lo, hi)
    ctx.set_option(E.EIS_OPT_MODE, E.EIS_MODE_PLAIN)
    try:
        f2, s2, c2 = ctx.classify_range(lo, hi)
    finally:
        ctx.set_option(E.EIS_OPT_MODE, E.EIS_MODE_PERSISTENT)
    assert c1 == c2
    assert np.array_equal(f1, f2) and np.array_equal(s1, s2)


def test_full_1e9_config(ctx, orc):
    lo, hi = W.CFG_1E9
    f, s, cnt = ctx.classify_range(lo, hi)
    n, d0 = E.num_candidates(lo, hi)
    _sampled_parity(orc, lo, hi, f, s, k=2000, seed=22)
    ivs = paper()["table1_totals"]["intervals"]
    for iv in ivs[:2]:
        a = max(0, (iv["lo"] - d0 + 7) // 8)
        b = (iv["hi"] - d0 + 7) // 8
        assert _count_bits(f, a, b) == iv["total"]
    assert _count_bits(s, 0, n) == count_D_mobius(lo, hi)


def test_full_batched_intervals(ctx, orc):
    """4096 seeded intervals in one persistent launch == the same intervals
    through the plain kernel; the cheapest intervals against the oracle; and
    sampled candidates of the expensive ones against the oracle one by one."""
    lo, hi = W.batched_intervals(n=4096, seed=4)
    counts = {}
    for mode in MODES:
        plan = ctx.plan_create(lo, hi, mode)
        plan.launch()
        counts[mode] = plan.counts()
        if mode == E.EIS_MODE_PERSISTENT:
            _, _, off, _ = plan.bitmaps()
            f_host, s_host = plan.copy_bitmaps()
        plan.destroy()
    assert np.array_equal(counts[E.EIS_MODE_PERSISTENT], counts[E.EIS_MODE_PLAIN])
    # the cheapest intervals (work ~ L sqrt(a)) in full against the oracle
    work = (hi - lo).astype(np.float64) * np.sqrt(lo.astype(np.float64))
    for i in np.argsort(work)[:40]:
        assert int(counts[E.EIS_MODE_PERSISTENT][i]) == orc.count_range(int(lo[i]), int(hi[i]))[1]
    # sampled candidates of the most expensive intervals
    rng = np.random.default_rng(5)
    for i in np.argsort(work)[-8:]:
        n, d0 = E.num_candidates(int(lo[i]), int(hi[i]))
        ks = rng.choice(n, size=min(n, 20), replace=False)
        ds = [d0 + 8 * int(k) for k in ks]
        with cf.ThreadPoolExecutor(max_workers=orc.default_threads()) as ex:
            res = list(ex.map(orc.walk_mod2, ds))
        base = int(off[i]) * 32
        for k, (rc, theta, _) in zip(ks, res):
            g = base + int(k)
            fbit = (int(f_host[g >> 5]) >> (g & 31)) & 1
            sbit = (int(s_host[g >> 5]) >> (g & 31)) & 1
            if rc == orc.ORC_ENOTD:
                assert sbit == 0 and fbit == 0
            else:
                assert sbit == 1 and fbit == int(theta == 1)

