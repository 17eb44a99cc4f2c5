"""GPU parity of the lane-per-d infrastructure search (EIS_GIANT_LANE).

With EIS_OPT_GIANT_THRESHOLD = N the recording walk keeps the marked states
of its first N baby steps and hands every d whose centre has not come yet to
the giant-step kernel.  Every result must equal the oracle's: per-candidate
codes and generator classes element by element on ranges the oracle walks in
seconds (spanning several sieve tiles, ragged tails and several rounds of the
survivor queue), sampled candidates where it cannot, and the whole benchmark
window [1e11 - 1e9, 1e11] bit for bit against the baby walk alone (plus the
paper's Table 1 total inside it).  The fallback walk (a giant cycle's walk
past its cap) and the decline (too few marked states) must give the same
results as well.
"""
import numpy as np
import pytest

import paper_2507_06579_gb300 as E
from paper_2507_06579_gb300 import workloads as W
from test_oracle import paper

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    E.build()
    c = E.Context(0)
    c.set_option(E.EIS_OPT_STEP_LIMIT, 1 << 25)
    yield c
    c.close()


class _opts:
    """Set context options for the duration of a block, then restore them."""

    def __init__(self, ctx, **kv):
        self.ctx = ctx
        self.kv = {getattr(E, "EIS_OPT_" + k.upper()): v for k, v in kv.items()}

    def __enter__(self):
        self.old = {k: self.ctx.get_option(k) for k in self.kv}
        for k, v in self.kv.items():
            self.ctx.set_option(k, v)

    def __exit__(self, *exc):
        for k, v in self.old.items():
            self.ctx.set_option(k, v)


def _codes(ctx, lo, hi):
    f, s, _ = ctx.classify_range(lo, hi)
    n, _ = E.num_candidates(lo, hi)
    fl = np.unpackbits(np.asarray(f, np.uint32).view(np.uint8), bitorder="little")[:n]
    sq = np.unpackbits(np.asarray(s, np.uint32).view(np.uint8), bitorder="little")[:n]
    return np.where(fl == 1, 2, sq).astype(np.uint8)


@pytest.mark.parametrize("compose", [E.EIS_COMPOSE_TEXTBOOK, E.EIS_COMPOSE_NUCOMP],
                         ids=["textbook", "nucomp"])
@pytest.mark.parametrize("N,m", [(512, 8), (1024, 16), (1536, 32)])
def test_codes_and_classes_match_oracle(ctx, orc, compose, N, m):
    """2^18 + 37 candidates near 1e9 (every d walked by the oracle), three
    rounds of the queue, per-candidate codes and classes."""
    lo = 10**9 - 8 * 300_000
    hi = lo + 8 * ((1 << 18) + 37)
    ref = orc.classify_range(lo, hi, thetas=True)
    with _opts(ctx, giant_threshold=N, mark_every=m, giant_compose=compose,
               giant_kernel=E.EIS_GIANT_LANE, bsgs_chunk=100_000):
        codes = _codes(ctx, lo, hi)
        st = ctx.stats()
        logs = ctx.classify_range_log(lo, hi)
    assert st["deferred"] > 10_000            # most d really went through the search
    assert st["giant_steps"] > st["deferred"]
    assert np.array_equal(codes, ref["codes"])
    assert np.array_equal(logs, ref["thetas"])


def test_benchmark_window_equals_the_walk(ctx):
    """[1e11 - 1e9, 1e11]: flags and square-free bitmaps identical to the
    baby walk alone; the Table 1 total of [9.99e10, 1e11] inside it."""
    lo, hi = W.CFG_TOP
    with _opts(ctx, giant_threshold=0):
        f0, s0, c0 = ctx.classify_range(lo, hi)
    with _opts(ctx, giant_threshold=1536, mark_every=16, giant_kernel=E.EIS_GIANT_LANE):
        f1, s1, c1 = ctx.classify_range(lo, hi)
        st = ctx.stats()
        iv = paper()["table1_totals"]["intervals"][3]
        total = ctx.count_range(iv["lo"], iv["hi"])
    assert c1 == c0
    assert np.array_equal(f1, f0) and np.array_equal(s1, s0)
    assert st["deferred"] > 0.8 * st["in_D"]
    assert total == iv["total"]


@pytest.mark.parametrize("lo,hi,k", [
    (10**12 - 8 * (1 << 18), 10**12, 40),                 # 1e12
    (4389999000000, 4389999000000 + 8 * (1 << 18), 12),   # fast quotient, just below its limit
    (E.EIS_D_LIMIT - 8 * (1 << 18) - 5, E.EIS_D_LIMIT, 8),  # corrected quotient, below 2^44
])
def test_large_d_sampled_against_oracle_and_walk(ctx, orc, lo, hi, k):
    with _opts(ctx, giant_threshold=2048, mark_every=16, giant_kernel=E.EIS_GIANT_LANE):
        logs = ctx.classify_range_log(lo, hi)
        st = ctx.stats()
    assert st["deferred"] > 0
    idx, d0 = W.sample_candidates(lo, hi, k, seed=13)
    for i in idx:
        d = d0 + 8 * int(i)
        rc, theta, _ = orc.walk_mod2(d)
        assert logs[i] == (0 if rc == orc.ORC_ENOTD else theta), d
    with _opts(ctx, giant_threshold=0):
        assert np.array_equal(ctx.classify_range_log(lo, hi), logs)


def test_fallback_and_decline_give_the_same_results(ctx, orc):
    """A walk cap of 4 steps sends most searches to the fallback walk; marks
    1 in 2048 leave too few marked states and the recording walk declines."""
    lo = 3 * 10**9
    hi = lo + 8 * ((1 << 18) + 5)
    ref = orc.classify_range(lo, hi)["codes"]
    with _opts(ctx, giant_threshold=1024, mark_every=16, bsgs_walk_cap=4,
               giant_kernel=E.EIS_GIANT_LANE):
        assert np.array_equal(_codes(ctx, lo, hi), ref)
        assert ctx.stats()["deferred"] > 0
    with _opts(ctx, giant_threshold=300, mark_every=2048, giant_kernel=E.EIS_GIANT_LANE):
        assert np.array_equal(_codes(ctx, lo, hi), ref)


def test_batched_intervals_with_the_search(ctx):
    """The 4096 seeded intervals in one plan: per-interval counts equal with
    and without the search."""
    blo, bhi = W.batched_intervals(n=4096, seed=4)
    with _opts(ctx, giant_threshold=0):
        p = ctx.plan_create(blo, bhi)
        p.launch()
        c0 = p.counts()
        p.destroy()
    with _opts(ctx, giant_threshold=2048, mark_every=16, giant_kernel=E.EIS_GIANT_LANE):
        p = ctx.plan_create(blo, bhi)
        p.launch()
        c1 = p.counts()
        st = p.stats()
        p.destroy()
    assert np.array_equal(c0, c1)
    assert st["deferred"] > 0


def test_pool_kept_for_the_next_plan_and_never_shared(ctx):
    """A freed plan's table pool goes to the context and the next plan takes
    it; two live plans never share one.  Plans built while another lives,
    launched on two streams at once, give the count of a plan alone, and the
    bytes in use come back to where they were (context tables and one kept
    pool)."""
    import torch
    lo, hi = 10**10, 10**10 + 8 * ((1 << 19) + 3)
    with _opts(ctx, giant_threshold=1024, mark_every=16, giant_kernel=E.EIS_GIANT_LANE):
        ref = ctx.count_range(lo, hi)
        used0 = ctx.get_option(E.EIS_OPT_MEM_IN_USE)
        a = ctx.plan_create([lo], [hi])
        b = ctx.plan_create([lo], [hi])
        s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
        a.launch(s1)
        b.launch(s2)
        torch.cuda.synchronize()
        assert int(a.counts()[0]) == ref and int(b.counts()[0]) == ref
        assert a.stats()["deferred"] > 0
        a.destroy()
        c = ctx.plan_create([lo], [hi])  # takes a's pool
        c.launch(s1)
        b.launch(s2)
        torch.cuda.synchronize()
        assert int(c.counts()[0]) == ref and int(b.counts()[0]) == ref
        b.destroy()
        c.destroy()
        assert ctx.get_option(E.EIS_OPT_MEM_IN_USE) == used0
