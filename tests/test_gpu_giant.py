"""Giant steps (Algorithm 1 with classes in Z/3): parity with the oracle.

The warp-per-d baby-step giant-step kernel answers single-d queries and,
with a deferral threshold, takes over the long walks of a plan.  Every
result is compared exactly with the oracle's full-period walk: the flag,
and for the log output the class of eps_d in F_4*.  Each test runs with
both giant-step compositions: the textbook product followed by rho steps,
and NUCOMP/NUDUPL/NUCOMPchoose (Algorithms 2-4), whose class bookkeeping
goes through gamma mod 2O_K -- a wrong class there changes log eps_d.
"""
import concurrent.futures as cf

import numpy as np
import pytest

import paper_2507_06579_gb300 as E
from paper_2507_06579_gb300 import workloads as W
from test_oracle import paper

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=[E.EIS_COMPOSE_TEXTBOOK, E.EIS_COMPOSE_NUCOMP],
                ids=["textbook", "nucomp"])
def ctx(request):
    E.build()
    c = E.Context(0)
    c.set_option(E.EIS_OPT_GIANT_COMPOSE, request.param)
    assert c.get_option(E.EIS_OPT_GIANT_COMPOSE) == request.param
    yield c
    c.close()


def test_compose_option_values(ctx):
    with pytest.raises(E.EisError) as ei:
        ctx.set_option(E.EIS_OPT_GIANT_COMPOSE, 2)
    assert ei.value.code == E.EIS_EINVAL


def _random_D(orc, rng, lo, hi, k):
    out = []
    while len(out) < k:
        d = int(rng.integers(lo // 8, hi // 8)) * 8 + 5
        if orc.in_D(d):
            out.append(d)
    return out


@pytest.mark.parametrize("lo,hi,k", [(10**6, 10**9, 60), (10**9, 10**12, 60),
                                      (10**12, E.EIS_D_LIMIT, 24)])
def test_single_queries_match_oracle(ctx, orc, lo, hi, k):
    rng = np.random.default_rng(lo % 1000 + 17)
    ds = _random_D(orc, rng, lo, hi, k)
    with cf.ThreadPoolExecutor(max_workers=orc.default_threads()) as ex:
        ref = list(ex.map(orc.walk_mod2, ds))
    giants = 0
    for d, (rc, theta, per) in zip(ds, ref):
        assert rc == 0
        assert ctx.is_eisenstein(d) == (theta == 1), d
        giants += ctx.stats()["giant_steps"] > 0
    assert giants > 0  # the giant phase really ran
    # the single-lane walk (plain mode) agrees
    ctx.set_option(E.EIS_OPT_MODE, E.EIS_MODE_PLAIN)
    try:
        for d, (rc, theta, per) in list(zip(ds, ref))[:8]:
            assert ctx.is_eisenstein(d) == (theta == 1), d
    finally:
        ctx.set_option(E.EIS_OPT_MODE, E.EIS_MODE_PERSISTENT)


def test_single_query_edge_cases(ctx):
    assert ctx.is_eisenstein(37) and not ctx.is_eisenstein(5)
    for d in (45, 9 * 125, 10**9):
        with pytest.raises(E.EisError) as ei:
            ctx.is_eisenstein(d)
        assert ei.value.code == E.EIS_ENOTD


@pytest.fixture
def deferring(ctx):
    """Plans hand walks past 600 steps to the warp-per-d kernel."""
    ctx.set_option(E.EIS_OPT_GIANT_KERNEL, E.EIS_GIANT_WARP)
    ctx.set_option(E.EIS_OPT_GIANT_THRESHOLD, 600)
    yield ctx
    ctx.set_option(E.EIS_OPT_GIANT_THRESHOLD, 0)
    ctx.set_option(E.EIS_OPT_GIANT_KERNEL, E.EIS_GIANT_LANE)


def test_deferral_log_matches_oracle_theta(deferring, orc):
    ctx = deferring
    for lo, hi in [(5, 400_001), (10**9, 10**9 + 80_000), (10**11, 10**11 + 16_000)]:
        ref = orc.classify_range(lo, hi, thetas=True)
        g = ctx.classify_range_log(lo, hi)
        assert np.array_equal(g, ref["thetas"]), (lo, hi)
        st = ctx.stats()
        if lo >= 10**9:
            assert st["deferred"] > 0 and st["giant_steps"] > 0


def test_deferral_parity_windows(deferring, orc):
    ctx = deferring
    for lo, hi in W.parity_windows(n=10, seed=13):
        ref = orc.classify_range(lo, hi)["codes"]
        codes, _ = ctx.classify_range_u8(lo, hi)
        assert np.array_equal(codes, ref), (lo, hi)


def test_deferral_table1_and_full_window(deferring):
    ctx = deferring
    ivs = paper()["table1_totals"]["intervals"]
    got = ctx.count_batch([iv["lo"] for iv in ivs], [iv["hi"] for iv in ivs])
    assert [int(x) for x in got] == [iv["total"] for iv in ivs]
    lo, hi = W.CFG_TOP
    f1, s1, c1 = ctx.classify_range(lo, hi)
    st = ctx.stats()
    assert st["deferred"] > 0
    ctx.set_option(E.EIS_OPT_GIANT_THRESHOLD, 0)
    f2, s2, c2 = ctx.classify_range(lo, hi)
    ctx.set_option(E.EIS_OPT_GIANT_THRESHOLD, 600)
    assert c1 == c2 and np.array_equal(f1, f2) and np.array_equal(s1, s2)
