"""Autotuner: picks persistent-walk / giant-step settings per d-decade; any
setting gives the same results."""
import json

import numpy as np
import pytest

import paper_2507_06579_gb300 as E

pytestmark = pytest.mark.gpu


def test_autotune_keeps_results_and_caches(orc, tmp_path):
    E.build()
    cache = str(tmp_path / "tune.json")
    lo, hi = 10**11 - 10**8, 10**11
    with E.Context(0) as ctx:
        r = ctx.autotune(lo, hi, cache_path=cache)
        assert r["cached"] is False and r["trials"] > 4
        assert r["ms_best"] <= r["ms_default"] + 1e-6
        assert 1 <= r["ctas_per_sm"] <= 64 and r["giant_threshold"] >= 0
        assert ctx.get_option(E.EIS_OPT_GIANT_THRESHOLD) == r["giant_threshold"]
        # results with the tuned setting are still exact
        w = (10**11 - 20_000, 10**11)
        ref = orc.classify_range(*w)["codes"]
        codes, _ = ctx.classify_range_u8(*w)
        assert np.array_equal(codes, ref)
    stored = json.load(open(cache))
    assert "decade_11" in stored
    with E.Context(0) as ctx2:
        r2 = ctx2.autotune(lo, hi, cache_path=cache)
        assert r2["cached"] is True
        assert ctx2.get_option(E.EIS_OPT_GIANT_THRESHOLD) == r["giant_threshold"]
        assert ctx2.get_option(E.EIS_OPT_CTAS_PER_SM) == r["ctas_per_sm"]


def test_decade_table_tuning_and_exact_results(orc):
    """eis_autotune_decades keys the lane search's settings by decade; a plan
    spanning two decades takes each d's row, and the codes equal the
    oracle's whatever the rows say; tables that break the rules are refused."""
    E.build()
    lo, hi = 10**10 - 8 * 150_000, 10**10 + 8 * 150_000
    ref = orc.classify_range(lo, hi)["codes"]
    with E.Context(0) as ctx:
        rows = ctx.autotune_decades(10**9, 2 * 10**10)
        assert [r[0] for r in rows] == [10**10, 10**11]
        assert all(b >= 0 and 2 <= m <= 4096 for _, b, m in rows)
        assert ctx.tune_table()
        codes, _ = ctx.classify_range_u8(lo, hi)
        assert np.array_equal(codes, ref)
        # an explicit table: the walk below 1e10, the search above it
        ctx.set_tune_table([(10**10, 0, 16), (10**11, 1024, 16)])
        assert ctx.tune_table() == [(10**10, 0, 16), (10**11, 1024, 16)]
        codes, _ = ctx.classify_range_u8(lo, hi)
        assert np.array_equal(codes, ref)
        assert 0 < ctx.stats()["deferred"] < int((ref > 0).sum())
        for bad in ([(10**10, 0, 1)], [(10**11, 0, 16), (10**10, 0, 16)], [(10**10, -1, 16)],
                    [(10**k, 0, 16) for k in range(3, 13)]):
            with pytest.raises(E.EisError):
                ctx.set_tune_table(bad)
        ctx.set_tune_table([])
        assert ctx.tune_table() == []
