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
