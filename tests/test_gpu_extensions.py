"""Prime subsequence (Section 3.2) and the class of eps_d in F_4*, on the GPU,
against the oracle."""
import numpy as np
import pytest

import paper_2507_06579_gb300 as E

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    E.build()
    c = E.Context(0)
    yield c
    c.close()


def _bits(words, n):
    return np.unpackbits(np.asarray(words, dtype=np.uint32).view(np.uint8), bitorder="little")[:n]


WINDOWS = [(5, 400_001), (10**6, 10**6 + 8 * 70_001 + 3), (10**9, 10**9 + 120_000),
           (10**11 - 16_000, 10**11 + 1), (10**12 - 5_000, 10**12)]


@pytest.mark.parametrize("lo,hi", WINDOWS)
def test_prime_mode_matches_oracle(ctx, orc, lo, hi):
    ref = orc.classify_range_primes(lo, hi, thetas=True)
    n = len(ref["codes"])
    plan = ctx.plan_create([lo], [hi], E.EIS_MODE_PERSISTENT, E.EIS_PLAN_PRIMES | E.EIS_PLAN_CLASSES)
    plan.launch()
    f, s = plan.copy_bitmaps()
    nE, nP, cls = int(plan.counts()[0]), int(plan.counts_D()[0]), plan.class_counts()[0]
    plan.destroy()
    assert np.array_equal(_bits(s, n), (ref["codes"] > 0).astype(np.uint8))
    assert np.array_equal(_bits(f, n), (ref["codes"] == 2).astype(np.uint8))
    assert nP == int((ref["codes"] > 0).sum()) and nE == int((ref["codes"] == 2).sum())
    th = ref["thetas"][ref["codes"] > 0]
    assert [int(x) for x in cls] == [int((th == 1).sum()), int((th == 2).sum()), int((th == 3).sum())]


@pytest.mark.parametrize("lo,hi", WINDOWS[:4])
def test_class_counts_match_oracle(ctx, orc, lo, hi):
    ref = orc.classify_range(lo, hi, thetas=True)["thetas"]
    got = ctx.class_counts(lo, hi)
    assert got == [int((ref == 1).sum()), int((ref == 2).sum()), int((ref == 3).sum())]
    gp = ctx.class_counts(lo, hi, primes_only=True)
    refp = orc.classify_range_primes(lo, hi, thetas=True)["thetas"]
    assert gp == [int((refp == 1).sum()), int((refp == 2).sum()), int((refp == 3).sum())]
    # the E class is the Eisenstein count
    assert got[0] == ctx.count_range(lo, hi)
