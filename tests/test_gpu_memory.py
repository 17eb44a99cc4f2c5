"""Device-memory accounting of a context: every table the context holds is
charged to its budget once, a plan that does not fit in what is left is
refused with EIS_ENOMEM and charges nothing, and a destroyed plan gives its
bytes back."""
import pytest

import paper_2507_06579_gb300 as E

pytestmark = pytest.mark.gpu

NPRIMES = 295_946        # odd primes below 2^22 (the context's sieve table)
BYTES_PER_CAND = 4.25    # survivor queue (4) + square-free and flag bitmaps (1/8 each)


def test_context_tables_are_charged_and_plans_refused_past_the_budget():
    E.build()
    budget = 16 << 20
    with E.Context(0, mem_budget_bytes=budget) as c:
        assert c.get_option(E.EIS_OPT_MEM_BUDGET) == budget
        used0 = c.get_option(E.EIS_OPT_MEM_IN_USE)
        # the prime table (4 B per prime) and the square-free test table (16 B)
        assert used0 >= NPRIMES * (4 + 16)
        free = budget - used0
        big = int(free / BYTES_PER_CAND) + (1 << 20)       # does not fit
        with pytest.raises(E.EisError) as ei:
            c.plan_create([10**9], [10**9 + 8 * big], E.EIS_MODE_PERSISTENT)
        assert ei.value.code == E.EIS_ENOMEM
        assert c.get_option(E.EIS_OPT_MEM_IN_USE) == used0
        small = int(free / BYTES_PER_CAND) // 3             # fits
        p = c.plan_create([10**9], [10**9 + 8 * small], E.EIS_MODE_PERSISTENT)
        assert c.get_option(E.EIS_OPT_MEM_IN_USE) > used0
        p.launch()
        assert int(p.counts()[0]) == c.count_range(10**9, 10**9 + 8 * small)
        p.destroy()
        assert c.get_option(E.EIS_OPT_MEM_IN_USE) == used0


def test_read_only_memory_options():
    E.build()
    with E.Context(0, mem_budget_bytes=64 << 20) as c:
        for key in (E.EIS_OPT_MEM_BUDGET, E.EIS_OPT_MEM_IN_USE):
            with pytest.raises(E.EisError):
                c.set_option(key, 1)
