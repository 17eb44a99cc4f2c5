"""A journaled sweep on the GPU reproduces the paper's pi_E(10^8)."""
import numpy as np
import pytest

import paper_2507_06579_gb300 as E
from paper_2507_06579_gb300 import sweep
from test_oracle import count_D_mobius, paper

pytestmark = pytest.mark.gpu


def test_sweep_to_1e8_matches_table1(tmp_path):
    E.build()
    iv = paper()["table1_totals"]["intervals"][0]
    blocks = sweep.plan_blocks(0, 10**8 + 1)
    path = str(tmp_path / "sweep.jsonl")
    with E.Context(0) as ctx:
        count = sweep.gpu_counter(ctx)
        # stop half-way, then resume from the journal
        half = blocks[: len(blocks) // 2]
        sweep.run_sweep(count, half, sweep.Journal(path), batch=4)
        tD, tE = sweep.run_sweep(count, blocks, sweep.Journal(path), batch=4)
    assert tE == iv["total"]
    assert tD == count_D_mobius(0, 10**8 + 1)
    curve = sweep.pi_E_curve(sweep.Journal(path), 0)
    assert curve[-1] == (10**8, tD, tE)
    assert all(b[2] >= a[2] and b[1] >= a[1] for a, b in zip(curve, curve[1:]))


def test_plan_counts_D_matches_oracle(orc):
    E.build()
    lo = np.array([5, 10**6, 10**9 + 1], dtype=np.uint64)
    hi = np.array([100_001, 10**6 + 80_000, 10**9 + 40_000], dtype=np.uint64)
    with E.Context(0) as ctx:
        plan = ctx.plan_create(lo, hi)
        plan.launch()
        nD, nE = plan.counts_D(), plan.counts()
        plan.destroy()
    for i in range(len(lo)):
        rD, rE, _ = orc.count_range(int(lo[i]), int(hi[i]))
        assert (int(nD[i]), int(nE[i])) == (rD, rE)
