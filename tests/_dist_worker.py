"""Worker for the multi-process sweep tests (gloo on CPU, no GPU).

Environment: RANK, WORLD_SIZE, MASTER_ADDR, MASTER_PORT.  Arguments:
lo hi block journal_prefix out_json [fail_after]
Counts its round-robin share of the blocks with the CPU oracle (test
infrastructure), journals them, and sums (#D, #E) over the ranks.  With
fail_after = k the rank raises after k counted batches, before the sum.
"""
import datetime
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import torch.distributed as dist  # noqa: E402

import oracle  # noqa: E402
from paper_2507_06579_gb300 import sweep  # noqa: E402


def main():
    lo, hi, block = int(sys.argv[1]), int(sys.argv[2]), int(sys.argv[3])
    prefix, out_path = sys.argv[4], sys.argv[5]
    fail_after = int(sys.argv[6]) if len(sys.argv) > 6 else -1
    rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
    dist.init_process_group(backend="gloo", timeout=datetime.timedelta(seconds=8))
    blocks = sweep.plan_blocks(lo, hi, block)
    mine = sweep.assign(blocks, rank, world)
    journal = sweep.Journal("%s.rank%d" % (prefix, rank))
    calls = []

    def count(chunk):
        if fail_after >= 0 and len(calls) >= fail_after:
            raise RuntimeError("injected failure on rank %d" % rank)
        calls.append([list(b) for b in chunk])
        return [oracle.count_range(a, b)[:2] for a, b in chunk]

    status = "ok"
    try:
        tD, tE = sweep.run_sweep(count, mine, journal, batch=2)
        tD, tE = sweep.all_reduce_sum([tD, tE])
    except Exception as e:  # the injected failure, or the peer's timeout
        status = "error: %s" % type(e).__name__
        tD = tE = -1
    with open("%s.rank%d" % (out_path, rank), "w") as f:
        json.dump({"status": status, "pi_D": tD, "pi_E": tE, "calls": calls}, f)
    try:
        dist.destroy_process_group()
    except Exception:
        pass


if __name__ == "__main__":
    main()
