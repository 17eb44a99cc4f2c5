"""Sweeps across ranks, checkpoint and resume -- on the CPU.

Blocks of a range are dealt round-robin to the ranks; each rank counts its
share and the only exchange is one sum of counts.  These tests run two gloo
ranks as processes with the CPU oracle standing in for the per-block GPU
count, and inject failures on the host: a rank that raises mid-sweep, a
journal with a torn last line.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

from paper_2507_06579_gb300 import sweep

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WORKER = os.path.join(ROOT, "tests", "_dist_worker.py")


def test_blocks_partition_the_range():
    for lo, hi, blk in [(0, 10**6, 1 << 14), (12345, 98765, 1000), (5, 6, 1 << 24), (7, 7, 64)]:
        blocks = sweep.plan_blocks(lo, hi, blk)
        assert sum(b - a for a, b in blocks) == max(0, hi - lo)
        for (a, b), (c, _) in zip(blocks, blocks[1:]):
            assert b == c and b % blk == 0
        for world in (1, 2, 3, 5):
            shares = [sweep.assign(blocks, r, world) for r in range(world)]
            assert sorted(x for s in shares for x in s) == sorted(blocks)
            assert max(map(len, shares)) - min(map(len, shares)) <= 1


def test_journal_resume_counts_each_block_once(orc, tmp_path):
    lo, hi, blk = 5, 400_001, 1 << 15
    blocks = sweep.plan_blocks(lo, hi, blk)
    path = str(tmp_path / "j.jsonl")
    seen = []

    def counter(limit):
        def count(chunk):
            if limit is not None and len(seen) >= limit:
                raise RuntimeError("crash")
            seen.extend(chunk)
            return [orc.count_range(a, b)[:2] for a, b in chunk]
        return count

    with pytest.raises(RuntimeError):
        sweep.run_sweep(counter(3), blocks, sweep.Journal(path), batch=2)
    first = list(seen)
    tD, tE = sweep.run_sweep(counter(None), blocks, sweep.Journal(path), batch=2)
    assert len(seen) == len(blocks) and len(set(seen)) == len(blocks)
    assert set(first) <= set(seen[:len(first)])
    nD, nE, _ = orc.count_range(lo, hi)
    assert (tD, tE) == (nD, nE)
    curve = sweep.pi_E_curve(sweep.Journal(path), lo)
    assert curve[-1] == (hi - 1, nD, nE)
    # a torn last line (crash during a write) is ignored
    with open(path, "a") as f:
        f.write('{"lo": 1, "hi"')
    assert len(sweep.Journal(path).rows) == len(blocks)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run_ranks(tmp_path, lo, hi, blk, fail=None):
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port))
        args = [sys.executable, WORKER, str(lo), str(hi), str(blk), str(tmp_path / "journal"),
                str(tmp_path / "out")]
        if fail is not None and fail[0] == r:
            args.append(str(fail[1]))
        procs.append(subprocess.Popen(args, env=env, stdout=subprocess.PIPE, stderr=subprocess.STDOUT))
    for p in procs:
        p.communicate(timeout=240)
    return [json.load(open(str(tmp_path / "out") + ".rank%d" % r)) for r in range(2)]


def test_two_ranks_sum_to_the_oracle(orc, tmp_path):
    lo, hi, blk = 5, 300_001, 1 << 14
    res = _run_ranks(tmp_path, lo, hi, blk)
    nD, nE, _ = orc.count_range(lo, hi)
    for r in res:
        assert r["status"] == "ok"
        assert (r["pi_D"], r["pi_E"]) == (nD, nE)
    # round-robin: the ranks counted disjoint blocks
    b0 = {tuple(b) for c in res[0]["calls"] for b in c}
    b1 = {tuple(b) for c in res[1]["calls"] for b in c}
    assert not (b0 & b1) and len(b0) + len(b1) == len(sweep.plan_blocks(lo, hi, blk))


def test_rank_failure_then_resume(orc, tmp_path):
    lo, hi, blk = 5, 300_001, 1 << 14
    # rank 1 dies after one batch; rank 0's sum then times out
    res = _run_ranks(tmp_path, lo, hi, blk, fail=(1, 1))
    assert res[1]["status"].startswith("error")
    assert res[0]["status"].startswith("error")
    done1 = len(res[1]["calls"])
    assert done1 == 1
    # restart both: the journals keep what was finished
    res2 = _run_ranks(tmp_path, lo, hi, blk)
    nD, nE, _ = orc.count_range(lo, hi)
    for r in res2:
        assert r["status"] == "ok" and (r["pi_D"], r["pi_E"]) == (nD, nE)
    redone = {tuple(b) for c in res2[1]["calls"] for b in c}
    first = {tuple(b) for c in res[1]["calls"] for b in c}
    assert not (redone & first)  # rank 1 did not recount its journaled blocks
    assert res2[0]["calls"] == []  # rank 0 had finished everything before the timeout


def test_bench_rank_windows_are_disjoint():
    import bench
    ws = [bench.rank_window(r, 10**9) for r in range(8)]
    for (lo, hi) in ws:
        assert hi - lo == 10**9 + 1 and hi <= 10**11 + 1
    for (a, b), (c, d) in zip(ws, ws[1:]):
        assert d <= a + 1  # rank r+1's window lies below rank r's
    # windows overlap only in their shared endpoint, which is == 0 mod 8 (no candidate)
    for (a, b), (c, d) in zip(ws, ws[1:]):
        assert d - 1 == a and a % 8 == 0
