"""Long sweeps of pi_E: blocks, ranks, checkpoint journal.

A sweep over [lo, hi) is cut into blocks of 2^24 consecutive integers
(aligned to multiples of 2^24).  Every d is independent, so blocks are dealt
round-robin to the ranks of a job -- the cost of a block grows like sqrt(d),
and dealing them in turn keeps the ranks balanced -- and each rank counts
its blocks with no device-side exchange.  The only communication is one sum
of uint64 counts at the end (torch.distributed all_reduce on CPU tensors:
gloo, or any backend).

Each finished block is appended to a JSON-lines journal; a restarted sweep
skips the blocks its journal already holds, so a rank that died mid-sweep
loses at most the blocks it had in flight.

Command line (one GPU, or one process per GPU under torchrun):

    python -m paper_2507_06579_gb300.sweep --hi 1e11 --journal sweep.jsonl

prints pi_E at every block boundary (as a JSON-lines curve file if --curve
is given) and the totals.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time
from typing import Callable, Dict, Iterable, List, Sequence, Tuple

BLOCK = 1 << 24


def plan_blocks(lo: int, hi: int, block: int = BLOCK) -> List[Tuple[int, int]]:
    """[lo, hi) cut at multiples of `block`."""
    if hi <= lo:
        return []
    out = []
    a = lo
    while a < hi:
        b = min(hi, (a // block + 1) * block)
        out.append((a, b))
        a = b
    return out


def assign(blocks: Sequence[Tuple[int, int]], rank: int, world: int) -> List[Tuple[int, int]]:
    """Round-robin share of `blocks` for `rank` of `world`."""
    return [blk for i, blk in enumerate(blocks) if i % world == rank]


class Journal:
    """Append-only JSON-lines record of finished blocks."""

    def __init__(self, path: str | None):
        self.path = path
        self.rows: Dict[Tuple[int, int], dict] = {}
        if path and os.path.exists(path):
            with open(path) as f:
                for line in f:
                    line = line.strip()
                    if not line:
                        continue
                    try:
                        r = json.loads(line)
                    except json.JSONDecodeError:
                        continue  # a torn last line from a crash
                    self.rows[(int(r["lo"]), int(r["hi"]))] = r

    def done(self, blk: Tuple[int, int]) -> bool:
        return blk in self.rows

    def add(self, blk: Tuple[int, int], nD: int, nE: int, extra: dict | None = None):
        r = {"lo": blk[0], "hi": blk[1], "nD": int(nD), "nE": int(nE)}
        if extra:
            r.update(extra)
        self.rows[blk] = r
        if self.path:
            with open(self.path, "a") as f:
                f.write(json.dumps(r) + "\n")
                f.flush()
                os.fsync(f.fileno())


CountFn = Callable[[Sequence[Tuple[int, int]]], List[Tuple[int, int]]]


def run_sweep(count_fn: CountFn, blocks: Iterable[Tuple[int, int]], journal: Journal,
              batch: int = 64, on_batch: Callable[[int], None] | None = None) -> Tuple[int, int]:
    """Count the blocks not yet in the journal, `batch` at a time.
    count_fn(list of (lo, hi)) -> list of (#D, #E).  Returns (#D, #E) over all
    the given blocks (journal rows included)."""
    todo = [b for b in blocks if not journal.done(b)]
    for i in range(0, len(todo), batch):
        chunk = todo[i:i + batch]
        res = count_fn(chunk)
        for blk, r in zip(chunk, res):
            journal.add(blk, r[0], r[1], {"cls": r[2]} if len(r) > 2 else None)
        if on_batch:
            on_batch(i + len(chunk))
    tD = tE = 0
    for b in blocks:
        r = journal.rows[b]
        tD += r["nD"]
        tE += r["nE"]
    return tD, tE


def all_reduce_sum(values: Sequence[int], group=None) -> List[int]:
    """Sum integer counts over the ranks of a torch.distributed job (CPU)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([int(v) for v in values], dtype=torch.int64)
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return [int(x) for x in t.tolist()]


def pi_E_curve(journal: Journal, lo: int = 0) -> List[Tuple[int, int, int]]:
    """(x, pi_D(x), pi_E(x)) at every block end x - 1, from journal rows that
    tile [lo, x) without gaps."""
    rows = sorted(journal.rows.values(), key=lambda r: r["lo"])
    out = []
    cD = cE = 0
    expect = lo
    for r in rows:
        if r["lo"] != expect:
            break
        cD += r["nD"]
        cE += r["nE"]
        expect = r["hi"]
        out.append((r["hi"] - 1, cD, cE))
    return out


def fit_five_sixths(curve: Sequence[Tuple[int, int, int]], x_min: float = 1e8) -> float:
    """Least-squares c in pi_E(x) ~ x/(3 pi^2) + c x^(5/6) over curve points
    with x >= x_min (Section 3.1 reports c ~ -0.024)."""
    num = den = 0.0
    for x, _, e in curve:
        if x < x_min:
            continue
        r = e - x / (3 * math.pi ** 2)
        t = x ** (5 / 6)
        num += r * t
        den += t * t
    return num / den if den else float("nan")


def fit_prime_coefficient(curve: Sequence[Tuple[int, int, int]], x_min: float = 1e8) -> float:
    """Least-squares c in pi_{E cap P}(x) ~ pi(x)/12 + c Li_{1/6}(x), with
    Li_{1/6}(x) = int_2^x dt / (t^(1/6) log t) (Section 3.2 reports c ~ -0.037).
    pi(x)/12 is taken as pi_{P, 5 mod 8}(x)/3 from the curve itself (primes
    == 5 mod 8 are a quarter of all primes), and the integral by the
    trapezoidal rule on a log grid."""
    import numpy as np
    pts = [(x, p, e) for x, p, e in curve if x >= x_min]
    if not pts:
        return float("nan")
    xs = np.array([float(x) for x, _, _ in pts])
    grid = np.exp(np.linspace(np.log(2.0), np.log(xs.max()), 200001))
    f = 1.0 / (grid ** (1 / 6) * np.log(grid))
    cum = np.concatenate([[0.0], np.cumsum(0.5 * (f[1:] + f[:-1]) * np.diff(grid))])
    li = np.interp(xs, grid, cum)
    resid = np.array([e - p / 3.0 for _, p, e in pts])
    return float((resid * li).sum() / (li * li).sum())


def gpu_counter(ctx, primes: bool = False, classes: bool = False):
    """count_fn over the GPU: one plan (one persistent launch) per batch.
    primes: count the prime d only (pi_{E cap P}, Section 3.2); classes: also
    return the class counts of eps_d in F_4* as a third element."""
    import numpy as np
    import paper_2507_06579_gb300 as E

    flags = (E.EIS_PLAN_PRIMES if primes else 0) | (E.EIS_PLAN_CLASSES if classes else 0)

    def count(chunk):
        lo = np.array([a for a, _ in chunk], dtype=np.uint64)
        hi = np.array([b for _, b in chunk], dtype=np.uint64)
        plan = ctx.plan_create(lo, hi, E.EIS_MODE_PERSISTENT, flags)
        try:
            plan.launch()
            nE = plan.counts()
            nD = plan.counts_D()
            cls = plan.class_counts() if classes else None
        finally:
            plan.destroy()
        if classes:
            return [(int(a), int(b), [int(x) for x in c]) for a, b, c in zip(nD, nE, cls)]
        return [(int(a), int(b)) for a, b in zip(nD, nE)]

    return count


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawTextHelpFormatter)
    ap.add_argument("--lo", type=float, default=0)
    ap.add_argument("--hi", type=float, required=True, help="sweep [lo, hi] (inclusive)")
    ap.add_argument("--journal", default=None)
    ap.add_argument("--curve", default=None, help="write (x, pi_D, pi_E) rows here")
    ap.add_argument("--batch", type=int, default=64, help="blocks per plan launch")
    ap.add_argument("--primes", action="store_true",
                    help="prime d only: pi_{E cap P} (Section 3.2)")
    ap.add_argument("--classes", action="store_true",
                    help="also count the class of eps_d in F_4* per block")
    args = ap.parse_args(argv)
    import torch
    import torch.distributed as dist
    import paper_2507_06579_gb300 as E

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world > 1:
        dist.init_process_group(backend="gloo")
    local = int(os.environ.get("LOCAL_RANK", "0"))
    lo, hi = int(args.lo), int(args.hi) + 1
    blocks = plan_blocks(lo, hi)
    mine = assign(blocks, rank, world)
    jpath = args.journal
    if jpath and world > 1:
        jpath = "%s.rank%d" % (jpath, rank)
    journal = Journal(jpath)
    E.build()
    t0 = time.time()
    with E.Context(local) as ctx:
        tD, tE = run_sweep(gpu_counter(ctx, args.primes, args.classes), mine, journal,
                           batch=args.batch)
    dt = time.time() - t0
    tD, tE = all_reduce_sum([tD, tE])
    if rank == 0:
        out = {"lo": lo, "hi": hi - 1, "pi_D": tD, "pi_E": tE, "blocks": len(blocks),
               "ranks": world, "seconds_rank0": dt, "primes_only": bool(args.primes)}
        if args.classes and world == 1:
            cls = [0, 0, 0]
            for b in mine:
                for g, v in enumerate(journal.rows[b].get("cls", [0, 0, 0])):
                    cls[g] += v
            out["classes"] = cls
        if world == 1 and not args.primes:
            curve = pi_E_curve(journal, lo)
            out["fit_c_5_6"] = fit_five_sixths(curve)
        if world == 1 and args.primes:
            curve = pi_E_curve(journal, lo)
            out["fit_c_prime"] = fit_prime_coefficient(curve)
            if args.curve:
                with open(args.curve, "w") as f:
                    for x, cD, cE in curve:
                        f.write(json.dumps({"x": x, "pi_D": cD, "pi_E": cE}) + "\n")
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
