"""Single-discriminant queries from the command line.

    python -m paper_2507_06579_gb300.query 37 1901 7053
    python -m paper_2507_06579_gb300.query --near 1e12 --count 20 --seed 1

Each d goes through eis_is_eisenstein (the warp-per-d giant-step kernel by
default, or the single-lane walk with --plain) and prints one JSON line:
d, whether d is in D (square-free, d == 5 mod 8) and in E (eps_d == 1 mod
2O_K), the baby and giant steps taken, and the host-side latency in ms.
With --near, the d are random d == 5 mod 8 just below the given point
(numbers that are not square-free answer in_D false).
"""
from __future__ import annotations

import argparse
import json
import sys
import time


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawTextHelpFormatter)
    ap.add_argument("d", nargs="*", type=float, help="discriminants to classify")
    ap.add_argument("--near", type=float, default=None,
                    help="classify --count random d == 5 mod 8 in [near - 8e9, near)")
    ap.add_argument("--count", type=int, default=10)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--plain", action="store_true", help="single-lane walk instead of giant steps")
    ap.add_argument("--nucomp", action="store_true", help="NUCOMP/NUDUPL giant-step composition")
    ap.add_argument("--device", type=int, default=0)
    args = ap.parse_args(argv)
    import numpy as np
    import paper_2507_06579_gb300 as E

    ds = [int(x) for x in args.d]
    if args.near is not None:
        top = int(args.near) // 8
        rng = np.random.default_rng(args.seed)
        lo = max(1, top - 10**9)
        ds += [int(x) * 8 + 5 for x in rng.integers(lo, top, size=args.count)]
    if not ds:
        ap.error("give d values or --near")
    E.build()
    with E.Context(args.device) as ctx:
        if args.plain:
            ctx.set_option(E.EIS_OPT_MODE, E.EIS_MODE_PLAIN)
        if args.nucomp:
            ctx.set_option(E.EIS_OPT_GIANT_COMPOSE, E.EIS_COMPOSE_NUCOMP)
        for d in ds:
            t0 = time.perf_counter()
            try:
                in_e = ctx.is_eisenstein(d)
                in_d = True
            except E.EisError as e:
                if e.code != E.EIS_ENOTD:
                    raise
                in_d, in_e = False, False
            ms = (time.perf_counter() - t0) * 1e3
            st = ctx.stats()
            print(json.dumps({"d": d, "in_D": in_d, "in_E": bool(in_e),
                              "baby_steps": st["baby_steps"], "giant_steps": st["giant_steps"],
                              "ms": round(ms, 4)}), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
