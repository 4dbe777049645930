"""Run one of the seeded workloads for a number of advection steps.

  python -m paper_2503_16082_gb300.run_case --workload oscillating_3d --adv 2 [--precision 32]

Prints one JSON line with the case totals (advection steps, acoustic substeps,
time reached, status) and the wall time.  Useful for profiling a fixed,
short piece of work.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import sphcases  # noqa: E402

import paper_2503_16082_gb300 as S  # noqa: E402

WORKLOADS = {
    "laplace_2d": sphcases.laplace_2d,
    "oscillating_3d": sphcases.oscillating_3d,
    "impact_3d": sphcases.impact_3d,
}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="oscillating_3d", choices=sorted(WORKLOADS))
    ap.add_argument("--adv", type=int, default=1)
    ap.add_argument("--precision", type=int, default=32, choices=[32, 64])
    ap.add_argument("--dx", type=float, default=None, help="override the particle spacing")
    ap.add_argument("--loop", default="graph", choices=["graph", "host"],
                    help="host: launch every kernel on its own (profilers cannot see "
                         "kernels inside a graph with a conditional node)")
    ap.add_argument("--nbr", default="list", choices=["list", "cells"])
    ap.add_argument("--block", type=int, default=0, help="threads per block (0: library default)")
    args = ap.parse_args(argv)
    spec = WORKLOADS[args.workload]() if args.dx is None else WORKLOADS[args.workload](dx=args.dx)
    h = S.case_from_spec(spec, precision=args.precision,
                         loop_mode=S.LOOP_HOST if args.loop == "host" else S.LOOP_GRAPH,
                         nbr_mode=S.NBR_CELLS if args.nbr == "cells" else S.NBR_LIST,
                         **({"block": args.block} if args.block else {}))
    t0 = time.perf_counter()
    info = S.step(h, args.adv, check=False)
    wall = time.perf_counter() - t0
    S.destroy(h)
    info.update(workload=args.workload, particles=spec.n, fluid=spec.n_fluid, wall_s=round(wall, 3))
    print(json.dumps(info))
    return 0 if info["rc"] == 0 else 1


if __name__ == "__main__":
    sys.exit(main())
