"""Run K GW iterations of a named synthetic workload on the GPU and print one
JSON line per iteration (mu, N, per-stage milliseconds).

    python -m paper_2604_22223_gb300.run --workload five-orbital-16x16x8 \\
        --precision mixed --steps 2
"""
from __future__ import annotations

import argparse
import json
import os
import sys


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="five-orbital-16x16x8")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="mixed")
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--pairs", choices=["auto", "full", "reduced"], default="auto")
    args = ap.parse_args(argv)
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import workloads
    from . import build, qa
    build()
    ctx = qa.Context(workloads.config(args.workload), args.precision, pairs=args.pairs)
    G = None
    for i in range(args.steps):
        G, mu, n, st = ctx.step(G, None, timing=True)
        print(json.dumps({"step": i, "pairs": ctx.nb, "mu": mu, "N": st["N"], "mu_evals": st["mu_evals"],
                          "launches": st["launches"], "stage_ms": st["stage_ms"]}))


if __name__ == "__main__":
    main()
