"""Run the cut-off autotuner (hrp_autotune) and report every candidate's median time.

    python -m paper_2601_08082_gb300.autotune --n 8192 --tree "[F16,F16,F16,F16,F32|F64@128]"

Prints one JSON line: the tuner's choice (leaf, trsm_leaf, median ms on its own seeded
matrix) and, for each candidate, the median of --reps factorizations of that same kind of
matrix timed here with CUDA events (the figures the choice can be checked against).
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=8192)
    ap.add_argument("--tree", default="[F16,F16,F16,F16,F32|F64@128]")
    ap.add_argument("--leaf", type=int, default=128)
    ap.add_argument("--reps", type=int, default=3)
    args = ap.parse_args()

    import numpy as np
    import torch

    from . import hrp

    h = hrp.Handle(0)
    t = hrp.tree_parse(args.tree, leaf=args.leaf)
    best, ms = h.autotune(t, args.n, reps=args.reps, retune=True)
    # the same seeded matrix family the tuner uses: uniform off-diagonal entries, n on the diagonal
    g = torch.Generator(device="cuda")
    g.manual_seed(2601008082 + args.n)
    B = torch.rand((args.n, args.n), generator=g, device="cuda", dtype=torch.float64) * 2.0 - 1.0
    A0 = torch.tril(B) + torch.tril(B, -1).T
    A0.diagonal().fill_(float(args.n))
    rows = []
    for c in hrp.autotune_candidates(t):
        ts = []
        info = 0
        for r in range(args.reps + 1):
            A = A0.clone()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            info = h.potrf(c, A)
            e1.record()
            torch.cuda.synchronize()
            if r:
                ts.append(e0.elapsed_time(e1))
        rows.append({"leaf": c.leaf, "trsm_leaf": c.trsm_leaf or c.leaf, "info": info,
                     "ms": float(np.median(ts)), "backward_error": h.backward_error(A0, A)})
    print(json.dumps({"n": args.n, "tree": hrp.tree_format(t),
                      "choice": {"leaf": best.leaf, "trsm_leaf": best.trsm_leaf or best.leaf, "ms": ms},
                      "candidates": rows}))
    h.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
