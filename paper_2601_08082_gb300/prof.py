"""Run a few factorizations (and optionally solves) of one workload, for profilers.

Example (launch list of two factorizations of the n = 8192 mixed workload):
    ncu --metrics gpu__time_duration.sum --clock-control none --csv \
        python -m paper_2601_08082_gb300.prof --n 8192 --reps 2
"""
from __future__ import annotations

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def print_timeline(tl) -> None:
    """Leaves on the critical stream (stream 0) and, grouped by their sequence of kernel
    classes, the launches between consecutive leaves."""
    import numpy as np

    names = ["leaf", "ltrsm", "tc", "simt", "other"]
    crit = tl[tl[:, 1] == 0]
    leaf = crit[crit[:, 0] == 0]
    print(f"launches {len(tl)} (critical stream {len(crit)}), span {tl[:, 3].max():.3f} ms")
    print(f"leaves: {len(leaf)}, {np.sum(leaf[:, 3] - leaf[:, 2]):.3f} ms, "
          f"{np.mean(leaf[:, 3] - leaf[:, 2]) * 1e3:.1f} us each")
    starts, ends = leaf[:, 2], leaf[:, 3]
    gaps = starts[1:] - ends[:-1]
    print(f"between consecutive leaves: {gaps.sum():.3f} ms in {len(gaps)} gaps")
    groups = {}
    for k in range(len(gaps)):
        sel = crit[(crit[:, 2] >= ends[k]) & (crit[:, 3] <= starts[k + 1])]
        key = " ".join(names[int(c)] for c in sel[:, 0])
        g = groups.setdefault(key, [0, 0.0, 0.0])
        g[0] += 1
        g[1] += gaps[k] * 1e3
        g[2] += float(np.sum(sel[:, 3] - sel[:, 2])) * 1e3
    for key, (cnt, gap_us, in_us) in sorted(groups.items(), key=lambda x: len(x[0])):
        nk = len(key.split()) if key else 0
        print(f"  {cnt:3d} gaps of {nk:2d} kernels: mean gap {gap_us / cnt:7.1f} us, in kernels {in_us / cnt:7.1f} us")
    for c in range(5):
        sel = crit[crit[:, 0] == c]
        if len(sel):
            print(f"  critical {names[c]}: {len(sel)} launches, {np.mean(sel[:, 3] - sel[:, 2]) * 1e3:.1f} us each")


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=8192)
    ap.add_argument("--rho", type=float, default=2.0)
    ap.add_argument("--tree", default="[F16,F16,F16,F16,F32|F64@128]")
    ap.add_argument("--leaf", type=int, default=128)
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--nrhs", type=int, default=0, help="also solve with this many right-hand sides")
    ap.add_argument("--device-gen", action="store_true",
                    help="draw the matrix on the device (seeded torch generator) instead of the host generator")
    ap.add_argument("--timing", action="store_true",
                    help="print per-kernel-class device time of the last factorization (event timing mode)")
    ap.add_argument("--timeline", action="store_true",
                    help="print the critical stream's leaves and the launches between them (event timing mode)")
    ap.add_argument("--no-lookahead", action="store_true", help="one stream: hrp_set_lookahead(h, 0)")
    ap.add_argument("--f8-fp16", action="store_true",
                    help="F8 levels on the kind::f16 GEMM with E4M3 values in FP16 storage (hrp_set_f8_gemm(h, 1))")
    args = ap.parse_args()

    import torch

    from synth import dominant_spd, rhs, seed_for
    from . import hrp

    h = hrp.Handle(0)
    if args.no_lookahead:
        h.set_lookahead(False)
    if args.f8_fp16:
        h.set_f8_gemm(True)
    if args.device_gen:
        g = torch.Generator(device="cuda")
        g.manual_seed(seed_for(1, 0))
        Bt = torch.randn((args.n, args.n), generator=g, device="cuda", dtype=torch.float64)
        A0 = Bt + Bt.T
        del Bt
        A0.mul_(0.5)
        A0.diagonal().zero_()
        A0.diagonal().copy_(args.rho * A0.abs().sum(dim=1))
    else:
        A0 = hrp.colmajor(dominant_spd(args.n, args.rho, seed_for(1, 0))).cuda()
    B0 = hrp.colmajor(rhs(args.n, args.nrhs, seed_for(1, 1))).cuda() if args.nrhs else None
    tree = hrp.tree_parse(args.tree, leaf=args.leaf)
    for _ in range(args.reps):
        A = A0.clone()
        info = h.potrf(tree, A)
        if info:
            print(f"info = {info}")
            return 1
        if B0 is not None:
            B = B0.clone()
            h.potrs(A, B)
    torch.cuda.synchronize()
    if args.timing:
        import json
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        A = A0.clone()
        torch.cuda.synchronize()
        e0.record()
        h.potrf(tree, A)
        e1.record()
        torch.cuda.synchronize()
        classes = h.timing(tree, A0.clone())
        print(json.dumps({"n": args.n, "tree": args.tree, "leaf": args.leaf, "ms": e0.elapsed_time(e1),
                          "classes": classes}))
    if args.timeline:
        h.timing(tree, A0.clone())
        print_timeline(h.timeline())
    print(f"{args.reps} factorizations of n={args.n} tree {args.tree}: {h.launch_count()} launches each")
    h.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
