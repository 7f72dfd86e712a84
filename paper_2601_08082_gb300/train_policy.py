"""Train the precision-tree policy on factorizations the method itself runs.

Data: matrices A = G G^T / k + alpha I (G n x k N(0,1), k = n/2, alpha log-uniform in
[1e-3, 10]) mixed 50/50 with diagonally dominant ones (rho uniform in [0.5, 8]; rho < 1
need not be SPD and such failures are part of the data), n in {1024, 2048, 4096, 8192}
with probabilities .25/.35/.25/.15 (the F8 trees need n = 128 * 2^k), drawn on the
device with a seeded torch generator.  For every matrix: the 12 features (hrp_policy_features) and, for
each of the 8 candidate trees (hrp_policy_tree), the device time of hrp_posv (factor,
solve, FP64 refinement to 1e-12 with one right-hand side; a tree whose factorization
fails is refactored with the fallback tree inside hrp_posv, so its time counts that
too).  Label = the fastest tree whose solve converged; matrices no tree solves are dropped.

Training: 80/10/10 split, inputs standardized with the training split's mean and scale,
full-batch Adam on the GPU with the library's own kernels (hrp_mlp_grad, hrp_mlp_adam).
The validation split picks the step with the best validation loss, and the order gate: the
smallest order from which, at every order of the grid, the feature pass plus the picked
tree's solve beat the fallback tree's solve on average ("min_n"; smaller systems take the
fallback without the feature pass).  The test split is reported with the gate applied.
Output: JSON with the parameters, the standardization, the gate and the split metrics.

    python -m paper_2601_08082_gb300.train_policy --samples 800 --out policy_weights.json
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

NTREES = 8


def make_matrix(i: int, seed0: int, torch):
    """Training matrix i, drawn on the device (torch generator seeded by seed0 and i)."""
    import numpy as np

    from synth import uniforms
    u = uniforms(seed0, 11, np.arange(4 * i, 4 * i + 4, dtype=np.uint64))
    n = [1024, 2048, 4096, 8192][int(np.searchsorted([0.25, 0.6, 0.85, 1.01], u[0], side="right"))]
    g = torch.Generator(device="cuda")
    g.manual_seed(int(seed0) * 100003 + i)
    if u[1] < 0.5:
        alpha = float(10.0 ** (-3.0 + 4.0 * u[2]))
        k = n // 2
        G = torch.randn((n, k), generator=g, device="cuda", dtype=torch.float64)
        A = G @ G.T / k
        A = 0.5 * (A + A.T)
        A.diagonal().add_(alpha)
        return A, {"kind": "gram", "n": n, "alpha": alpha}
    rho = float(0.5 + 7.5 * u[2])
    B = torch.randn((n, n), generator=g, device="cuda", dtype=torch.float64)
    A = 0.5 * (B + B.T)
    A.diagonal().zero_()
    A.diagonal().copy_(rho * A.abs().sum(dim=1))
    return A, {"kind": "dominant", "n": n, "rho": rho}


def label_one(h, A, hrp, torch):
    """features, per-tree posv times (inf where the solve did not converge), and the time of
    the feature pass.  A: symmetric (n, n) float64 CUDA tensor (its own transpose, so also
    column-major)."""
    import numpy as np

    from synth import rhs, seed_for
    n = A.shape[0]
    A = A.contiguous()
    torch.cuda.synchronize()
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    f0.record()
    feat = h.policy_features(A, lanczos_steps=10)
    f1.record()
    torch.cuda.synchronize()
    t_feat = f0.elapsed_time(f1)
    B = hrp.colmajor(rhs(n, 1, seed_for(5, 7))).cuda()
    X = torch.zeros_like(B)
    times = np.full(NTREES, np.inf)
    for t in range(NTREES):
        tree = hrp.policy_tree(t)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        out = h.posv(tree, A, B, X, max_iter=30, tol=1e-12)
        e1.record()
        torch.cuda.synchronize()
        if out["status"] == 0:
            times[t] = e0.elapsed_time(e1)
    return feat, times, t_feat


def order_gate(ns, t_feat, t_pick, t_fb):
    """Smallest order from which the policy (feature pass + the picked tree) beats the fixed
    fallback on average at every order of the grid, from matrices not used for training
    (numpy arrays over the same matrices); 2^30 when it never does."""
    import numpy as np
    grid = sorted(set(int(n) for n in ns))
    wins = {}
    for n in grid:
        sel = ns == n
        wins[n] = bool(np.mean(t_feat[sel] + t_pick[sel]) < np.mean(t_fb[sel]))
    gate = 1 << 30
    for n in reversed(grid):
        if not wins[n]:
            break
        gate = n
    return gate, wins


def train(h, hrp, torch, Xtr, ytr, Xva, yva, steps: int, lr: float, seed: int):
    import numpy as np
    npar = hrp.mlp_param_count()
    rng = np.random.default_rng(seed)
    # He-style initialization
    p = np.zeros(npar, dtype=np.float32)
    o = 0
    for shape in [(64, 12), (64,), (64, 64), (64,), (8, 64), (8,)]:
        k = int(np.prod(shape))
        if len(shape) == 2:
            p[o:o + k] = rng.standard_normal(k) * np.sqrt(2.0 / shape[1])
        o += k
    P = torch.tensor(p, device="cuda")
    G = torch.zeros_like(P)
    M = torch.zeros_like(P)
    V = torch.zeros_like(P)
    loss = torch.zeros(1, device="cuda")
    Xt = torch.tensor(Xtr, dtype=torch.float32, device="cuda")
    yt = torch.tensor(ytr, dtype=torch.int32, device="cuda")
    Xv = torch.tensor(Xva, dtype=torch.float32, device="cuda")
    yv = torch.tensor(yva, dtype=torch.int32, device="cuda")
    Gv = torch.zeros_like(P)
    lv = torch.zeros(1, device="cuda")
    best = (np.inf, None, 0)
    hist = []
    for step in range(1, steps + 1):
        h.mlp_grad(P, Xt, yt, G, loss)
        h.mlp_adam(P, G, M, V, step, lr)
        if step % 50 == 0 or step == steps:
            h.mlp_grad(P, Xv, yv, Gv, lv)
            vl = float(lv.item())
            hist.append((step, float(loss.item()), vl))
            if vl < best[0]:
                best = (vl, P.clone(), step)
    return best, hist


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--samples", type=int, default=800)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--seed", type=int, default=2601)
    ap.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)), "policy_weights.json"))
    ap.add_argument("--data-out", default="")
    args = ap.parse_args()

    import numpy as np
    import torch

    from . import hrp

    h = hrp.Handle(0)
    t0 = time.time()
    feats, times, meta, tfeat = [], [], [], []
    for i in range(args.samples):
        A, m = make_matrix(i, args.seed, torch)
        f, t, tf = label_one(h, A, hrp, torch)
        del A
        feats.append(f)
        times.append(t)
        meta.append(m)
        tfeat.append(tf)
    feats = np.array(feats, dtype=np.float64)
    times = np.array(times)
    tfeat = np.array(tfeat)
    orders = np.array([m["n"] for m in meta])
    ok = np.isfinite(times).any(axis=1)
    labels = np.where(ok, np.argmin(times, axis=1), -1)
    idx = np.nonzero(ok)[0]
    n_tr, n_va = int(0.8 * len(idx)), int(0.1 * len(idx))
    tr, va, te = idx[:n_tr], idx[n_tr:n_tr + n_va], idx[n_tr + n_va:]
    mean = feats[tr].mean(axis=0)
    scale = feats[tr].std(axis=0)
    scale[scale < 1e-6] = 1.0
    norm = lambda F: (F - mean) / scale
    best, hist = train(h, hrp, torch, norm(feats[tr]), labels[tr], norm(feats[va]), labels[va], args.steps,
                       args.lr, args.seed)
    params = best[1].cpu().numpy()

    # the order gate from the validation split, then held-out evaluation with the GPU forward pass
    h.policy_set(params, mean, scale)
    pred_va = np.array([h.policy_predict(feats[i]) for i in va])
    tp_va = np.where(np.isfinite(times[va, pred_va]), times[va, pred_va], 1e9)
    tf_va = np.where(np.isfinite(times[va, 0]), times[va, 0], 1e9)
    gate, wins = order_gate(orders[va], tfeat[va], tp_va, tf_va)
    pred = np.array([h.policy_predict(feats[i]) if orders[i] >= gate else 0 for i in te])
    t_pred = times[te, pred]
    t_fb = times[te, 0]
    t_total = np.where(orders[te] >= gate, tfeat[te] + t_pred, t_pred)
    result = {
        "format": "hrp-policy-v1",
        "trees": [hrp.tree_format(hrp.policy_tree(t)) for t in range(NTREES)],
        "params": [float(x) for x in params],
        "mean": [float(x) for x in mean],
        "scale": [float(x) for x in scale],
        "min_n": [int(gate)],
        "gate": {"validation_wins_by_order": {str(k): v for k, v in wins.items()},
                 "mean_feature_ms_by_order": {str(n): float(np.mean(tfeat[orders == n])) for n in sorted(set(orders))}},
        "train": {"samples": int(len(tr)), "best_step": int(best[2]), "val_loss": float(best[0]),
                  "history": hist[-10:], "label_counts": np.bincount(labels[tr], minlength=NTREES).tolist()},
        "test": {"samples": int(len(te)), "accuracy": float((pred == labels[te]).mean()),
                 "mean_ms_policy": float(np.mean(np.where(np.isfinite(t_pred), t_pred, np.nan))),
                 "mean_ms_policy_with_features": float(np.mean(np.where(np.isfinite(t_total), t_total, np.nan))),
                 "mean_ms_fallback": float(np.mean(np.where(np.isfinite(t_fb), t_fb, np.nan))),
                 "policy_failures": int((~np.isfinite(t_pred)).sum()),
                 "fallback_failures": int((~np.isfinite(t_fb)).sum()),
                 "mean_ms_oracle_best": float(np.mean(times[te].min(axis=1)))},
        "data": {"samples": args.samples, "unsolvable": int((~ok).sum()), "seed": args.seed,
                 "seconds": time.time() - t0},
    }
    with open(args.out, "w") as f:
        json.dump(result, f)
    if args.data_out:
        np.savez(args.data_out, feats=feats, times=times, labels=labels)
    print(json.dumps({k: v for k, v in result.items() if k not in ("params", "mean", "scale")}))
    h.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
