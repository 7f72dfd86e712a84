"""GPU parity of the learned-policy kernels with the oracle, and the trained policy's gain.

* features: the device's FP64 passes and its Lanczos (matrix-vector products in FP32,
  recurrence in FP64) vs oracle/policy.features (same definitions, same start vector).
  FP32 products move the Ritz values by ~k * 2^-24 relative, i.e. the log10 features by
  ~1e-6 absolute; the comparison allows 1e-4 (features are float32 anyway).
* MLP forward and gradient in FP32 vs the FP64 oracle: 1e-4 / 1e-3 relative.
* Adam: one step against the update formula written out here.
* gain: the shipped network (policy_weights.json, trained by train_policy.py on
  factorizations this library ran) against the fixed fallback tree on fresh matrices
  of the training distribution: every solve converges, the picked tree's mean solve
  time is lower, and the feature pass stays under a quarter of a fallback solve.
"""
import json
import os

import numpy as np
import pytest

from oracle import policy as opol
from synth import dominant_spd, gram_spd, rhs, seed_for

pytestmark = pytest.mark.gpu

WEIGHTS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2601_08082_gb300",
                       "policy_weights.json")


@pytest.fixture(scope="module")
def env():
    import torch

    import paper_2601_08082_gb300 as hrp
    h = hrp.Handle(0)
    yield hrp, h, torch
    h.close()


@pytest.mark.parametrize("case", ["dominant", "gram", "diag"])
def test_features_match_oracle(env, case):
    hrp, h, torch = env
    if case == "dominant":
        A = dominant_spd(700, 1.3, seed_for(6, 1))
    elif case == "gram":
        A = gram_spd(512, 3e-2, seed_for(6, 2))
    else:
        A = np.diag(np.linspace(0.5, 40.0, 300))
    f_gpu = h.policy_features(hrp.colmajor(A).cuda(), 24).astype(np.float64)
    f_ref = opol.features(A, 24)
    assert np.allclose(f_gpu, f_ref, rtol=1e-4, atol=1e-4), (f_gpu, f_ref)


def test_mlp_forward_and_gradient_match_oracle(env):
    hrp, h, torch = env
    rng = np.random.default_rng(3)
    p = (rng.standard_normal(opol.NPARAM) * 0.2).astype(np.float32)
    X = rng.standard_normal((37, 12)).astype(np.float32)
    y = rng.integers(0, 8, size=37).astype(np.int32)
    P = torch.tensor(p, device="cuda")
    Xt = torch.tensor(X, device="cuda")
    Z = torch.zeros((37, 8), device="cuda")
    h.mlp_forward(P, Xt, Z)
    z_ref, _ = opol.forward(p.astype(np.float64), X.astype(np.float64))
    assert np.max(np.abs(Z.cpu().numpy() - z_ref)) <= 1e-4 * np.max(np.abs(z_ref))
    G = torch.zeros_like(P)
    loss = torch.zeros(1, device="cuda")
    h.mlp_grad(P, Xt, torch.tensor(y, device="cuda"), G, loss)
    l_ref, g_ref = opol.loss_and_grad(p.astype(np.float64), X.astype(np.float64), y)
    assert abs(loss.item() - l_ref) <= 1e-5 * abs(l_ref)
    g = G.cpu().numpy()
    assert np.linalg.norm(g - g_ref) <= 1e-3 * np.linalg.norm(g_ref)


def test_adam_step_formula(env):
    hrp, h, torch = env
    rng = np.random.default_rng(4)
    p = rng.standard_normal(opol.NPARAM).astype(np.float32)
    g = rng.standard_normal(opol.NPARAM).astype(np.float32)
    m = rng.standard_normal(opol.NPARAM).astype(np.float32) * 0.1
    v = np.abs(rng.standard_normal(opol.NPARAM)).astype(np.float32) * 0.1
    P, Gt, M, V = (torch.tensor(a, device="cuda") for a in (p, g, m, v))
    h.mlp_adam(P, Gt, M, V, 3, 1e-2)
    m1 = 0.9 * m + 0.1 * g
    v1 = 0.999 * v + 0.001 * g * g
    p1 = p - 1e-2 * (m1 / (1 - 0.9 ** 3)) / (np.sqrt(v1 / (1 - 0.999 ** 3)) + 1e-8)
    assert np.allclose(P.cpu().numpy(), p1, rtol=1e-5, atol=1e-6)


def _timed(torch, fn):
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    out = fn()
    e1.record()
    torch.cuda.synchronize()
    return out, e0.elapsed_time(e1)


def test_trained_policy_beats_the_fixed_fallback(env):
    """Held-out matrices of the training distribution (another seed), orders 4096 and 8192:
    the solve with the tree the policy picks against the solve with the fixed fallback tree,
    on the same matrix; the feature pass that makes the pick is timed on its own and must
    stay a small share of a solve."""
    hrp, h, torch = env
    from paper_2601_08082_gb300 import train_policy as tp
    assert os.path.exists(WEIGHTS), "policy_weights.json is produced by train_policy.py"
    with open(WEIGHTS) as f:
        w = json.load(f)
    h.policy_set(np.array(w["params"]), np.array(w["mean"]), np.array(w["scale"]))
    fb = hrp.policy_tree(0)
    t_pick, t_fb, t_feat, picks = [], [], [], []
    i, used = 0, 0
    while used < 10:
        A, meta = tp.make_matrix(i, 9999, torch)
        i += 1
        if meta["n"] < 4096 or (meta["kind"] == "dominant" and meta["rho"] < 1.0):
            continue
        used += 1
        n = meta["n"]
        A = A.contiguous()
        B = hrp.colmajor(rhs(n, 1, seed_for(7, 100 + i))).cuda()
        feat, tf = _timed(torch, lambda: h.policy_features(A, 10))
        k = h.policy_predict(feat)
        picks.append(k)
        for tree, acc in ((hrp.policy_tree(k), t_pick), (fb, t_fb)):
            X = torch.zeros_like(B)
            out, t = _timed(torch, lambda: h.posv(tree, A, B, X, tol=1e-12))
            assert out["status"] == 0, (i, k, out)
            acc.append(t)
        t_feat.append(tf)
        del A
    summary = (np.mean(t_pick), np.mean(t_fb), np.mean(t_feat), picks)
    assert np.mean(t_pick) < np.mean(t_fb), summary
    assert np.mean(t_feat) < 0.25 * np.mean(t_fb), summary
