"""Oracle for the learned precision policy: matrix features, Lanczos, and the MLP.

Not in the paper (an extension of it): a small network predicts the precision tree
from cheap matrix features.  Definitions written here in float64 numpy:

* Features of a symmetric A (lower triangle read as symmetric), in this order:
   0 log2(n)
   1 min(min_i r_i, 1e6), r_i = a_ii / sum_{j != i} |a_ij|  (diagonal dominance ratio)
   2 mean_i min(r_i, 1e6)
   3 fraction of rows with r_i > 1
   4 log10 ||A||_F
   5 log10 max|a_ii| ... (diag max)
   6 log10 of diag min (clamped at 1e-300)
   7 log10(diag max / diag min)
   8 log10 lambda_max (largest Ritz value of k-step Lanczos)
   9 log10 lambda_min (smallest Ritz value, clamped at 1e-300)
  10 log10 cond estimate = feature 8 - feature 9
  11 log10(n * lambda_min / ||A||_F)    (how far the spectrum's bottom is from the bulk)
* Lanczos: start vector v_i = (1 + (i mod 7) / 7), normalized; k steps of the plain
  three-term recurrence (no reorthogonalization) w = A v_j - alpha_j v_j - beta_j v_{j-1},
  alpha_j = v_j . A v_j, beta_{j+1} = ||w||; Ritz values are the eigenvalues of the k x k
  tridiagonal T (numpy's symmetric eigensolver, a library primitive).
* MLP 12 -> 64 -> 64 -> 8 with ReLU, logits z; parameters packed as
  W1 (64x12, row-major), b1 (64), W2 (64x64), b2 (64), W3 (8x64), b3 (8) = 5512 floats.
  Loss: mean softmax cross-entropy; gradients by the chain rule (pinned by finite
  differences in tests/test_oracle_policy.py).
"""
from __future__ import annotations

import numpy as np

from . import dense

SIZES = [(64, 12), (64,), (64, 64), (64,), (8, 64), (8,)]
NPARAM = sum(int(np.prod(s)) for s in SIZES)      # 5512


def unpack(p: np.ndarray):
    out, o = [], 0
    for s in SIZES:
        k = int(np.prod(s))
        out.append(np.asarray(p[o:o + k], dtype=np.float64).reshape(s))
        o += k
    return out


def pack(parts) -> np.ndarray:
    return np.concatenate([np.asarray(x, dtype=np.float64).ravel() for x in parts])


def lanczos_start(n: int) -> np.ndarray:
    v = 1.0 + (np.arange(n) % 7) / 7.0
    return v / np.linalg.norm(v)


def lanczos(A: np.ndarray, k: int):
    """(alpha, beta) of k Lanczos steps on the symmetric A from lanczos_start(n)."""
    As = dense.sym_from_lower(A)
    n = As.shape[0]
    k = min(k, n)
    v_prev = np.zeros(n)
    v = lanczos_start(n)
    alpha, beta = [], []
    b = 0.0
    for j in range(k):
        w = As @ v
        a = float(w @ v)
        w = w - a * v - b * v_prev
        alpha.append(a)
        b = float(np.linalg.norm(w))
        if j + 1 < k:
            beta.append(b)
            if b == 0.0:
                break
            v_prev, v = v, w / b
    return np.array(alpha), np.array(beta[:len(alpha) - 1])


def ritz_extremes(alpha: np.ndarray, beta: np.ndarray):
    T = np.diag(alpha) + np.diag(beta, 1) + np.diag(beta, -1)
    ev = np.linalg.eigvalsh(T)
    return float(ev[0]), float(ev[-1])


def features(A: np.ndarray, k: int = 24) -> np.ndarray:
    As = dense.sym_from_lower(A)
    n = As.shape[0]
    d = np.diag(As).copy()
    off = np.abs(As).sum(axis=1) - np.abs(d)
    with np.errstate(divide="ignore"):
        r = np.where(off > 0, d / np.where(off > 0, off, 1.0), 1e30)
    fro = float(np.linalg.norm(As))
    dmin, dmax = float(d.min()), float(np.abs(d).max())
    lmin, lmax = ritz_extremes(*lanczos(A, k))
    f = np.zeros(12)
    f[0] = np.log2(n)
    f[1] = min(float(r.min()), 1e6)
    f[2] = float(np.minimum(r, 1e6).mean())
    f[3] = float((r > 1.0).mean())
    f[4] = np.log10(fro)
    f[5] = np.log10(max(dmax, 1e-300))
    f[6] = np.log10(max(dmin, 1e-300))
    f[7] = f[5] - f[6]
    f[8] = np.log10(max(lmax, 1e-300))
    f[9] = np.log10(max(lmin, 1e-300))
    f[10] = f[8] - f[9]
    f[11] = np.log10(max(n * max(lmin, 1e-300) / fro, 1e-300))
    return f


def forward(p: np.ndarray, X: np.ndarray):
    W1, b1, W2, b2, W3, b3 = unpack(p)
    h1 = np.maximum(X @ W1.T + b1, 0.0)
    h2 = np.maximum(h1 @ W2.T + b2, 0.0)
    z = h2 @ W3.T + b3
    return z, (h1, h2)


def loss_and_grad(p: np.ndarray, X: np.ndarray, y: np.ndarray):
    """Mean softmax cross-entropy and its gradient with respect to the packed parameters."""
    W1, b1, W2, b2, W3, b3 = unpack(p)
    B = X.shape[0]
    z, (h1, h2) = forward(p, X)
    zs = z - z.max(axis=1, keepdims=True)
    pz = np.exp(zs)
    pz /= pz.sum(axis=1, keepdims=True)
    loss = float(-np.log(pz[np.arange(B), y]).mean())
    dz = pz.copy()
    dz[np.arange(B), y] -= 1.0
    dz /= B
    gW3 = dz.T @ h2
    gb3 = dz.sum(axis=0)
    dh2 = (dz @ W3) * (h2 > 0)
    gW2 = dh2.T @ h1
    gb2 = dh2.sum(axis=0)
    dh1 = (dh2 @ W2) * (h1 > 0)
    gW1 = dh1.T @ X
    gb1 = dh1.sum(axis=0)
    return loss, pack([gW1, gb1, gW2, gb2, gW3, gb3])
