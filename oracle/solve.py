"""Solve A X = B with a (possibly mixed-precision) Cholesky factor plus FP64 refinement.

The paper solves SPD systems through the Cholesky factor (title, abstract) and
cites mixed-precision iterative refinement as the standard way to recover full
accuracy from a low-precision factorization (Sec. 1-2, Higham et al., Carson and
Higham).  Reading used here:
  x_0 = POTRS(L, b); repeat r = b - A x (float64, A's lower triangle read as
  symmetric), d = POTRS(L, r), x = x + d; stop when every column's
  ||b_j - A x_j||_2 / ||b_j||_2 <= tol, or after max_iter corrections.
"""
from __future__ import annotations

import numpy as np

from . import dense


def posv_ir(A: np.ndarray, L: np.ndarray, B: np.ndarray, tol: float = 1e-12, max_iter: int = 30):
    """(X, iterations, final max column residual, converged)."""
    As = dense.sym_from_lower(A)
    B2 = np.asarray(B, dtype=np.float64).reshape(As.shape[0], -1)
    X = dense.potrs(L, B2)
    it = 0
    while True:
        R = B2 - As @ X
        res = float(np.max(np.linalg.norm(R, axis=0) / np.linalg.norm(B2, axis=0)))
        if res <= tol:
            return X, it, res, True
        if it >= max_iter:
            return X, it, res, False
        X = X + dense.potrs(L, R)
        it += 1
