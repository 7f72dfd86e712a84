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


# ---------------------------------------------------------------------------------------
# GMRES-based iterative refinement (Carson and Higham, cited in Sec. 1-2 for refinement
# with low-precision factorizations).  Reading used here: the outer loop is the one above,
# r = b - A x in float64; each correction d solves A d = r by GMRES preconditioned on the
# left with M = L_hat L_hat^T, i.e. GMRES on M^{-1} A d = M^{-1} r from d_0 = 0, applying
# M^{-1} with the two triangular solves in float64, classical Gram-Schmidt applied twice,
# Givens rotations for the small least-squares problem, stopped when the preconditioned
# residual estimate falls to inner_tol times its initial value or after `restart` steps.
# ---------------------------------------------------------------------------------------
def gmres(apply_A, apply_Minv, r: np.ndarray, restart: int, inner_tol: float):
    """(d, steps): left-preconditioned GMRES for A d = r from d = 0."""
    z = apply_Minv(r)
    beta = float(np.linalg.norm(z))
    n = r.shape[0]
    if beta == 0.0:
        return np.zeros(n), 0
    V = np.zeros((n, restart + 1))
    H = np.zeros((restart + 1, restart))
    V[:, 0] = z / beta
    cs, sn = np.zeros(restart), np.zeros(restart)
    g = np.zeros(restart + 1)
    g[0] = beta
    k = 0
    while k < restart:
        w = apply_Minv(apply_A(V[:, k]))
        for _ in range(2):                          # classical Gram-Schmidt, twice
            h = V[:, :k + 1].T @ w
            w = w - V[:, :k + 1] @ h
            H[:k + 1, k] += h
        H[k + 1, k] = float(np.linalg.norm(w))
        for i in range(k):                          # previous rotations on the new column
            a, b = H[i, k], H[i + 1, k]
            H[i, k], H[i + 1, k] = cs[i] * a + sn[i] * b, -sn[i] * a + cs[i] * b
        a, b = H[k, k], H[k + 1, k]
        rho = float(np.hypot(a, b))
        cs[k], sn[k] = (a / rho, b / rho) if rho > 0 else (1.0, 0.0)
        H[k, k], H[k + 1, k] = rho, 0.0
        g[k + 1] = -sn[k] * g[k]
        g[k] = cs[k] * g[k]
        hn = float(np.linalg.norm(w))
        if hn > 0:
            V[:, k + 1] = w / hn
        k += 1
        if abs(g[k]) <= inner_tol * beta or hn == 0.0:
            break
    y = np.zeros(k)
    for i in range(k - 1, -1, -1):                  # back substitution with the rotated H
        y[i] = (g[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]
    return V[:, :k] @ y, k


def posv_gmres_ir(A: np.ndarray, L: np.ndarray, B: np.ndarray, tol: float = 1e-12, max_iter: int = 30,
                  restart: int = 20, inner_tol: float = 1e-6):
    """(X, outer corrections, total GMRES steps, final max column residual, converged)."""
    As = dense.sym_from_lower(A)
    B2 = np.asarray(B, dtype=np.float64).reshape(As.shape[0], -1)
    X = dense.potrs(L, B2)
    it, steps = 0, 0
    while True:
        R = B2 - As @ X
        res = float(np.max(np.linalg.norm(R, axis=0) / np.linalg.norm(B2, axis=0)))
        if res <= tol:
            return X, it, steps, res, True
        if it >= max_iter:
            return X, it, steps, res, False
        for c in range(B2.shape[1]):
            d, k = gmres(lambda v: As @ v, lambda v: dense.potrs(L, v), R[:, c], restart, inner_tol)
            X[:, c] += d
            steps += k
        it += 1
