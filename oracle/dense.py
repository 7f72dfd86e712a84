"""Plain dense Cholesky factorization, triangular solves and error measures.

These are the definitions the FP64 path reaches exactly up to rounding order
(Alg. 1-3 only reorder the same arithmetic, Sec. 3.2):

  * Cholesky: the unique lower-triangular L with positive diagonal and A = L L^T,
    computed column by column (l_jj = sqrt(a_jj - sum_k l_jk^2),
    l_ij = (a_ij - sum_k l_ik l_jk) / l_jj).  A non-positive or non-finite pivot
    stops the factorization; info is its 1-based column, as LAPACK POTRF reports.
  * TRSM_{R,L,T}: X = B L^{-T}, column by column (the operation of Alg. 2).
  * POTRS: L y = b (forward), then L^T x = y (backward); the "linear solve" of the
    paper's title and abstract.
  * Errors: ||A - L L^T||_F / ||A||_F (Sec. 4.2, Cholesky accuracy), forward error
    of L, relative residuals.
"""
from __future__ import annotations

import numpy as np


def cholesky(A: np.ndarray, dtype=np.float64) -> tuple[np.ndarray, int]:
    """Lower Cholesky factor of the lower triangle of A, computed in ``dtype``.

    Returns (L, info): info = 0 on success, else the 1-based column of the first
    pivot that is not positive and finite (L then holds the columns before it).
    """
    A = np.asarray(A)
    n = A.shape[0]
    Ad = np.tril(A).astype(dtype)
    L = np.zeros((n, n), dtype=dtype)
    for j in range(n):
        d = Ad[j, j] - np.dot(L[j, :j], L[j, :j])
        if not (np.isfinite(d) and d > 0):
            return L.astype(np.float64), j + 1
        ljj = np.sqrt(d)
        L[j, j] = ljj
        if j + 1 < n:
            L[j + 1:, j] = (Ad[j + 1:, j] - L[j + 1:, :j] @ L[j, :j]) / ljj
    return L.astype(np.float64), 0


def trsm_rlt(B: np.ndarray, L: np.ndarray, dtype=np.float64) -> np.ndarray:
    """X = B L^{-T} for lower-triangular L, by column substitution in ``dtype``.

    Each row is an independent substitution x_j = (b_j - sum_{k<j} x_k l_jk) / l_jj; the
    sum of a row is reduced along that row alone, so a row's result does not depend on
    which other rows are solved in the same call (a matrix-vector product would let the
    library's blocking, and with it the rounding order, vary with the number of rows).
    """
    B = np.asarray(B).astype(dtype)
    L = np.tril(np.asarray(L)).astype(dtype)
    m, n = B.shape
    X = np.zeros((m, n), dtype=dtype)
    for j in range(n):
        s = np.sum(X[:, :j] * L[j, :j], axis=1, dtype=dtype) if j else np.zeros(m, dtype=dtype)
        X[:, j] = (B[:, j] - s) / L[j, j]
    return X.astype(np.float64)


def forward_solve(L: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Y with L Y = B (L lower triangular), row by row in float64."""
    L = np.asarray(L, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    vec = B.ndim == 1
    Bm = B[:, None] if vec else B
    n = L.shape[0]
    Y = np.zeros_like(Bm)
    for i in range(n):
        Y[i] = (Bm[i] - L[i, :i] @ Y[:i]) / L[i, i]
    return Y[:, 0] if vec else Y


def backward_solve_t(L: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """X with L^T X = Y (L lower triangular), from the last row up, in float64."""
    L = np.asarray(L, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    vec = Y.ndim == 1
    Ym = Y[:, None] if vec else Y
    n = L.shape[0]
    X = np.zeros_like(Ym)
    for i in range(n - 1, -1, -1):
        X[i] = (Ym[i] - L[i + 1:, i] @ X[i + 1:]) / L[i, i]
    return X[:, 0] if vec else X


def potrs(L: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Solve A X = B given A = L L^T."""
    return backward_solve_t(L, forward_solve(L, B))


def sym_from_lower(A: np.ndarray) -> np.ndarray:
    """Full symmetric matrix from the lower triangle of A."""
    Lw = np.tril(A)
    return Lw + np.tril(Lw, -1).T


def backward_error(A: np.ndarray, L: np.ndarray) -> float:
    """||A - L L^T||_F / ||A||_F with A taken from its lower triangle (symmetric)."""
    As = sym_from_lower(np.asarray(A, dtype=np.float64))
    Lt = np.tril(np.asarray(L, dtype=np.float64))
    return float(np.linalg.norm(As - Lt @ Lt.T) / np.linalg.norm(As))


def scaled_backward_error(A: np.ndarray, L: np.ndarray) -> float:
    """Backward error of the diagonally scaled problem: ||S (A - L L^T) S||_F / ||S A S||_F with
    S = diag(a_ii^-1/2), the measure that sees every row whatever its scale."""
    As = sym_from_lower(np.asarray(A, dtype=np.float64))
    s = 1.0 / np.sqrt(np.diag(As))
    Lt = np.tril(np.asarray(L, dtype=np.float64)) * s[:, None]
    Ss = As * s[:, None] * s[None, :]
    return float(np.linalg.norm(Ss - Lt @ Lt.T) / np.linalg.norm(Ss))


def factor_error(L_hat: np.ndarray, L: np.ndarray) -> float:
    """||L_hat - L||_F / ||L||_F over the lower triangles."""
    return float(np.linalg.norm(np.tril(L_hat) - np.tril(L)) / np.linalg.norm(np.tril(L)))


def column_residuals(A: np.ndarray, X: np.ndarray, B: np.ndarray) -> np.ndarray:
    """||b_j - A x_j||_2 / ||b_j||_2 per column (A symmetric from its lower triangle)."""
    As = sym_from_lower(np.asarray(A, dtype=np.float64))
    X2 = np.asarray(X, dtype=np.float64).reshape(As.shape[0], -1)
    B2 = np.asarray(B, dtype=np.float64).reshape(As.shape[0], -1)
    R = B2 - As @ X2
    return np.linalg.norm(R, axis=0) / np.linalg.norm(B2, axis=0)


def normwise_backward_error(A: np.ndarray, X: np.ndarray, B: np.ndarray) -> float:
    """max_j ||r_j||_inf / (||A||_inf ||x_j||_inf + ||b_j||_inf)."""
    As = sym_from_lower(np.asarray(A, dtype=np.float64))
    X2 = np.asarray(X, dtype=np.float64).reshape(As.shape[0], -1)
    B2 = np.asarray(B, dtype=np.float64).reshape(As.shape[0], -1)
    R = B2 - As @ X2
    anorm = np.max(np.abs(As).sum(axis=1))
    num = np.max(np.abs(R), axis=0)
    den = anorm * np.max(np.abs(X2), axis=0) + np.max(np.abs(B2), axis=0)
    return float(np.max(num / den))
