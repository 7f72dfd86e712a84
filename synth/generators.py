"""Counter-based seeded generators for the synthetic SPD workloads.

Every random number is a pure function of (seed, counter): SplitMix64's output
mixer applied to ``key + (counter + 1) * GAMMA`` (Steele, Lea, Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014), turned into a
53-bit uniform and, for normals, by the Box-Muller transform.  Because a value
depends only on its counter, any block of a matrix can be drawn on its own and
the same bits come out on every machine and numpy version.

Workloads (matrix definitions):
  * ``dominant_spd``: B iid N(0,1), A = (B + B^T)/2, A_ii = rho * sum_{j!=i} |A_ij| + shift.
    rho=1, shift=1 is the plain FP64 workload (n=1024); rho in {1.05, 2, 8}, shift=0
    the mixed-tree workloads (n=8192, n=32768).
  * ``paper_spd``: symmetric uniform [0,1) entries with n added to the diagonal, the
    synthetic matrices of the paper's evaluation (Sec. 4.1).
  * ``rbf_spd``: A_ij = exp(-|x_i - x_j|^2 / (2 l^2)) + jitter * delta_ij, x_i ~ U[0,1]^3.
  * ``gram_spd``: A = G G^T / k + alpha I with G n x k N(0,1), k = n/2.
  * ``wide_range_spd``: D C D with a dominant or Gram core and a diagonal D spanning many
    decades (extreme dynamic range).
  * ``known_factor``: a random lower-triangular L with positive diagonal (for A = L L^T tests).

All matrices are returned as full symmetric float64 numpy arrays (C order; since
they are symmetric the same buffer is also the column-major matrix).
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 2601008082
GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_TWO_M53 = float(2.0 ** -53)

# Streams: distinct sub-keys so that matrix, rhs and point draws never overlap.
STREAM_MATRIX = 1
STREAM_RHS = 2
STREAM_POINTS = 3
STREAM_FACTOR = 4
STREAM_GRAM = 5
STREAM_SCALE = 6


def seed_for(config_index: int, instance: int = 0) -> int:
    """Seed of instance ``instance`` of workload ``config_index``."""
    return SEED_BASE + 1000 * config_index + instance


def _mix(z: np.ndarray) -> np.ndarray:
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def _key(seed: int, stream: int) -> np.uint64:
    s = np.array([(seed * 0x100000001B3 + stream) & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
    return _mix(s)[0]


def _raw(key: np.uint64, counters: np.ndarray) -> np.ndarray:
    c = counters.astype(np.uint64, copy=False)
    with np.errstate(over="ignore"):
        return _mix(key + (c + np.uint64(1)) * GAMMA)


def uniforms(seed: int, stream: int, counters: np.ndarray) -> np.ndarray:
    """U[0,1) float64 for each counter."""
    return (_raw(_key(seed, stream), counters) >> np.uint64(11)).astype(np.float64) * _TWO_M53


def normals(seed: int, stream: int, counters: np.ndarray) -> np.ndarray:
    """N(0,1) float64 for each counter (Box-Muller, cosine branch)."""
    key = _key(seed, stream)
    c = counters.astype(np.uint64, copy=False) * np.uint64(2)
    u1 = ((_raw(key, c) >> np.uint64(11)).astype(np.float64) + 1.0) * _TWO_M53   # (0, 1]
    u2 = (_raw(key, c + np.uint64(1)) >> np.uint64(11)).astype(np.float64) * _TWO_M53
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def _sym_normal(n: int, seed: int, block: int = 1024) -> np.ndarray:
    """(B + B^T)/2 for B_ij = normal(counter i*n + j), drawn by row blocks."""
    A = np.empty((n, n), dtype=np.float64)
    cols = np.arange(n, dtype=np.uint64)
    for r0 in range(0, n, block):
        r1 = min(n, r0 + block)
        rows = np.arange(r0, r1, dtype=np.uint64)[:, None]
        b_rows = normals(seed, STREAM_MATRIX, rows * np.uint64(n) + cols[None, :])   # B[r, :]
        b_cols = normals(seed, STREAM_MATRIX, cols[None, :] * np.uint64(n) + rows)   # B[:, r]^T
        A[r0:r1, :] = 0.5 * (b_rows + b_cols)
    return A


def dominant_spd(n: int, rho: float, seed: int, shift: float = 0.0) -> np.ndarray:
    """Strictly diagonally dominant symmetric matrix: A_ii = rho*sum_{j!=i}|A_ij| + shift."""
    A = _sym_normal(n, seed)
    idx = np.arange(n)
    A[idx, idx] = 0.0
    off = np.abs(A).sum(axis=1)
    A[idx, idx] = rho * off + shift
    return A


def paper_spd(n: int, seed: int) -> np.ndarray:
    """Symmetric uniform [0,1) entries with n added to the diagonal (paper Sec. 4.1)."""
    A = np.empty((n, n), dtype=np.float64)
    cols = np.arange(n, dtype=np.uint64)
    for r0 in range(0, n, 1024):
        r1 = min(n, r0 + 1024)
        rows = np.arange(r0, r1, dtype=np.uint64)[:, None]
        u_rows = uniforms(seed, STREAM_MATRIX, rows * np.uint64(n) + cols[None, :])
        u_cols = uniforms(seed, STREAM_MATRIX, cols[None, :] * np.uint64(n) + rows)
        A[r0:r1, :] = 0.5 * (u_rows + u_cols)
    A[np.arange(n), np.arange(n)] += n
    return A


def rbf_spd(n: int, seed: int, length: float = 0.5, jitter: float = 1e-2) -> np.ndarray:
    """Squared-exponential kernel matrix on x_i ~ U[0,1]^3 plus jitter * I."""
    x = uniforms(seed, STREAM_POINTS, np.arange(3 * n, dtype=np.uint64)).reshape(n, 3)
    d2 = ((x[:, None, :] - x[None, :, :]) ** 2).sum(axis=2)
    A = np.exp(-d2 / (2.0 * length * length))
    A[np.arange(n), np.arange(n)] += jitter
    return A


def gram_spd(n: int, alpha: float, seed: int) -> np.ndarray:
    """A = G G^T / k + alpha I, G n x k iid N(0,1), k = n // 2 (rank-deficient Gram plus shift)."""
    k = max(1, n // 2)
    G = normals(seed, STREAM_GRAM, np.arange(n * k, dtype=np.uint64)).reshape(n, k)
    A = (G @ G.T) / k
    A = 0.5 * (A + A.T)
    A[np.arange(n), np.arange(n)] += alpha
    return A


def wide_range_spd(n: int, decades: float, seed: int, core: str = "dominant", rho: float = 1.5,
                   alpha: float = 1e-2) -> np.ndarray:
    """A = D C D with C a "dominant" (rho) or "gram" (alpha) SPD core and D = diag(d),
    d_i = 10^((decades / 4)(2 u_i - 1)), u_i ~ U[0,1): the diagonal spans about `decades`
    decades and the entries far more (matrices with an extreme dynamic range, Sec. 4.5)."""
    C = dominant_spd(n, rho, seed) if core == "dominant" else gram_spd(n, alpha, seed)
    u = uniforms(seed, STREAM_SCALE, np.arange(n, dtype=np.uint64))
    d = 10.0 ** ((decades / 4.0) * (2.0 * u - 1.0))
    return C * d[:, None] * d[None, :]


def rhs(n: int, nrhs: int, seed: int) -> np.ndarray:
    """n x nrhs iid N(0,1) right-hand sides (Fortran order: column j is contiguous)."""
    z = normals(seed, STREAM_RHS, np.arange(n * nrhs, dtype=np.uint64))
    return np.asfortranarray(z.reshape(nrhs, n).T)


def known_factor(n: int, seed: int, integer: bool = False) -> np.ndarray:
    """Random lower-triangular L with positive diagonal.

    float: diagonal U[1,2], strictly lower N(0,1)/sqrt(n).
    integer: diagonal in {1,2,3}, strictly lower in {-3..3}, so that L L^T is exact in float64
    for moderate n.
    """
    idx = np.arange(n * n, dtype=np.uint64)
    if integer:
        u = uniforms(seed, STREAM_FACTOR, idx).reshape(n, n)
        L = np.floor(u * 7.0) - 3.0
        d = 1.0 + np.floor(uniforms(seed, STREAM_FACTOR + 10, np.arange(n, dtype=np.uint64)) * 3.0)
    else:
        L = normals(seed, STREAM_FACTOR, idx).reshape(n, n) / np.sqrt(n)
        d = 1.0 + uniforms(seed, STREAM_FACTOR + 10, np.arange(n, dtype=np.uint64))
    L = np.tril(L, -1)
    L[np.arange(n), np.arange(n)] = d
    return L
