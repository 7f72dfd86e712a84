"""Precision tree and a step-by-step emulator of the nested recursive Cholesky.

The emulator walks Algorithms 1-3 (Sec. 3.2) in the paper's order on a float64
master copy of A, applying the tree-structured precision assignment of Sec. 3.3
and the per-block scaling of Sec. 3.4 at every low-precision GEMM.  It is the
definition the mixed-precision GPU path is compared against.

Readings of the paper (each one listed in the design notes):
  * Split point (Alg. 1-3 "e.g. n1 = floor(n/2)"): n1 = n/2 rounded to the nearest
    multiple of q, q = 128 for n >= 512, q = 16 for 32 <= n < 512, and floor(n/2)
    below 32 (or whenever the rounded split would be empty).  TRSM and SYRK use
    the same rule, so their sub-blocks are the POTRF tree's blocks.
  * Leaf tests: n <= b (Alg. 1, 3) and min(m, n) <= b (Alg. 2).
  * Precision list [p0, ..., p_{d-1}] (Sec. 4.2, outermost to innermost): the
    off-diagonal TRSM/SYRK work of a node at depth t uses p_t; nodes at depth
    >= d-1 use p_{d-1} throughout.  An optional inner precision ("|F64@128")
    takes over for every node of order <= inner_size.
  * Operand precision: every GEMM inside a node's TRSM or SYRK takes both operands
    in that node's precision p (L blocks of deeper nodes are rounded down to p),
    and the exact products are accumulated in float64 here (FP32 on the GPU).
  * Leaf TRSM at a reduced-precision level runs in FP32 on FP32-rounded B and L;
    at an F64 level in FP64.  Leaf SYRK at level p is the lower triangle of the
    GEMM at p.  A leaf POTRF at F32 runs in FP32 on FP32-rounded input; at F16 in
    FP32 on FP16-rounded input with the result rounded to FP16.
  * Storage: the master keeps the unrounded computed values (FP64 storage); the
    reduced-precision copies exist only as GEMM operands.
"""
from __future__ import annotations

import re
from dataclasses import dataclass, field

import numpy as np

from . import dense, lowprec

PRECS = ("F64", "F32", "F16", "F8")


@dataclass
class Tree:
    levels: list = field(default_factory=lambda: ["F64"])
    leaf: int = 128
    inner: str | None = None
    inner_size: int = 0
    trsm_leaf: int = 0
    syrk_leaf: int = 0
    scale_block: int = 128

    def tleaf(self) -> int:
        return self.trsm_leaf or self.leaf

    def sleaf(self) -> int:
        return self.syrk_leaf or self.leaf


def parse(spec: str, leaf: int = 128, trsm_leaf: int = 0, syrk_leaf: int = 0) -> Tree:
    """Parse "[F16,F16,F32]" or "[F8,F16,F32|F64@128]" (F8 = E4M3)."""
    m = re.fullmatch(r"\s*\[([^\]|]*)(?:\|\s*(F64|F32)\s*@\s*(\d+))?\]\s*", spec)
    if not m:
        raise ValueError(f"bad tree spec {spec!r}")
    levels = [t.strip().upper() for t in m.group(1).split(",") if t.strip()]
    levels = ["F8" if t in ("F8E4M3", "E4M3") else t for t in levels]
    if not levels or any(t not in PRECS for t in levels):
        raise ValueError(f"bad precision list in {spec!r}")
    inner = m.group(2)
    inner_size = int(m.group(3)) if m.group(3) else 0
    return Tree(levels=levels, leaf=leaf, inner=inner, inner_size=inner_size,
                trsm_leaf=trsm_leaf, syrk_leaf=syrk_leaf)


def split(n: int) -> int:
    """n1 of a node of order n (n2 = n - n1)."""
    if n >= 512:
        q = 128
    elif n >= 32:
        q = 16
    else:
        return n // 2
    n1 = q * ((n + q) // (2 * q))
    if n1 <= 0 or n1 >= n:
        return n // 2
    return n1


def node_prec(tree: Tree, depth: int, n: int) -> str:
    if tree.inner and n <= tree.inner_size:
        return tree.inner
    return tree.levels[min(depth, len(tree.levels) - 1)]


def _compute_dtype(p: str):
    return np.float64 if p == "F64" else np.float32


class Emulator:
    """State of one emulated factorization: the float64 master and counters."""

    def __init__(self, A: np.ndarray, tree: Tree, leaf_compute: str | None = None, f32_split: bool = False):
        self.M = np.array(A, dtype=np.float64, copy=True)
        self.f32_split = f32_split           # FP32-level GEMMs by the TF32 split (lowprec)
        self.n = self.M.shape[0]
        self.tree = tree
        self.leaf_compute = leaf_compute     # None, or "F64" to run every leaf in FP64
        self.info = 0
        self.flops = {p: 0.0 for p in PRECS}
        self.gemm_calls = []                 # (prec, m, n, k) per low-level GEMM

    # -- leaves --------------------------------------------------------------
    def _leaf_potrf(self, off: int, n: int, p: str) -> None:
        blk = self.M[off:off + n, off:off + n]
        if self.leaf_compute == "F64":
            p = "F64"
        if p == "F64":
            L, info = dense.cholesky(blk, np.float64)
        elif p == "F32":
            L, info = dense.cholesky(lowprec.round_f32(blk), np.float32)
        elif p == "F16":
            L, info = dense.cholesky(lowprec.round_f16(blk), np.float32)
            L = lowprec.round_f16(L)
        else:
            raise ValueError("an FP8 diagonal leaf is not defined")
        if info:
            self.info = off + info
            return
        low = np.tril_indices(n)
        blk[low] = L[low]
        self.flops[p] += n ** 3 / 3.0

    def _leaf_trsm(self, r0: int, m: int, c0: int, nc: int, p: str) -> None:
        cp = "F64" if (p == "F64" or self.leaf_compute == "F64") else "F32"
        B = self.M[r0:r0 + m, c0:c0 + nc]
        Ld = self.M[c0:c0 + nc, c0:c0 + nc]
        self.M[r0:r0 + m, c0:c0 + nc] = dense.trsm_rlt(B, Ld, _compute_dtype(cp))
        self.flops[p] += float(m) * nc * nc

    # -- GEMM in precision p: D -= X Y^T ----------------------------------------
    def _operands(self, p: str, r0, m, c0, nd, k0, k):
        X = self.M[r0:r0 + m, k0:k0 + k]
        Y = self.M[c0:c0 + nd, k0:k0 + k]
        if p == "F64":
            return X, Y, 1.0
        if p == "F32":
            return lowprec.round_f32(X), lowprec.round_f32(Y), 1.0
        if p == "F16":
            Xq, ax = lowprec.quantize_f16(X)
            Yq, ay = lowprec.quantize_f16(Y)
            return Xq, Yq, ax * ay
        if p == "F8":
            sb = self.tree.scale_block
            Xq, sx = lowprec.quantize_e4m3_tiles(self.M, r0, k0, m, k, sb)
            Yq, sy = lowprec.quantize_e4m3_tiles(self.M, c0, k0, nd, k, sb)
            # the tile scales are constant on each (row-tile, k-tile) cell: fold them in
            return Xq * sx, Yq * sy, 1.0
        raise ValueError(p)

    def _gemm(self, p, r0, m, c0, nd, k0, k, lower=False):
        if m == 0 or nd == 0 or k == 0:
            return
        if p == "F32" and self.f32_split:
            prod = lowprec.gemm_tf32x3(self.M[r0:r0 + m, k0:k0 + k], self.M[c0:c0 + nd, k0:k0 + k])
        else:
            X, Y, scale = self._operands(p, r0, m, c0, nd, k0, k)
            prod = scale * (X @ Y.T)
        D = self.M[r0:r0 + m, c0:c0 + nd]
        if lower:
            # only entries on or below the diagonal of the (square) destination
            mask = (np.arange(r0, r0 + m)[:, None] >= np.arange(c0, c0 + nd)[None, :])
            D -= np.where(mask, prod, 0.0)
            self.flops[p] += float(m) * m * k
        else:
            D -= prod
            self.flops[p] += 2.0 * m * nd * k
        self.gemm_calls.append((p, m, nd, k))

    # -- Alg. 2: Tree-TRSM_{R,L,T}(B, L) with B = M[r0:r0+m, c0:c0+nc] -----------
    def trsm(self, r0, m, c0, nc, p):
        if min(m, nc) <= self.tree.tleaf():
            self._leaf_trsm(r0, m, c0, nc, p)
            return
        n1 = split(nc)
        self.trsm(r0, m, c0, n1, p)
        self._gemm(p, r0, m, c0 + n1, nc - n1, c0, n1)       # B2 -= B1 L21^T
        self.trsm(r0, m, c0 + n1, nc - n1, p)

    # -- Alg. 3: Tree-SYRK_L(C, A, -1, 1) with C = M[c0:c0+nc, c0:c0+nc], A = M[c0:c0+nc, a0:a0+k]
    def syrk(self, c0, nc, a0, k, p):
        if nc <= self.tree.sleaf():
            self._gemm(p, c0, nc, c0, nc, a0, k, lower=True)
            return
        n1 = split(nc)
        self.syrk(c0, n1, a0, k, p)
        self._gemm(p, c0 + n1, nc - n1, c0, n1, a0, k)       # C21 -= A2 A1^T
        self.syrk(c0 + n1, nc - n1, a0, k, p)

    # -- Alg. 1: Tree-POTRF_L(A) with A = M[off:off+n, off:off+n] -----------------
    def potrf(self, off, n, depth=0):
        if self.info or n == 0:
            return
        p = node_prec(self.tree, depth, n)
        if n <= self.tree.leaf:
            self._leaf_potrf(off, n, p)
            return
        n1 = split(n)
        n2 = n - n1
        self.potrf(off, n1, depth + 1)
        if self.info:
            return
        self.trsm(off + n1, n2, off, n1, p)
        self.syrk(off + n1, n2, off, n1, p)
        self.potrf(off + n1, n2, depth + 1)


def emulate_potrf(A: np.ndarray, tree: Tree, leaf_compute: str | None = None, f32_split: bool = False):
    """(L, info, emulator) of the tree-precision recursive Cholesky of A's lower triangle.
    f32_split: FP32-level GEMMs by the TF32 split (lowprec.gemm_tf32x3)."""
    em = Emulator(A, tree, leaf_compute, f32_split)
    em.potrf(0, em.n, 0)
    return np.tril(em.M), em.info, em


def level_flop_split(n: int, tree: Tree) -> dict:
    """Share of n^3/3 flops per precision implied by the tree (counted on the node sizes)."""
    out = {p: 0.0 for p in PRECS}

    def walk(m, depth):
        p = node_prec(tree, depth, m)
        if m <= tree.leaf:
            out[p] += m ** 3 / 3.0
            return
        m1 = split(m)
        m2 = m - m1
        out[p] += m2 * m1 * m1 + m2 * m2 * m1     # TRSM (m2 x m1 by m1) + SYRK lower (m2^2 m1)
        walk(m1, depth + 1)
        walk(m2, depth + 1)

    walk(n, 0)
    tot = sum(out.values())
    return {p: v / tot for p, v in out.items()}


# ---------------------------------------------------------------------------------------
# Standalone Tree-SYRK (Alg. 3) and Tree-TRSM (Alg. 2), the kernels of the paper's SYRK and
# TRSM experiments (Sec. 4.2).  Reading of a precision list for them: the GEMM of a node at
# recursion depth t is computed at levels[t] (deeper nodes at the last entry; a node of
# order <= inner_size at `inner`), a base case at the precision of its node: the leaf SYRK
# as the lower triangle of the product at that precision, the leaf TRSM in FP32 arithmetic
# on FP32-rounded B and L unless the precision is F64.  Operands are rounded per Sec. 3.4
# (alpha = max(1, amax / 65504) per operand block for FP16) and their exact products summed
# in float64.
# ---------------------------------------------------------------------------------------
def _operand(p: str, X: np.ndarray):
    if p == "F64":
        return X, 1.0
    if p == "F32":
        return lowprec.round_f32(X), 1.0
    if p == "F16":
        return lowprec.quantize_f16(X)
    raise ValueError("F8 levels are defined on the factorization's 128 x 128 tiles only")


def emulate_syrk(C: np.ndarray, A: np.ndarray, tree: Tree, f32_split: bool = False) -> np.ndarray:
    """Lower triangle of C - A A^T by Alg. 3 with the precision list applied by depth
    (f32_split: FP32-level GEMMs by the TF32 split)."""
    C = np.array(C, dtype=np.float64, copy=True)
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]

    def gemm(p, r0, m, c0, nd, lower):
        if p == "F32" and f32_split:
            prod = lowprec.gemm_tf32x3(A[r0:r0 + m], A[c0:c0 + nd])
        else:
            X, ax = _operand(p, A[r0:r0 + m])
            Y, ay = _operand(p, A[c0:c0 + nd])
            prod = (ax * ay) * (X @ Y.T)
        if lower:
            prod = np.tril(prod)
        C[r0:r0 + m, c0:c0 + nd] -= prod

    def rec(c0, nc, depth):
        if nc == 0:
            return
        p = node_prec(tree, depth, nc)
        if nc <= tree.sleaf():
            gemm(p, c0, nc, c0, nc, True)
            return
        n1 = split(nc)
        rec(c0, n1, depth + 1)
        gemm(p, c0 + n1, nc - n1, c0, n1, False)          # C21 -= A2 A1^T
        rec(c0 + n1, nc - n1, depth + 1)

    rec(0, n, 0)
    return np.tril(C)


def emulate_trsm(B: np.ndarray, L: np.ndarray, tree: Tree) -> np.ndarray:
    """X = B L^{-T} (L lower) by Alg. 2 with the precision list applied by depth."""
    X = np.array(B, dtype=np.float64, copy=True)
    L = np.tril(np.asarray(L, dtype=np.float64))
    m, n = X.shape

    def leaf(c0, nc, p):
        dt = np.float64 if p == "F64" else np.float32
        X[:, c0:c0 + nc] = dense.trsm_rlt(X[:, c0:c0 + nc], L[c0:c0 + nc, c0:c0 + nc], dt)

    def gemm(p, c0, n1, n2):
        X1, a1 = _operand(p, X[:, c0:c0 + n1])
        L21, a2 = _operand(p, L[c0 + n1:c0 + n1 + n2, c0:c0 + n1])
        X[:, c0 + n1:c0 + n1 + n2] -= (a1 * a2) * (X1 @ L21.T)   # B2 -= B1 L21^T

    def rec(c0, nc, depth):
        p = node_prec(tree, depth, nc)
        if min(m, nc) <= tree.tleaf():
            leaf(c0, nc, p)
            return
        n1 = split(nc)
        rec(c0, n1, depth + 1)
        gemm(p, c0, n1, nc - n1)
        rec(c0 + n1, nc - n1, depth + 1)

    if m and n:
        rec(0, n, 0)
    return X


# ---------------------------------------------------------------------------------------
# Dynamic quantization (the paper's future work, Sec. 4.5 and 5): two-sided diagonal scaling
# by powers of two before the recursion.  Reading: with a_ii = m 2^ex (m in [0.5, 1)),
# d_i = 2^floor(ex / 2) (d_i = 1 for a_ii <= 0 or not finite), so that a_ii / d_i^2 lies in
# [0.5, 2); A_hat = D^-1 A D^-1 (exact in float64), L_hat by the tree, then L = D L_hat
# (exact).  Every row then meets the FP16 range at the scale of its own diagonal, whatever the
# dynamic range of A; powers of two keep the scaling itself free of rounding.
# ---------------------------------------------------------------------------------------
def diagonal_scale_exponents(A: np.ndarray) -> np.ndarray:
    d = np.diag(np.asarray(A, dtype=np.float64)).copy()
    ok = np.isfinite(d) & (d > 0)
    e = np.zeros(d.shape[0], dtype=np.int64)
    _, ex = np.frexp(d[ok])
    e[ok] = np.floor_divide(ex, 2)
    return e


def emulate_potrf_scaled(A: np.ndarray, tree: Tree, leaf_compute: str | None = None):
    """(L, info, emulator) of the tree on D^-1 A D^-1, unscaled (see above)."""
    e = diagonal_scale_exponents(A)
    A = np.asarray(A, dtype=np.float64)
    Ah = np.ldexp(np.ldexp(A, -e[:, None]), -e[None, :])
    Lh, info, em = emulate_potrf(Ah, tree, leaf_compute)
    return np.ldexp(Lh, e[:, None]), info, em
