"""Pins of the standalone Tree-SYRK (Alg. 3) and Tree-TRSM (Alg. 2) emulators
(oracle/tree.py: emulate_syrk, emulate_trsm) with the precision list applied by depth.

* All-FP64 lists: the recursion only reorders the arithmetic, so the results are the plain
  definitions, C - A A^T (computed as one product) and the column substitution of
  dense.trsm_rlt, to rounding order.
* Pure F16 SYRK: every product is of two FP16-rounded operands, exact in float64, so the
  result is C - r16(A) r16(A)^T as one product.
* Two-level lists: the off-diagonal block of the depth-0 node takes the level-0 rounding and
  the diagonal blocks the level-1 arithmetic, block by block in closed form.
* A GEMM rounded at the next depth's precision (a plausible indexing mistake) is detected.
"""
import numpy as np
import pytest

from oracle import dense, lowprec, tree
from synth import dominant_spd, seed_for


def _data(n, k, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, k))
    C = rng.standard_normal((n, n))
    return A, C + C.T


@pytest.mark.parametrize("n,k,leaf", [(1, 3, 64), (64, 64, 64), (300, 77, 64), (700, 512, 128)])
def test_f64_syrk_is_the_plain_product(n, k, leaf):
    A, C = _data(n, k, seed_for(5, n))
    out = tree.emulate_syrk(C, A, tree.parse("[F64]", leaf=leaf))
    ref = np.tril(C - A @ A.T)
    assert np.max(np.abs(out - ref)) <= 1e-13 * np.max(np.abs(ref))
    assert np.array_equal(np.triu(out, 1), np.zeros_like(out))


def test_pure_f16_syrk_is_one_product_of_rounded_operands():
    n, k = 500, 300
    A, C = _data(n, k, seed_for(5, 1))
    out = tree.emulate_syrk(C, A, tree.parse("[F16]", leaf=64))
    A16 = lowprec.round_f16(A)
    ref = np.tril(C - A16 @ A16.T)
    assert np.max(np.abs(out - ref)) <= 1e-13 * np.max(np.abs(ref))
    assert np.max(np.abs(out - np.tril(C - A @ A.T))) > 1e-4    # the rounding is there


def test_two_level_syrk_blocks_in_closed_form():
    n, k, leaf = 256, 200, 128
    A, C = _data(n, k, seed_for(5, 2))
    out = tree.emulate_syrk(C, A, tree.parse("[F16,F64]", leaf=leaf))
    n1 = tree.split(n)
    A1, A2 = A[:n1], A[n1:]
    assert np.allclose(out[:n1, :n1], np.tril(C[:n1, :n1] - A1 @ A1.T), rtol=0, atol=1e-12)
    assert np.allclose(out[n1:, n1:], np.tril(C[n1:, n1:] - A2 @ A2.T), rtol=0, atol=1e-12)
    r = C[n1:, :n1] - lowprec.round_f16(A2) @ lowprec.round_f16(A1).T
    assert np.max(np.abs(out[n1:, :n1] - r)) <= 1e-12


@pytest.mark.parametrize("m,n,leaf", [(1, 1, 64), (70, 64, 64), (300, 500, 64), (128, 700, 128)])
def test_f64_trsm_is_the_plain_substitution(m, n, leaf):
    L = np.tril(dense.cholesky(dominant_spd(n, 1.5, seed_for(5, 10 + n), shift=1.0))[0])
    B = np.random.default_rng(seed_for(5, 20 + m)).standard_normal((m, n))
    X = tree.emulate_trsm(B, L, tree.parse("[F64]", leaf=leaf))
    X0 = dense.trsm_rlt(B, L)
    assert np.max(np.abs(X - X0)) <= 1e-13 * np.max(np.abs(X0))
    assert np.max(np.abs(X @ L.T - B)) <= 1e-12 * np.max(np.abs(B))


def test_two_level_trsm_in_closed_form():
    m, n, leaf = 200, 256, 128
    L = np.tril(dense.cholesky(dominant_spd(n, 1.5, seed_for(5, 30), shift=1.0))[0])
    B = np.random.default_rng(seed_for(5, 31)).standard_normal((m, n))
    X = tree.emulate_trsm(B, L, tree.parse("[F16,F64]", leaf=leaf))
    n1 = tree.split(n)
    X1 = dense.trsm_rlt(B[:, :n1], L[:n1, :n1])
    B2 = B[:, n1:] - lowprec.round_f16(X1) @ lowprec.round_f16(L[n1:, :n1]).T
    X2 = dense.trsm_rlt(B2, L[n1:, n1:])
    assert np.max(np.abs(X[:, :n1] - X1)) <= 1e-14 * np.max(np.abs(X1))
    assert np.max(np.abs(X[:, n1:] - X2)) <= 1e-13 * np.max(np.abs(X2))


def test_a_gemm_at_the_wrong_depth_is_detected():
    n, k = 1024, 1024
    A, C = _data(n, k, seed_for(5, 40))
    t = tree.parse("[F16,F32]", leaf=128)
    ok = tree.emulate_syrk(C, A, t)
    shifted = tree.emulate_syrk(C, A, tree.parse("[F32]", leaf=128))    # depth 0 read as depth 1
    f64 = tree.emulate_syrk(C, A, tree.parse("[F64]", leaf=128))
    assert np.linalg.norm(ok - shifted) > 100 * np.linalg.norm(shifted - f64)
