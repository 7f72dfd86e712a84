"""Pins of the precision-tree emulator (oracle/tree.py).

The emulator walks Alg. 1-3 recursively.  It is pinned by
  * the all-FP64 tree, which must reproduce the plain Cholesky (Sec. 3.2: the
    recursion only reorders the arithmetic);
  * an independent, non-recursive formulation written here: a left-looking
    block Cholesky in which every update term l_ik * l_jk is rounded in the
    precision of the shallower of the two tree nodes that separate (i, j) and
    (j, k).  Following Alg. 1-3 by hand, an update to an entry of a node's A21
    is made by that node's TRSM and an update to its A22 by that node's SYRK,
    so this is the precision the tree assigns to the term.  With every leaf in
    FP64 the two computations differ only in float64 rounding order;
  * flop shares of a level, which follow from Alg. 1-3 in closed form;
  * the accuracy ladder of Sec. 4.2 (ordering only).
"""
import json
import os

import numpy as np
import pytest

from oracle import dense, lowprec, tree
from synth import dominant_spd, paper_spd, seed_for

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_parse_and_split():
    t = tree.parse("[F16,F16,F16,F16,F32|F64@128]")
    assert t.levels == ["F16"] * 4 + ["F32"] and t.inner == "F64" and t.inner_size == 128
    t = tree.parse("[F8,F16,F16,F32|F64@128]")
    assert t.levels[0] == "F8"
    for bad in ["F16,F32", "[F12]", "[]", "[F16|F16@12]"]:
        with pytest.raises(ValueError):
            tree.parse(bad)
    assert tree.split(8192) == 4096 and tree.split(1000) == 512 and tree.split(7) == 3
    for n in range(2, 3000):
        n1 = tree.split(n)
        assert 0 < n1 < n
        if n >= 512:
            assert n1 % 128 == 0
        elif n >= 32:
            assert n1 % 16 == 0


def test_precision_assignment_by_depth_and_inner():
    t = tree.parse("[F16,F16,F32|F64@128]")
    assert tree.node_prec(t, 0, 4096) == "F16"
    assert tree.node_prec(t, 1, 2048) == "F16"
    assert tree.node_prec(t, 2, 1024) == "F32"
    assert tree.node_prec(t, 5, 256) == "F32"
    assert tree.node_prec(t, 6, 128) == "F64"


@pytest.mark.parametrize("n,leaf", [(1, 64), (64, 64), (65, 64), (300, 64), (1000, 128), (777, 96)])
def test_all_f64_tree_equals_plain_cholesky(n, leaf):
    A = dominant_spd(n, 1.0, seed_for(0, n), shift=1.0)
    L0, info0 = dense.cholesky(A)
    L1, info1, _ = tree.emulate_potrf(A, tree.parse("[F64]", leaf=leaf))
    assert info0 == info1 == 0
    assert dense.factor_error(L1, L0) <= 1e-14
    assert dense.backward_error(A, L1) <= 1e-13


def test_level_flop_shares_closed_form():
    # level l of a power-of-two tree carries 0.75 * 4^-l of n^3/3 (m^3/4 per node of order m)
    t = tree.parse("[F16,F16,F16,F16,F32|F64@128]")
    s = tree.level_flop_split(8192, t)
    assert abs(s["F16"] - (1 - 4.0 ** -4)) < 1e-12
    assert abs(s["F64"] - 4.0 ** -6) < 1e-12
    t = tree.parse("[F8,F16,F16,F32|F64@128]")
    s = tree.level_flop_split(32768, t)
    assert abs(s["F8"] - 0.75) < 1e-12 and abs(s["F16"] - (0.25 - 4.0 ** -3)) < 1e-12


# ---------------------------------------------------------------------------------------
# independent left-looking formulation with per-term precision
# ---------------------------------------------------------------------------------------
def _leaves_and_nodes(n, t):
    """Leaf ranges with their depth, and for each internal node its (depth, order, split index)."""
    leaves, nodes = [], []

    def walk(off, m, depth):
        if m <= t.leaf:
            leaves.append((off, m, depth))
            return
        m1 = tree.split(m)
        nodes.append((off, m, depth, off + m1))
        walk(off, m1, depth + 1)
        walk(off + m1, m - m1, depth + 1)

    walk(0, n, 0)
    return leaves, nodes


def _separating_node(nodes, a, b):
    """Deepest node containing indices a < b with a left of its split and b right of it."""
    best = None
    for off, m, depth, s in nodes:
        if off <= a < s <= b < off + m:
            if best is None or depth > best[0]:
                best = (depth, m)
    return best


def _round(p, X, M=None, r0=0, c0=0, sb=128):
    if p == "F64":
        return X
    if p == "F32":
        return lowprec.round_f32(X)
    if p == "F16":
        q, a = lowprec.quantize_f16(X)
        assert a == 1.0
        return q
    q, s = lowprec.quantize_e4m3_tiles(M, r0, c0, X.shape[0], X.shape[1], sb)
    return q * s


def _leaf_potrf_at(p, S):
    """Diagonal leaf of precision p (the tree's reading of a leaf POTRF at that level)."""
    if p == "F64":
        return dense.cholesky(S)
    if p == "F32":
        return dense.cholesky(lowprec.round_f32(S), np.float32)
    L, info = dense.cholesky(lowprec.round_f16(S), np.float32)
    return lowprec.round_f16(L), info


def left_looking_reference(A, t, leaf_compute="F64"):
    """Left-looking block Cholesky over the tree's leaves, every update term l_ik l_jk
    rounded at the precision of the shallower separating node.  leaf_compute="F64" runs
    every leaf in FP64; None runs each diagonal leaf at its own node's precision and each
    off-diagonal leaf solve in FP32 when its separating node is not F64."""
    n = A.shape[0]
    leaves, nodes = _leaves_and_nodes(n, t)
    L = np.zeros((n, n))
    for J, (j0, nj, dj) in enumerate(leaves):
        for I in range(J, len(leaves)):
            i0, ni, _ = leaves[I]
            S = np.array(np.tril(A)[i0:i0 + ni, j0:j0 + nj]) if I == J else np.array(A[i0:i0 + ni, j0:j0 + nj])
            for K in range(J):
                k0, nk, _ = leaves[K]
                njk = _separating_node(nodes, k0, j0)
                if I == J:
                    node = njk
                else:
                    nij = _separating_node(nodes, j0, i0)
                    node = nij if nij[0] < njk[0] else njk
                p = tree.node_prec(t, node[0], node[1])
                Xi = _round(p, L[i0:i0 + ni, k0:k0 + nk], L, i0, k0)
                Xj = _round(p, L[j0:j0 + nj, k0:k0 + nk], L, j0, k0)
                S -= Xi @ Xj.T
            if I == J:
                p = "F64" if leaf_compute == "F64" else tree.node_prec(t, dj, nj)
                Lj, info = _leaf_potrf_at(p, S)
                assert info == 0
                L[j0:j0 + nj, j0:j0 + nj] = Lj
            else:
                nij = _separating_node(nodes, j0, i0)
                p = tree.node_prec(t, nij[0], nij[1])
                dt = np.float64 if (p == "F64" or leaf_compute == "F64") else np.float32
                L[i0:i0 + ni, j0:j0 + nj] = dense.trsm_rlt(S, L[j0:j0 + nj, j0:j0 + nj], dt)
    return L


def _leaf_solves_are_per_leaf(n, t):
    """True when every leaf TRSM of Alg. 2 covers the columns of exactly one POTRF leaf:
    a node's A21 has more rows than the TRSM base case, or its A11 is itself one leaf.
    (Otherwise one FP32 substitution spans several leaves, which the per-leaf left-looking
    order does not model.)"""
    ok = True

    def walk(m):
        nonlocal ok
        if m <= t.leaf:
            return
        m1 = tree.split(m)
        if not (m - m1 > t.tleaf() or m1 <= t.leaf):
            ok = False
        walk(m1)
        walk(m - m1)

    walk(n)
    return ok


@pytest.mark.parametrize("spec,n,leaf", [
    ("[F16,F32]", 384, 64),
    ("[F16,F16,F32|F64@64]", 640, 64),
    ("[F32,F16,F64]", 520, 64),
    ("[F16,F16,F16,F32|F64@128]", 1024, 128),
    ("[F8,F16,F32|F64@128]", 1024, 128),
])
def test_emulator_matches_left_looking_term_precision(spec, n, leaf):
    t = tree.parse(spec, leaf=leaf)
    A = dominant_spd(n, 1.05, seed_for(1, n))
    L_emu, info, _ = tree.emulate_potrf(A, t, leaf_compute="F64")
    assert info == 0
    L_ref = left_looking_reference(A, t)
    err = np.max(np.abs(L_emu - L_ref)) / np.max(np.abs(L_ref))
    assert err <= 1e-13, err
    # and the reduced precision did something: far from the FP64 factor
    L64, _ = dense.cholesky(A)
    assert dense.factor_error(L_emu, L64) > 1e-9


def test_a_misplaced_precision_is_detected():
    """Rounding the TRSM terms by the (deeper) L-node level instead of the destination
    level is a plausible mistake; the left-looking reference must tell them apart."""
    t = tree.parse("[F16,F32]", leaf=64)
    A = dominant_spd(384, 1.05, seed_for(1, 384))
    L_ref = left_looking_reference(A, t)

    class Wrong(tree.Emulator):
        def trsm(self, r0, m, c0, nc, p):
            super().trsm(r0, m, c0, nc, "F32" if p == "F16" else p)

    em = Wrong(A, t, leaf_compute="F64")
    em.potrf(0, em.n, 0)
    err = np.max(np.abs(np.tril(em.M) - L_ref)) / np.max(np.abs(L_ref))
    assert err > 1e-8


def test_accuracy_ladder_of_the_paper_in_shape():
    with open(os.path.join(GOLD, "paper_numbers.json")) as f:
        ladder = json.load(f)["accuracy_digits_ladder"]
    n = 1024
    A = paper_spd(n, seed_for(9, 0))
    errs = []
    for spec in ladder["order_best_to_worst"]:
        L, info, _ = tree.emulate_potrf(A, tree.parse(spec, leaf=128))
        assert info == 0
        errs.append(dense.backward_error(A, L))
    assert -np.log10(errs[0]) >= ladder["F64_min_digits"]
    assert -np.log10(errs[-1]) <= ladder["F16_max_digits"]
    # mixed configurations sit between pure FP32-level and pure FP16
    assert errs[0] < errs[1] < errs[2]
    assert errs[3] < errs[-1] and errs[4] < errs[-1]


def test_fp8_level_uses_tile_scales():
    t = tree.parse("[F8,F32|F64@128]", leaf=128)
    A = dominant_spd(512, 2.0, seed_for(2, 512))
    L, info, em = tree.emulate_potrf(A, t)
    assert info == 0
    be = dense.backward_error(A, L)
    # E4M3 keeps 3 mantissa bits: the error is far above FP16's but bounded
    assert 1e-5 < be < 5e-2
    assert any(c[0] == "F8" for c in em.gemm_calls)


# ---------------------------------------------------------------------------------------
# FP32 (and FP16) leaves: the emulator's reduced-precision leaf POTRF and leaf TRSM
# ---------------------------------------------------------------------------------------
FP32_LEAF_CASES = [
    ("[F32]", 384, 64),
    ("[F16,F32]", 384, 64),
    ("[F16,F16,F32|F64@64]", 640, 64),
    ("[F16,F16,F16,F32|F64@128]", 1024, 128),
    ("[F16]", 384, 64),
]


@pytest.mark.parametrize("spec,n,leaf", FP32_LEAF_CASES)
def test_emulator_reduced_precision_leaves_match_left_looking(spec, n, leaf):
    """With every leaf at its tree precision, the independent left-looking order must
    reproduce the emulator (both take each leaf's input from float64 sums of the same
    rounded terms, so only their float64 order differs), and both must sit far from the
    same tree with FP64 leaves (the FP32 leaf arithmetic is really there)."""
    t = tree.parse(spec, leaf=leaf)
    assert _leaf_solves_are_per_leaf(n, t)
    A = dominant_spd(n, 1.05, seed_for(1, n))
    L_emu, info, _ = tree.emulate_potrf(A, t)
    assert info == 0
    L_ref = left_looking_reference(A, t, leaf_compute=None)
    L_f64leaves, _, _ = tree.emulate_potrf(A, t, leaf_compute="F64")
    d_ref = np.linalg.norm(L_emu - L_ref)
    d_leaf = np.linalg.norm(L_emu - L_f64leaves)
    assert d_leaf > 1e-9 * np.linalg.norm(L_ref)
    assert d_ref <= 1e-4 * d_leaf, (d_ref, d_leaf)


def test_a_leaf_computed_in_fp64_is_detected():
    """Plausible mistake: an F32 diagonal leaf (or an FP32 leaf solve) evaluated in
    float64.  The left-looking FP32-leaf reference must reject both."""
    t = tree.parse("[F16,F32]", leaf=64)
    n = 384
    A = dominant_spd(n, 1.05, seed_for(1, n))
    L_ref = left_looking_reference(A, t, leaf_compute=None)

    class LeafF64(tree.Emulator):
        def _leaf_potrf(self, off, nb, p):
            super()._leaf_potrf(off, nb, "F64" if p == "F32" else p)

    class SolveF64(tree.Emulator):
        def _leaf_trsm(self, r0, m, c0, nc, p):
            B = self.M[r0:r0 + m, c0:c0 + nc]
            self.M[r0:r0 + m, c0:c0 + nc] = dense.trsm_rlt(B, self.M[c0:c0 + nc, c0:c0 + nc])

    L_ok, _, _ = tree.emulate_potrf(A, t)
    d_ok = np.linalg.norm(L_ok - L_ref)
    for cls in (LeafF64, SolveF64):
        em = cls(A, t)
        em.potrf(0, em.n, 0)
        d_bad = np.linalg.norm(np.tril(em.M) - L_ref)
        assert d_bad > 1e3 * d_ok, (cls.__name__, d_bad, d_ok)


def _f32_exact(x):
    return np.array_equal(np.asarray(x, np.float64), np.asarray(x, np.float32).astype(np.float64))


@pytest.mark.parametrize("n", [1, 2, 17, 64, 128])
def test_fp32_cholesky_is_single_precision_arithmetic(n):
    """dense.cholesky(., float32), the emulator's F32 leaf: every entry of L is a float32
    value; the entrywise backward error meets Higham's bound for Cholesky in floating point
    (Thm. 10.3: |A - L L^T| <= gamma_{n+1} |L| |L^T|, u = 2^-24); and on a generic matrix
    it is not the float64 factor rounded once (most entries differ from that rounding,
    since a float32 sum accumulates several roundings)."""
    A = dominant_spd(n, 1.05, seed_for(1, 500 + n), shift=1.0)
    A32 = lowprec.round_f32(A)
    L, info = dense.cholesky(A, np.float32)
    assert info == 0 and _f32_exact(L)
    u = 2.0 ** -24
    g = (n + 1) * u / (1 - (n + 1) * u)
    R = np.abs(np.tril(A32) - np.tril(L @ L.T))
    assert np.all(R <= g * np.tril(np.abs(L) @ np.abs(L).T) + 1e-300)
    if n >= 64:
        L64r = lowprec.round_f32(dense.cholesky(A32)[0])
        low = np.tril_indices(n)
        assert np.mean(L[low] != L64r[low]) > 0.1


def test_fp32_cholesky_recovers_an_exact_factor():
    """L with power-of-two diagonal and small integer entries: A = L L^T and every
    intermediate of the column formula are integers below 2^24 (or exact quotients by a
    power of two), so single-precision arithmetic returns L exactly."""
    n = 48
    rng = np.random.default_rng(seed_for(1, 600))
    L = np.tril(rng.integers(-3, 4, (n, n)).astype(np.float64), -1)
    np.fill_diagonal(L, 2.0 ** rng.integers(0, 3, n))
    A = L @ L.T
    assert np.max(np.abs(A)) < 2 ** 24
    L32, info = dense.cholesky(A, np.float32)
    assert info == 0 and np.array_equal(L32, L)


@pytest.mark.parametrize("m,n", [(1, 1), (5, 16), (70, 64), (300, 128)])
def test_fp32_trsm_is_single_precision_arithmetic(m, n):
    """dense.trsm_rlt(., float32), the emulator's FP32 leaf solve X = B L^{-T}: float32
    entries; each row meets the triangular-solve backward bound (Higham Thm. 8.5:
    |b - x L^T| <= gamma_n |x| |L^T| with u = 2^-24); not the float64 solve rounded once;
    and a row's result does not depend on the other rows solved with it."""
    rng = np.random.default_rng(seed_for(1, 700 + n))
    L = lowprec.round_f32(np.tril(rng.standard_normal((n, n))) / np.sqrt(n) + 2.0 * np.eye(n))
    B = lowprec.round_f32(rng.standard_normal((m, n)))
    X = dense.trsm_rlt(B, L, np.float32)
    assert _f32_exact(X)
    u = 2.0 ** -24
    g = n * u / (1 - n * u)
    assert np.all(np.abs(B - X @ L.T) <= g * (np.abs(X) @ np.abs(L).T) + 1e-300)
    if m * n >= 4000:
        X64r = lowprec.round_f32(dense.trsm_rlt(B, L))
        assert np.mean(X != X64r) > 0.1
    if m > 3:
        assert np.array_equal(dense.trsm_rlt(B[2:m - 1], L, np.float32), X[2:m - 1])


def test_fp32_trsm_recovers_an_exact_solution():
    n, m = 40, 30
    rng = np.random.default_rng(seed_for(1, 800))
    L = np.tril(rng.integers(-2, 3, (n, n)).astype(np.float64), -1)
    np.fill_diagonal(L, 2.0 ** rng.integers(0, 3, n))
    X = rng.integers(-4, 5, (m, n)).astype(np.float64)
    B = X @ L.T
    assert np.max(np.abs(B)) < 2 ** 24
    assert np.array_equal(dense.trsm_rlt(B, L, np.float32), X)


# ---------------------------------------------------------------------------------------
# dynamic quantization: power-of-two two-sided diagonal scaling (emulate_potrf_scaled)
# ---------------------------------------------------------------------------------------
def test_scaled_factor_is_row_scaled_exactly():
    """For A = P C P with P a diagonal of powers of two, the scaled emulation returns exactly
    P times C's scaled factor: the exponents shift by those of P and the tree sees the same
    A_hat.  A mistake in the exponents (one-sided scaling, wrong sign, rounding of the scale)
    breaks the equality."""
    n = 300
    from synth import dominant_spd
    C = dominant_spd(n, 1.5, seed_for(10, 1))
    rng = np.random.default_rng(5)
    p = 2.0 ** rng.integers(-40, 41, n)
    A = C * p[:, None] * p[None, :]
    t = tree.parse("[F16,F32]", leaf=64)
    LA, infoA, _ = tree.emulate_potrf_scaled(A, t)
    LC, infoC, _ = tree.emulate_potrf_scaled(C, t)
    assert infoA == infoC == 0
    assert np.array_equal(LA, LC * p[:, None])


def test_scaling_is_the_identity_on_a_unit_diagonal():
    n = 256
    from synth import dominant_spd
    C = dominant_spd(n, 1.5, seed_for(10, 2))
    s = 1 / np.sqrt(np.diag(C))
    C1 = C * s[:, None] * s[None, :]           # unit diagonal: every exponent is 0
    assert not tree.diagonal_scale_exponents(C1).any()
    t = tree.parse("[F16,F16,F32|F64@64]", leaf=64)
    assert np.array_equal(tree.emulate_potrf_scaled(C1, t)[0], tree.emulate_potrf(C1, t)[0])


def test_static_quantization_fails_on_an_extreme_range_and_scaling_does_not():
    """Sec. 4.5: with an extreme dynamic range the static per-block scaling flushes the small
    values and the factorization loses positive definiteness (info > 0); the dynamic scheme
    factors the same matrix with the scaled backward error of the core matrix alone."""
    from synth import gram_spd, wide_range_spd
    n = 512
    t = tree.parse("[F16,F16,F32|F64@128]", leaf=64)
    A = wide_range_spd(n, 24, seed_for(10, 3), core="gram", alpha=1e-3)
    _, info, _ = tree.emulate_potrf(A, t)
    assert info > 0
    L, info_s, _ = tree.emulate_potrf_scaled(A, t)
    assert info_s == 0
    C = gram_spd(n, 1e-3, seed_for(10, 3))
    Lc, _, _ = tree.emulate_potrf_scaled(C, t)
    assert dense.scaled_backward_error(A, L) <= 2 * dense.scaled_backward_error(C, Lc)


def test_scaled_diagonal_lies_in_half_to_two():
    """The exponents bring every positive, finite diagonal entry into [0.5, 2) whatever its
    magnitude (including subnormal and near-overflow entries), and leave the others alone."""
    rng = np.random.default_rng(7)
    d = np.ldexp(rng.uniform(0.5, 1.0, 400), rng.integers(-1070, 1020, 400))
    A = np.diag(d)
    e = tree.diagonal_scale_exponents(A)
    s = np.ldexp(np.ldexp(d, -e), -e)
    assert np.all((s >= 0.5) & (s < 2.0))
    bad = np.diag(np.array([0.0, -3.0, np.inf, np.nan, 1e300]))
    assert tree.diagonal_scale_exponents(bad).tolist()[:4] == [0, 0, 0, 0]


def test_split_fp32_levels_recover_an_exact_factor():
    """Integer L with a unit diagonal and entries in {-3..3}: every operand is exact in TF32 and
    every leaf exact in FP32, so the split emulation returns L itself."""
    n = 300
    L = np.tril(np.floor(np.random.default_rng(15).uniform(0, 7, (n, n))) - 3.0, -1) + np.eye(n)
    A = L @ L.T
    Le, info, _ = tree.emulate_potrf(A, tree.parse("[F32,F32|F64@64]", leaf=64), f32_split=True)
    assert info == 0 and np.array_equal(Le, L)


def test_split_fp32_levels_are_fp32_accurate_and_differ_from_plain_fp32():
    from synth import dominant_spd
    n = 512
    A = dominant_spd(n, 1.5, seed_for(10, 20))
    t = tree.parse("[F32,F32|F64@64]", leaf=64)
    Ls, _, _ = tree.emulate_potrf(A, t, f32_split=True)
    Lp, _, _ = tree.emulate_potrf(A, t)
    L64, _ = dense.cholesky(A)
    assert not np.array_equal(Ls, Lp)
    for L in (Ls, Lp):
        assert dense.backward_error(A, L) <= 8 * 2.0 ** -24
        assert dense.factor_error(L, L64) <= 1e-6
