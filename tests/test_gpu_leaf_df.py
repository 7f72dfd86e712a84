"""GPU parity of the FP64 leaf factored in double-float arithmetic (hrp_set_leaf_chain(h, 1)).

The double-float leaf holds every entry as a pair of binary32 numbers (about 48 significant
bits); each of its operations has a relative error of a few units of 2^-48 (Joldes, Muller
and Popescu 2017), so the pair arithmetic's unit roundoff is taken as u = 2^-46 here.
Bounds, as for the FP64 leaf with u in place of FP64's:
* backward: |L L^T - A| <= gamma_{n+1} |L| |L^T| <= (n + 1) u max a_ii per entry (Higham,
  Thm. 10.3), times 4 for the residual product and the reciprocals;
* forward against the plain FP64 Cholesky on the well-conditioned dominant matrices: the
  same 1e-12 relative bound as the FP64 tree (measured ~1e-14).
Leaves outside the pair arithmetic's range (a diagonal spread over 2^36 or more, a pivot
that is not positive) are factored again by the FP64 schedule in the same launch: those
results equal the FP64 leaf's bit for bit, and a failing column is reported as FP64 does.
"""
import numpy as np
import pytest

from oracle import dense
from synth import dominant_spd, seed_for

pytestmark = pytest.mark.gpu

U_DF = 2.0 ** -46


@pytest.fixture(scope="module")
def hrp_mod():
    import torch
    import paper_2601_08082_gb300 as hrp
    assert torch.cuda.is_available()
    return hrp


def _factor(hrp, A, spec, leaf, mode):
    h = hrp.Handle(0)
    try:
        h.set_leaf_chain(mode)
        At = hrp.colmajor(A).cuda()
        info = h.potrf(hrp.tree_parse(spec, leaf=leaf), At)
        return np.tril(hrp.from_colmajor(At)), info
    finally:
        h.close()


def _backward_bound(A):
    n = A.shape[0]
    return 4 * (n + 1) * U_DF * np.max(np.diag(A))


@pytest.mark.parametrize("n", [33, 47, 64, 100, 127, 128])
def test_df_leaf_matches_plain_cholesky(hrp_mod, n):
    A = dominant_spd(n, 1.05, seed_for(0, 40 + n))
    L, info = _factor(hrp_mod, A, "[F64]", 128, 1)
    assert info == 0
    L0, _ = dense.cholesky(A)
    assert np.max(np.abs(L - L0)) <= 1e-12 * np.max(np.abs(L0))
    assert np.max(np.abs(L @ L.T - A)) <= _backward_bound(A)


@pytest.mark.parametrize("scale", [1.0, 1e-40, 1e40, 2.0 ** 600])
def test_df_leaf_graded_pivots(hrp_mod, scale):
    # A = G G^T with rows 2i + 1 = row 2i + eps_i h_i (eps_i from 1e-3 to 1): every odd pivot
    # is about eps_i^2 under diagonal entries about 1 (inside the pair range); the scales move
    # the whole leaf far outside binary32's exponent range, which the leaf's power-of-two
    # scale absorbs
    n = 128
    rng = np.random.default_rng(seed_for(0, 42))
    G0 = rng.standard_normal((n, 2 * n)) / np.sqrt(2 * n)
    G = G0.copy()
    G[1::2] = G0[0::2] + (10.0 ** rng.uniform(-3, 0, n // 2))[:, None] * G0[1::2]
    A = (G @ G.T) * scale
    A = 0.5 * (A + A.T)
    L, info = _factor(hrp_mod, A, "[F64]", 128, 1)
    assert info == 0
    assert np.max(np.abs(L @ L.T - A)) <= _backward_bound(A)


def test_df_tree_matches_plain_cholesky(hrp_mod):
    n = 1000
    A = dominant_spd(n, 1.0, seed_for(0, n), shift=1.0)
    L, info = _factor(hrp_mod, A, "[F64]", 128, 1)
    assert info == 0
    L0, _ = dense.cholesky(A)
    assert np.max(np.abs(L - L0)) <= 1e-12 * np.max(np.abs(L0))


@pytest.mark.parametrize("spread", [1e-12, 1e-30])
def test_df_leaf_out_of_range_refactors_in_fp64(hrp_mod, spread):
    # D A D with D_ii from 1 down to sqrt(spread): the diagonal spans 2^40 or more, so the
    # leaf is factored again by the FP64 schedule: bitwise the FP64 leaf's result
    n = 120
    A = dominant_spd(n, 1.05, seed_for(0, 43))
    d = np.sqrt(np.geomspace(1.0, spread, n))
    A = d[:, None] * A * d[None, :]
    L1, info1 = _factor(hrp_mod, A, "[F64]", 128, 1)
    L0, info0 = _factor(hrp_mod, A, "[F64]", 128, 0)
    assert info1 == info0 == 0
    assert np.array_equal(L1, L0)


@pytest.mark.parametrize("col", [1, 16, 17, 90, 127])
def test_df_leaf_reports_failing_column(hrp_mod, col):
    n = 127
    A = dominant_spd(n, 2.0, seed_for(0, 41))
    A[col - 1, col - 1] = -1e3
    _, info0 = dense.cholesky(A)
    _, info = _factor(hrp_mod, A, "[F64]", 128, 1)
    assert info == info0 == col


def test_df_leaf_failing_pivot_after_updates(hrp_mod):
    # positive diagonal, not positive definite: the pivot of column 70 turns negative only
    # after the updates of earlier columns; the double-float leaf detects the pivot and the
    # FP64 schedule reports the column exactly as the plain Cholesky does
    n = 128
    A = dominant_spd(n, 2.0, seed_for(0, 44))
    v = A[69, :69].copy()
    A[69, 69] = 0.5 * v @ np.linalg.solve(A[:69, :69], v)
    _, info0 = dense.cholesky(A)
    _, info = _factor(hrp_mod, A, "[F64]", 128, 1)
    assert info0 == 70
    assert info == info0
