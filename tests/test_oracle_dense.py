"""Pins of the plain FP64 oracle (oracle/dense.py) to facts outside of it.

Each test checks the oracle against something it does not compute itself:
hand-worked factors, closed forms, exact rational arithmetic, a known factor,
exact scaling identities and the backward-error invariant of Cholesky.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import dense
from synth import dominant_spd, known_factor, rhs, seed_for

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read_small():
    cases = []
    with open(os.path.join(GOLD, "chol_small.txt")) as f:
        for line in f:
            if not line.strip() or line.startswith("#"):
                continue
            name, n, a, l = [t.strip() for t in line.split("|")]
            n = int(n)
            A = np.array([float(x) for x in a.split()]).reshape(n, n)
            L = np.array([float(x) for x in l.split()]).reshape(n, n)
            cases.append((name, A, L))
    return cases


@pytest.mark.parametrize("name,A,L", _read_small())
def test_golden_small_factors(name, A, L):
    Lh, info = dense.cholesky(A)
    assert info == 0
    np.testing.assert_allclose(Lh, L, rtol=0, atol=1e-15 * np.abs(L).max())


def test_two_by_two_closed_form():
    rng = np.random.default_rng(7)
    for _ in range(50):
        a11 = rng.uniform(0.5, 4)
        a21 = rng.uniform(-1, 1)
        a22 = a21 * a21 / a11 + rng.uniform(0.1, 3)
        Lh, info = dense.cholesky(np.array([[a11, a21], [a21, a22]]))
        l11 = np.sqrt(a11)
        l21 = a21 / l11
        l22 = np.sqrt(a22 - l21 * l21)
        assert info == 0
        np.testing.assert_allclose(Lh, [[l11, 0], [l21, l22]], rtol=4e-16, atol=1e-16)


def _rational_ldl(A):
    """Exact LDL^T of a small integer SPD matrix with Python fractions."""
    n = len(A)
    a = [[Fraction(int(A[i][j])) for j in range(n)] for i in range(n)]
    L = [[Fraction(0)] * n for _ in range(n)]
    D = [Fraction(0)] * n
    for j in range(n):
        D[j] = a[j][j] - sum(L[j][k] * L[j][k] * D[k] for k in range(j))
        L[j][j] = Fraction(1)
        for i in range(j + 1, n):
            L[i][j] = (a[i][j] - sum(L[i][k] * L[j][k] * D[k] for k in range(j))) / D[j]
    return L, D


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6, 7, 8])
def test_exact_rational_small(n):
    rng = np.random.default_rng(100 + n)
    for _ in range(5):
        B = rng.integers(-3, 4, size=(n, n))
        A = B + B.T
        np.fill_diagonal(A, 0)
        np.fill_diagonal(A, np.abs(A).sum(axis=1) + rng.integers(1, 4, size=n))
        Lu, D = _rational_ldl(A)
        Lexp = np.array([[float(Lu[i][j]) * np.sqrt(float(D[j])) for j in range(n)] for i in range(n)])
        Lh, info = dense.cholesky(A.astype(float))
        assert info == 0
        np.testing.assert_allclose(Lh, Lexp, rtol=1e-14, atol=1e-15 * np.abs(Lexp).max())


def test_exhaustive_small_integer_matrices():
    # every 2 x 2 with a21 in -3..3 and a_ii = |a21| + t (t = 1..3), and every 3 x 3 with the
    # three off-diagonal entries in -3..3 and a_ii = 1 + sum_{j!=i} |a_ij|: the factor against
    # exact rational LDL^T
    cases = []
    for a21 in range(-3, 4):
        for t1 in range(1, 4):
            for t2 in range(1, 4):
                cases.append(np.array([[abs(a21) + t1, a21], [a21, abs(a21) + t2]], dtype=np.int64))
    for a21 in range(-3, 4):
        for a31 in range(-3, 4):
            for a32 in range(-3, 4):
                A = np.array([[0, a21, a31], [a21, 0, a32], [a31, a32, 0]], dtype=np.int64)
                np.fill_diagonal(A, np.abs(A).sum(axis=1) + 1)
                cases.append(A)
    assert len(cases) == 63 + 343
    for A in cases:
        n = A.shape[0]
        Lu, D = _rational_ldl(A)
        Lexp = np.array([[float(Lu[i][j]) * np.sqrt(float(D[j])) for j in range(n)] for i in range(n)])
        Lh, info = dense.cholesky(A.astype(float))
        assert info == 0
        np.testing.assert_allclose(Lh, Lexp, rtol=4e-16 * n, atol=4e-16 * n * np.abs(Lexp).max())


@pytest.mark.parametrize("n", [1, 17, 64, 129, 300])
def test_recovers_known_factor(n):
    L = known_factor(n, seed_for(90, n))
    A = L @ L.T
    Lh, info = dense.cholesky(A)
    assert info == 0
    cond = np.linalg.cond(L)
    assert dense.factor_error(Lh, L) <= 1e-15 * cond * max(1, n) ** 0.5 + 1e-15


@pytest.mark.parametrize("n", [5, 40])
def test_recovers_integer_factor(n):
    L = known_factor(n, seed_for(91, n), integer=True)
    A = L @ L.T                      # integer entries, exact in float64
    assert np.all(A == np.round(A))
    Lh, info = dense.cholesky(A)
    assert info == 0
    np.testing.assert_allclose(Lh, L, rtol=0, atol=1e-10)


@pytest.mark.parametrize("n,rho", [(100, 1.0), (257, 1.05), (500, 2.0)])
def test_backward_error_invariant(n, rho):
    A = dominant_spd(n, rho, seed_for(0, n), shift=1.0)
    Lh, info = dense.cholesky(A)
    assert info == 0
    assert dense.backward_error(A, Lh) <= 1e-13


def test_special_cases():
    # identity
    Lh, _ = dense.cholesky(np.eye(9))
    assert np.array_equal(Lh, np.eye(9))
    # diagonal -> sqrt
    d = np.array([4.0, 9.0, 0.25, 2.0])
    Lh, _ = dense.cholesky(np.diag(d))
    assert np.array_equal(np.diag(Lh), np.sqrt(d)) and np.count_nonzero(np.tril(Lh, -1)) == 0
    # 1x1
    Lh, _ = dense.cholesky(np.array([[6.25]]))
    assert Lh[0, 0] == 2.5
    # block diagonal factors per block
    A1 = dominant_spd(20, 1.0, 11, shift=1.0)
    A2 = dominant_spd(13, 2.0, 12)
    A = np.zeros((33, 33))
    A[:20, :20] = A1
    A[20:, 20:] = A2
    Lh, _ = dense.cholesky(A)
    # equal up to the summation order of the (zero-padded) dot products
    np.testing.assert_allclose(Lh[:20, :20], dense.cholesky(A1)[0], rtol=1e-15, atol=1e-16)
    np.testing.assert_allclose(Lh[20:, 20:], dense.cholesky(A2)[0], rtol=1e-15, atol=1e-16)
    assert np.count_nonzero(Lh[20:, :20]) == 0


@pytest.mark.parametrize("k", [-3, 1, 5])
def test_scaling_by_powers_of_four_is_exact(k):
    A = dominant_spd(64, 1.05, 21)
    L1, _ = dense.cholesky(A)
    L2, _ = dense.cholesky(A * 4.0 ** k)
    assert np.array_equal(L2, L1 * 2.0 ** k)


def test_not_spd_reports_first_failing_column():
    A = dominant_spd(10, 2.0, 31)
    A[6, 6] = -1.0
    _, info = dense.cholesky(A)
    # the pivot at column 7 (1-based) is a66 - sum l6k^2 < 0 since a66 < 0
    assert info == 7
    A = dominant_spd(10, 2.0, 31)
    A[3, 3] = np.nan
    _, info = dense.cholesky(A)
    assert info == 4
    # exactly singular 2x2: pivot 2 is 1 - 1 = 0
    _, info = dense.cholesky(np.array([[1.0, 1.0], [1.0, 1.0]]))
    assert info == 2


def test_trsm_recovers_known_solution():
    L = known_factor(60, 5)
    X = np.random.default_rng(3).standard_normal((25, 60))
    B = X @ L.T
    Xh = dense.trsm_rlt(B, L)
    assert np.max(np.abs(Xh - X)) <= 1e-12 * np.abs(X).max()


@pytest.mark.parametrize("n,nrhs", [(50, 1), (200, 4)])
def test_solve_forward_error_bound(n, nrhs):
    A = dominant_spd(n, 1.0, seed_for(0, 1), shift=1.0)
    Xt = rhs(n, nrhs, 77)
    B = A @ Xt
    L, _ = dense.cholesky(A)
    Xh = dense.potrs(L, B)
    kappa = np.linalg.cond(A)
    err = np.linalg.norm(Xh - Xt) / np.linalg.norm(Xt)
    assert err <= 10 * n * 2.0 ** -53 * kappa
    # the two triangular halves separately
    Y = dense.forward_solve(L, B)
    np.testing.assert_allclose(L @ Y, B, rtol=0, atol=1e-12 * np.abs(B).max())
    Z = dense.backward_solve_t(L, Y)
    np.testing.assert_allclose(L.T @ Z, Y, rtol=0, atol=1e-12 * np.abs(Y).max())


def test_error_measures_on_known_perturbation():
    L = known_factor(30, 8)
    A = L @ L.T
    assert dense.backward_error(A, L) <= 1e-15
    E = np.zeros_like(L)
    E[5, 2] = 1e-3
    # ||A - (L+E)(L+E)^T||_F with a single perturbed entry, worked out from the product
    Lp = L + E
    direct = np.linalg.norm(A - Lp @ Lp.T) / np.linalg.norm(A)
    assert abs(dense.backward_error(A, Lp) - direct) <= 1e-15
    assert abs(dense.factor_error(Lp, L) - 1e-3 / np.linalg.norm(L)) <= 1e-15
