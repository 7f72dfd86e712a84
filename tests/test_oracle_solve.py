"""Pins of the refinement oracle (oracle/solve.py, POSV with FP64 iterative refinement).

Closed form: with the factor scaled uniformly, L_hat = c L (A = L L^T exactly), every
correction solves with (c^2 A)^{-1}, so the error and the residual shrink by exactly
q = 1 - 1/c^2 per step: after k corrections r_k = q^{k+1} b.  That fixes the iteration count
at the first k with |q|^{k+1} <= tol, and non-convergence when |q| >= 1.
"""
import math

import numpy as np
import pytest

from oracle import dense, solve
from synth import dominant_spd, seed_for


def _diag_case(n=6):
    d = np.array([1.0, 4.0, 9.0, 0.25, 16.0, 2.25])[:n]   # exact square roots
    return np.diag(d), np.diag(np.sqrt(d)), np.arange(1.0, n + 1.0)[:, None]


@pytest.mark.parametrize("c", [1.01, 1.1, 0.95, 1.3])
def test_uniformly_scaled_factor_contracts_by_the_closed_form(c):
    A, L, b = _diag_case()
    q = 1.0 - 1.0 / c ** 2
    tol = 1e-12
    k_expected = max(0, math.ceil(math.log(tol) / math.log(abs(q))) - 1)
    X, its, res, ok = solve.posv_ir(A, c * L, b, tol=tol, max_iter=60)
    assert ok and its == k_expected, (its, k_expected)
    # the residual after k corrections is |q|^(k+1) up to rounding
    assert res == pytest.approx(abs(q) ** (its + 1), rel=1e-6, abs=1e-16)
    np.testing.assert_allclose(X[:, 0], b[:, 0] / np.diag(A), rtol=1e-11)


def test_exact_factor_needs_no_correction():
    A = dominant_spd(80, 2.0, seed_for(12, 1))
    L, info = dense.cholesky(A)
    assert info == 0
    B = np.random.default_rng(seed_for(12, 2)).standard_normal((80, 3))
    X, its, res, ok = solve.posv_ir(A, L, B, tol=1e-12)
    assert ok and its == 0 and res <= 1e-12
    np.testing.assert_array_equal(X, dense.potrs(L, B))


def test_fp16_rounded_factor_refines_to_the_true_solution():
    # a low-precision factor (every entry of L rounded to binary16): the refinement reaches the
    # FP64 solution; forward error within 10 n u kappa of a known x
    n = 120
    A = dominant_spd(n, 1.5, seed_for(12, 3))
    L, _ = dense.cholesky(A)
    L16 = L.astype(np.float16).astype(np.float64)
    x_true = np.random.default_rng(seed_for(12, 4)).standard_normal((n, 2))
    B = A @ x_true
    X, its, res, ok = solve.posv_ir(A, L16, B, tol=1e-12)
    assert ok and 1 <= its <= 10 and res <= 1e-12
    kappa = np.linalg.cond(A)
    err = np.linalg.norm(X - x_true) / np.linalg.norm(x_true)
    assert err <= 10 * n * np.finfo(np.float64).eps * kappa


def test_a_factor_too_far_off_does_not_converge():
    A, L, b = _diag_case()
    X, its, res, ok = solve.posv_ir(A, 0.5 * L, b, tol=1e-12, max_iter=7)   # q = -3
    assert not ok and its == 7
    assert res == pytest.approx(3.0 ** 8, rel=1e-9)


# ---------------------------------------------------------------------------------------
# GMRES and GMRES-IR (oracle/solve.py: gmres, posv_gmres_ir)
# ---------------------------------------------------------------------------------------
def test_gmres_iterate_is_the_minimal_residual_point_of_the_krylov_space():
    """After k steps, GMRES returns argmin over K_k(M^-1 A, M^-1 r) of ||M^-1 (r - A d)||:
    computed here directly, by least squares on an orthonormal basis of the Krylov space."""
    n = 40
    A = dominant_spd(n, 1.1, seed_for(6, 50), shift=1.0)
    L = np.linalg.cholesky(A + 0.3 * np.diag(np.diag(A)))          # an inexact factor
    r = np.random.default_rng(1).standard_normal(n)
    Minv = lambda v: dense.potrs(L, v)
    As = dense.sym_from_lower(A)
    for k in (1, 3, 6):
        d, steps = solve.gmres(lambda v: As @ v, Minv, r, restart=k, inner_tol=0.0)
        assert steps == k
        K = [Minv(r)]
        for _ in range(k - 1):
            K.append(Minv(As @ K[-1]))
        Q, _ = np.linalg.qr(np.array(K).T)
        MA_Q = np.array([Minv(As @ Q[:, j]) for j in range(k)]).T
        y, *_ = np.linalg.lstsq(MA_Q, Minv(r), rcond=None)
        d_ref = Q @ y
        assert np.linalg.norm(d - d_ref) <= 1e-10 * np.linalg.norm(d_ref)


def test_gmres_terminates_within_n_steps():
    n = 12
    A = dominant_spd(n, 1.2, seed_for(6, 51), shift=1.0)
    As = dense.sym_from_lower(A)
    r = np.arange(1.0, n + 1.0)
    d, steps = solve.gmres(lambda v: As @ v, lambda v: v, r, restart=n, inner_tol=1e-14)
    assert steps <= n
    assert np.linalg.norm(As @ d - r) <= 1e-11 * np.linalg.norm(r)


def test_gmres_ir_with_the_exact_factor_needs_no_correction_or_one():
    n = 200
    A = dominant_spd(n, 2.0, seed_for(6, 52))
    L, _ = dense.cholesky(A)
    b = np.random.default_rng(2).standard_normal(n)
    X, its, steps, res, ok = solve.posv_gmres_ir(A, L, b)
    assert ok and its <= 1 and res <= 1e-12


def test_gmres_ir_converges_where_plain_refinement_does_not():
    """A Gram matrix with kappa ~ 1e4 and a factor carrying relative perturbations of 1e-2:
    each plain correction multiplies the error by about kappa * 1e-2 > 1 and refinement
    diverges, while GMRES preconditioned by the same factor converges in two corrections
    (Carson and Higham).  kappa stays small enough that u kappa is below the 1e-12 target."""
    n = 300
    from synth import gram_spd
    A = gram_spd(n, 6e-4, seed_for(6, 53))
    L, info = dense.cholesky(A)
    assert info == 0
    rng = np.random.default_rng(3)
    Lp = L * (1.0 + 1e-2 * rng.standard_normal(L.shape))
    b = rng.standard_normal(n)
    _, _, res_ir, ok_ir = solve.posv_ir(A, Lp, b, tol=1e-12, max_iter=10)
    X, its, steps, res, ok = solve.posv_gmres_ir(A, Lp, b, tol=1e-12, max_iter=10, restart=30, inner_tol=1e-8)
    assert not ok_ir and res_ir > 1.0 and ok and its <= 3, (res_ir, res, its)
    assert np.linalg.norm(dense.sym_from_lower(A) @ X[:, 0] - b) <= 1e-12 * np.linalg.norm(b)
