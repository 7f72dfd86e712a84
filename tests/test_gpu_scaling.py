"""Dynamic quantization on the GPU: two-sided power-of-two diagonal scaling before the
recursion (hrp_set_scaling mode 1), the remedy the paper names for matrices of extreme
dynamic range (Sec. 4.5, 5).

* The GPU's exponents and scalings are those of the oracle: the scaled factor of A, divided
  row by row by 2^e_i, equals the unscaled factor of A_hat = D^-1 A D^-1 formed on the host.
* With an FP64 tree the scaling is exact: the factor equals the plain FP64 Cholesky factor.
* On a 24-decade matrix the static path refuses the FP16 operands (HRP_ERR_RANGE; the
  emulator's static rule loses definiteness there), while the scaled factor carries the
  tree's precisions on A_hat and reaches the emulator's scaled backward error.
* hrp_posv with scaling solves the same systems on the FP16 tree without the fallback.
"""
import numpy as np
import pytest

from oracle import dense, solve, tree as otree
from synth import dominant_spd, rhs, seed_for, wide_range_spd

from mixed_check import check_mixed_factor

pytestmark = pytest.mark.gpu

SPEC, LEAF = "[F16,F16,F32|F64@128]", 128


@pytest.fixture(scope="module")
def env():
    import torch

    import paper_2601_08082_gb300 as hrp
    h = hrp.Handle(0)
    hs = hrp.Handle(0)
    hs.set_scaling(True)
    yield hrp, h, hs, torch
    h.close()
    hs.close()


def _scaled(A):
    e = otree.diagonal_scale_exponents(A)
    return e, np.ldexp(np.ldexp(A, -e[:, None]), -e[None, :])


def _factor(hrp, h, A, spec=SPEC, leaf=LEAF):
    At = hrp.colmajor(A).cuda()
    info = h.potrf(hrp.tree_parse(spec, leaf), At)
    return info, np.tril(hrp.from_colmajor(At))


@pytest.mark.parametrize("n", [640, 1024])
def test_scaled_factor_is_the_factor_of_the_scaled_matrix(env, n):
    hrp, h, hs, torch = env
    A = wide_range_spd(n, 12, seed_for(12, n), core="dominant")
    e, Ah = _scaled(A)
    info_s, L = _factor(hrp, hs, A)
    info_h, Lh = _factor(hrp, h, Ah)
    assert info_s == info_h == 0
    Lhat = np.ldexp(L, -e[:, None])
    assert np.max(np.abs(Lhat - Lh)) <= 1e-13 * np.max(np.abs(Lh))
    assert hs.check() == 0


def test_scaling_with_an_fp64_tree_is_exact(env):
    hrp, h, hs, torch = env
    n = 768
    A = wide_range_spd(n, 24, seed_for(12, 3), core="dominant")
    info, L = _factor(hrp, hs, A, "[F64]", 64)
    assert info == 0
    L0, _ = dense.cholesky(A)
    # row i of both factors carries the scale 2^e_i: compare row-relative
    r = np.max(np.abs(L - L0), axis=1) / np.max(np.abs(L0), axis=1)
    assert np.max(r) <= 1e-13


def test_extreme_range_static_refuses_and_scaled_factors(env):
    hrp, h, hs, torch = env
    n = 512
    A = wide_range_spd(n, 24, seed_for(10, 3), core="gram", alpha=1e-3)
    # the static rule (emulator, alpha per operand) loses definiteness on this matrix
    assert otree.emulate_potrf(A, otree.parse(SPEC, leaf=LEAF))[1] > 0
    At = hrp.colmajor(A).cuda()
    with pytest.raises(hrp.HrpError) as err:
        h.potrf(hrp.tree_parse(SPEC, LEAF), At)
    assert hrp.STATUS[err.value.status] == "HRP_ERR_RANGE"
    assert h.check() == 0
    info, L = _factor(hrp, hs, A)
    assert info == 0
    e, Ah = _scaled(A)
    L_emu, info_e, _ = otree.emulate_potrf_scaled(A, otree.parse(SPEC, leaf=LEAF))
    assert info_e == 0
    check_mixed_factor(np.ldexp(L, -e[:, None]), Ah, SPEC, LEAF, L_emu=np.ldexp(L_emu, -e[:, None]))
    assert dense.scaled_backward_error(A, L) <= 2 * dense.scaled_backward_error(A, L_emu)


@pytest.mark.parametrize("core", ["dominant", "gram"])
def test_posv_with_scaling_needs_no_fallback(env, core):
    hrp, h, hs, torch = env
    n = 1024
    kw = {"alpha": 1e-3} if core == "gram" else {}
    A = wide_range_spd(n, 24, seed_for(11, 1), core=core, **kw)
    e, _ = _scaled(A)
    z = rhs(n, 2, seed_for(11, 2))
    B = dense.sym_from_lower(A) @ np.ldexp(z, -e[:, None])     # a solution in the unknowns' units
    L_emu, _, _ = otree.emulate_potrf_scaled(A, otree.parse(SPEC, leaf=LEAF))
    its_emu = solve.posv_ir(A, L_emu, B, tol=1e-12)[1]
    for handle, fallback in ((h, 1), (hs, 0)):
        A_t = hrp.colmajor(A).cuda()
        B_t = hrp.colmajor(B).cuda()
        X_t = torch.zeros_like(B_t)
        out = handle.posv(hrp.tree_parse(SPEC, LEAF), A_t, B_t, X_t, tol=1e-12)
        assert out["status"] == 0 and out["used_fallback"] == fallback, out
        assert np.max(dense.column_residuals(A, hrp.from_colmajor(X_t), B)) <= 1e-12
        if fallback == 0:
            assert out["iters"] <= 2 * its_emu + 3, (out, its_emu)


def test_scaling_leaves_a_well_scaled_matrix_alone(env):
    hrp, h, hs, torch = env
    n = 640
    C = dominant_spd(n, 2.0, seed_for(12, 9))
    s = 1 / np.sqrt(np.diag(C))
    C1 = C * s[:, None] * s[None, :]
    assert not otree.diagonal_scale_exponents(C1).any()
    _, L1 = _factor(hrp, hs, C1)
    _, L0 = _factor(hrp, h, C1)
    assert np.max(np.abs(L1 - L0)) <= 1e-13 * np.max(np.abs(L0))
