"""GPU parity of the standalone Tree-SYRK (Alg. 3) and Tree-TRSM (Alg. 2), and of the Pure F16
factorization, against the emulators of oracle/tree.py (through the C ABI).

* All-FP64 lists: 1e-12 relative to the plain definitions.
* SYRK, any list: GPU and emulator round the same operands (FP16 by round to nearest even,
  FP32); the emulator sums the exact products in float64, the GPU in FP32 with at most k
  roundings per entry, so entrywise |C_gpu - C_emu| <= 2 gamma_k(2^-24) (|A| |A|^T)
  (Higham, Sec. 3.1, inner products), doubled for the operands' own rounding.
* TRSM, lists with FP16 levels: the FP32 noise is far below the FP16 effect, so the GPU must
  be within 0.1 of the emulator's distance from the FP64 solve.  Lists whose only reduced
  precision is FP32: the GPU solve must meet the FP32 triangular-solve backward bound
  |X L^T - B| <= 3 gamma_n(2^-24) |X| |L|^T (Higham, Thm. 8.5; the factor 3 covers the GEMM
  splitting of Alg. 2).
* Every reduced list: the GPU result is at least 0.3x as far from the FP64 result as the
  emulator's (a reduced level run in FP64 would sit far closer).
"""

import numpy as np
import pytest

from mixed_check import check_mixed_factor
from oracle import dense, tree as otree
from synth import dominant_spd, seed_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    import paper_2601_08082_gb300 as hrp
    h = hrp.Handle(0)
    yield hrp, h, torch
    h.close()


def _gamma(k):
    u = 2.0 ** -24
    return k * u / (1 - k * u)


def _not_fp64(out, emu, f64, spec):
    g, e = np.linalg.norm(out - f64), np.linalg.norm(emu - f64)
    assert g >= 0.3 * e, (spec, g, e)


SPECS = ["[F64]", "[F32]", "[F16,F16,F32]", "[F16,F16,F16,F16,F32]", "[F16]", "[F16,F64]"]


@pytest.mark.parametrize("spec", SPECS)
@pytest.mark.parametrize("n,k", [(1000, 1000), (777, 333), (2048, 512)])
def test_syrk_matches_emulator(env, spec, n, k):
    hrp, h, torch = env
    rng = np.random.default_rng(seed_for(8, n + k))
    A = rng.standard_normal((n, k))
    C0 = rng.standard_normal((n, n))
    C0 = C0 + C0.T + 4.0 * np.eye(n)
    t = otree.parse(spec, leaf=128)
    At = hrp.colmajor(A).cuda()
    Ct = hrp.colmajor(C0).cuda()
    h.syrk(hrp.tree_parse(spec, leaf=128), At, Ct)
    assert h.check() == 0
    C = hrp.from_colmajor(Ct)
    assert np.array_equal(np.triu(C, 1), np.triu(C0, 1))          # strict upper untouched
    out = np.tril(C)
    emu = otree.emulate_syrk(C0, A, t)
    f64 = np.tril(C0 - A @ A.T)
    if spec == "[F64]":
        assert np.max(np.abs(out - f64)) <= 1e-12 * np.max(np.abs(f64))
        return
    bound = 2 * _gamma(k) * np.tril(np.abs(A) @ np.abs(A).T)
    assert np.all(np.abs(out - emu) <= bound), (spec, np.max(np.abs(out - emu) / np.maximum(bound, 1e-300)))
    _not_fp64(out, emu, f64, spec)


@pytest.mark.parametrize("spec", SPECS)
@pytest.mark.parametrize("m,n", [(1000, 1000), (300, 777), (2048, 1024)])
def test_trsm_matches_emulator(env, spec, m, n):
    hrp, h, torch = env
    L = np.tril(dense.cholesky(dominant_spd(n, 1.5, seed_for(8, 500 + n), shift=1.0))[0])
    B = np.random.default_rng(seed_for(8, 600 + m)).standard_normal((m, n))
    t = otree.parse(spec, leaf=128)
    Lt = hrp.colmajor(L).cuda()
    Bt = hrp.colmajor(B).cuda()
    h.trsm(hrp.tree_parse(spec, leaf=128), Lt, Bt)
    assert h.check() == 0
    X = hrp.from_colmajor(Bt)
    emu, f64 = otree.emulate_trsm(B, L, t), dense.trsm_rlt(B, L)
    if spec == "[F64]":
        assert np.max(np.abs(X - f64)) <= 1e-12 * np.max(np.abs(f64))
        return
    if "F16" in spec:
        d, e = np.linalg.norm(X - emu), np.linalg.norm(emu - f64)
        assert d <= 0.1 * e, (spec, d, e)
    else:
        bound = 3 * _gamma(n) * (np.abs(X) @ np.abs(L).T)
        assert np.all(np.abs(X @ L.T - B) <= bound)
    _not_fp64(X, emu, f64, spec)


def test_syrk_reports_an_fp16_operand_out_of_range(env):
    hrp, h, torch = env
    A = np.full((200, 64), 1e5)
    C = np.eye(200)
    h.syrk(hrp.tree_parse("[F16,F32]", leaf=128), hrp.colmajor(A).cuda(), hrp.colmajor(C).cuda())
    assert hrp.STATUS[h.check()] == "HRP_ERR_RANGE"
    h.syrk(hrp.tree_parse("[F32]", leaf=128), hrp.colmajor(A).cuda(), hrp.colmajor(C).cuda())
    assert h.check() == 0


@pytest.mark.parametrize("n,rho", [(1000, 2.0), (1536, 8.0)])
def test_pure_f16_factorization_matches_emulator(env, n, rho):
    """[F16]: every GEMM on FP16 operands and the diagonal leaves in FP32 on FP16-rounded
    input, rounded to FP16 (the reading of a leaf POTRF at an F16 level)."""
    hrp, h, torch = env
    A = dominant_spd(n, rho, seed_for(8, 900 + n))
    At = hrp.colmajor(A).cuda()
    assert h.potrf(hrp.tree_parse("[F16]", leaf=128), At) == 0
    L = np.tril(hrp.from_colmajor(At))
    L_emu, info, _ = otree.emulate_potrf(A, otree.parse("[F16]", leaf=128))
    assert info == 0
    check_mixed_factor(L, A, "[F16]", 128, L_emu=L_emu)
    be, be_emu = dense.backward_error(A, L), dense.backward_error(A, L_emu)
    assert abs(be - be_emu) <= 0.2 * be_emu
