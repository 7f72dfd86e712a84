"""GMRES-IR in hrp_posv (hrp_set_refinement mode 1) against the oracle's GMRES-IR.

Gram matrices A = G G^T / k + alpha I (kappa ~ 5.8 / alpha) with an FP16 tree: the FP16
factor's backward error (~1.6e-4) times kappa decides whether classical refinement
converges.  At alpha = 5e-4 (kappa ~ 1.2e4) it diverges in the oracle, and hrp_posv falls
back to the FP32 tree; GMRES preconditioned by the same FP16 factor converges (Carson and
Higham) to the tolerance 1e-11 (u kappa bounds what any FP64 residual can show).  At
alpha = 1e-3 both converge, GMRES-IR in a few corrections where the classical loop needs
many.
"""
import numpy as np
import pytest

from oracle import dense, solve, tree as otree
from synth import gram_spd, rhs, seed_for

pytestmark = pytest.mark.gpu

SPEC = "[F16,F32|F64@128]"


@pytest.fixture(scope="module")
def env():
    import torch

    import paper_2601_08082_gb300 as hrp
    h = hrp.Handle(0)
    yield hrp, h, torch
    h.set_refinement(False)
    h.close()


def _posv(hrp, h, torch, A, B, gmres, tol):
    h.set_refinement(gmres, restart=20, inner_tol=1e-8)
    A_t = hrp.colmajor(A).cuda()
    B_t = hrp.colmajor(B).cuda()
    X_t = torch.zeros_like(B_t)
    out = h.posv(hrp.tree_parse(SPEC, 128), A_t, B_t, X_t, max_iter=30, tol=tol)
    out["inner"] = h.inner_iterations()
    return out, hrp.from_colmajor(X_t)


def test_gmres_ir_converges_where_classical_refinement_falls_back(env):
    hrp, h, torch = env
    n = 1024
    A = gram_spd(n, 5e-4, seed_for(6, 60))
    B = rhs(n, 2, seed_for(6, 61))
    L_emu, info, _ = otree.emulate_potrf(A, otree.parse(SPEC, leaf=128))
    assert info == 0
    _, _, res_ir, ok_ir = solve.posv_ir(A, L_emu, B, tol=1e-11, max_iter=30)
    _, _, _, res_g, ok_g = solve.posv_gmres_ir(A, L_emu, B, tol=1e-11, max_iter=30, restart=20, inner_tol=1e-8)
    assert not ok_ir and ok_g, (res_ir, res_g)
    out0, X0 = _posv(hrp, h, torch, A, B, False, 1e-11)
    assert out0["status"] == 0 and out0["used_fallback"] == 1 and out0["inner"] == 0
    out1, X1 = _posv(hrp, h, torch, A, B, True, 1e-11)
    assert out1["status"] == 0 and out1["used_fallback"] == 0 and out1["inner"] > 0, out1
    assert np.max(dense.column_residuals(A, X1, B)) <= 1e-11
    assert np.max(dense.column_residuals(A, X0, B)) <= 1e-11


def test_gmres_ir_needs_fewer_corrections(env):
    hrp, h, torch = env
    n = 1024
    A = gram_spd(n, 1e-3, seed_for(6, 62))
    B = rhs(n, 1, seed_for(6, 63))
    out0, X0 = _posv(hrp, h, torch, A, B, False, 1e-12)
    out1, X1 = _posv(hrp, h, torch, A, B, True, 1e-12)
    assert out0["status"] == 0 and out1["status"] == 0
    assert out1["used_fallback"] == 0 and out1["iters"] <= 4 and out1["iters"] < out0["iters"], (out0, out1)
    assert np.max(dense.column_residuals(A, X1, B)) <= 1e-12


def test_refinement_arguments(env):
    hrp, h, torch = env
    with pytest.raises(hrp.HrpError):
        h.set_refinement(True, restart=0)
    with pytest.raises(hrp.HrpError):
        h.set_refinement(True, restart=20, inner_tol=1.5)
    h.set_refinement(False)
