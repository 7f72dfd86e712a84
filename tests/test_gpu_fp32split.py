"""FP32 levels on tensor cores by the error-corrected TF32 split (hrp_set_fp32_split).

The oracle's split product (lowprec.gemm_tf32x3: hi hi^T + hi lo^T + lo hi^T of the TF32
splits, summed exactly) differs from the GPU's only by the FP32 accumulation of the two
tcgen05 accumulators, so:

* standalone Alg. 3 with an [F32] list: the GPU result lies within the FP32 error bound
  gamma_k |A||A|^T plus the split's 3 2^-22 |A||A|^T of the exact product of the FP32
  operands; its median distance to the oracle's split product is below 2^-22 |A||A|^T,
  which neither plain TF32 (hi hi^T alone) nor a split missing one correction term reaches
  (the tensor core accumulates toward zero, so same-sign sums, such as the diagonal, drift
  by up to one FP32 ulp per K = 8 instruction);
* the factorization with FP32 levels on tensor cores carries the tree's precisions (the
  mixed-tree check against the emulator with split FP32 levels) and an FP32-level backward
  error, and its solves refine to 1e-12;
* the tensor-core class actually ran (per-class launch counts).
"""
import numpy as np
import pytest

from oracle import dense, lowprec, tree as otree
from synth import dominant_spd, normals, rhs, seed_for

from mixed_check import check_mixed_factor

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def env():
    import torch

    import paper_2601_08082_gb300 as hrp
    h = hrp.Handle(0)
    h.set_fp32_split(True)
    h0 = hrp.Handle(0)
    yield hrp, h, h0, torch
    h.close()
    h0.close()


def _syrk(hrp, h, spec, leaf, A, C):
    n, k = A.shape
    At = hrp.colmajor(A).cuda()
    Ct = hrp.colmajor(C).cuda()
    h.syrk(hrp.tree_parse(spec, leaf), At, Ct)
    return np.tril(hrp.from_colmajor(Ct))


@pytest.mark.parametrize("n,k", [(1024, 512), (700, 333), (2048, 96), (4096, 256)])
def test_split_syrk_is_fp32_accurate_and_matches_the_split_oracle(env, n, k):
    hrp, h, h0, torch = env
    A = normals(seed_for(13, n), 0, np.arange(n * k, dtype=np.uint64)).reshape(n, k)
    C = np.zeros((n, n))
    got = _syrk(hrp, h, "[F32]", 128, A, C)
    A32 = lowprec.round_f32(A)
    exact = np.tril(-(A32 @ A32.T))
    mag = np.tril(np.abs(A32) @ np.abs(A32).T)
    low = np.tril(np.ones((n, n), bool))
    gamma = k * U32 / (1 - k * U32)
    assert np.all(np.abs(got - exact)[low] <= ((gamma + 3.01 * 2.0 ** -22) * mag)[low])
    # The tensor core accumulates toward zero: sums of same-sign terms (the diagonal) drift by
    # up to one FP32 ulp per K = 8 instruction, inside the bound above.  Elsewhere the GPU
    # sits on the split product, which a dropped correction term moves off by orders of
    # magnitude at almost every entry.
    split = otree.emulate_syrk(C, A, otree.parse("[F32]", leaf=128), f32_split=True)
    rel = np.abs(got - split)[low] / mag[low]
    assert np.median(rel) <= 2.0 ** -22, np.median(rel)
    assert rel.max() <= (k / 8 + 2) * 2.0 ** -23, rel.max()
    hx, lx = lowprec.split_tf32(A)
    for wrong in (hx @ hx.T, hx @ hx.T + hx @ lx.T):
        assert np.median(np.abs(np.tril(-wrong) - split)[low] / mag[low]) > 2.0 ** -19
    # the SIMT FP32 path meets the same FP32 bound
    simt = _syrk(hrp, h0, "[F32]", 128, A, C)
    assert np.all(np.abs(simt - exact)[low] <= (gamma * mag)[low])


def test_split_factor_runs_on_tensor_cores(env):
    hrp, h, h0, torch = env
    n = 2048
    A = dominant_spd(n, 1.5, seed_for(13, 1))
    tree = hrp.tree_parse("[F32|F64@128]", 128)        # no F16 level: every tcgen05 GEMM is a split
    tc = h.timing(tree, hrp.colmajor(A).cuda())
    simt = h0.timing(tree, hrp.colmajor(A).cuda())
    assert tc["gemm_f16_tcgen05"]["launches"] > 0, tc
    assert simt["gemm_f16_tcgen05"]["launches"] == 0, simt
    assert tc["gemm_simt"]["flops"] < 0.1 * simt["gemm_simt"]["flops"], (tc, simt)


@pytest.mark.parametrize("spec,n", [("[F32|F64@128]", 2048), ("[F16,F32|F64@128]", 2048),
                                    ("[F16,F16,F32|F64@128]", 4096)])
def test_split_factor_carries_the_tree_and_solves(env, spec, n):
    hrp, h, h0, torch = env
    A = dominant_spd(n, 1.5, seed_for(13, 100 + n))
    At = hrp.colmajor(A).cuda()
    assert h.potrf(hrp.tree_parse(spec, 128), At) == 0
    L = np.tril(hrp.from_colmajor(At))
    t = otree.parse(spec, leaf=128)
    L_emu, info, _ = otree.emulate_potrf(A, t, f32_split=True)
    assert info == 0
    check_mixed_factor(L, A, spec, 128, L_emu=L_emu)
    be = dense.backward_error(A, L)
    assert be <= 2 * dense.backward_error(A, L_emu) + 1e-7
    A0 = hrp.colmajor(A).cuda()
    assert h0.potrf(hrp.tree_parse(spec, 128), A0) == 0
    L0 = np.tril(hrp.from_colmajor(A0))
    assert not np.array_equal(L, L0)          # the split path ran
    B = rhs(n, 2, seed_for(13, 200 + n))
    A_t, B_t = hrp.colmajor(A).cuda(), hrp.colmajor(B).cuda()
    X_t = torch.zeros_like(B_t)
    out = h.posv(hrp.tree_parse(spec, 128), A_t, B_t, X_t, tol=1e-12)
    assert out["status"] == 0 and out["used_fallback"] == 0, out
    assert np.max(dense.column_residuals(A, hrp.from_colmajor(X_t), B)) <= 1e-12
