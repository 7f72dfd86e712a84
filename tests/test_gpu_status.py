"""Device-side status, range and replay behaviour of the GPU path (through the C ABI).

* Bounded waits: a kernel waits on a mailbox entry that nothing fills with a short limit; the wait
  expires, the status word records it and the call returns HRP_ERR_TIMEOUT with the
  context still usable.  Solves run with a 1 us limit either finish or report the
  timeout with NaN rows (never a plausible wrong answer).
* Sec. 3.4 scaling: alpha = max(1, amax / 65504) is 1 on every FP16 operand the GPU
  handles; an operand beyond 65504 is reported as HRP_ERR_RANGE, and hrp_posv refactors
  with the FP32 fallback tree.  The emulator applies the general rule to the same input.
* Graph replay: factor + solve captured once and replayed must solve every system every
  time (the solve's kernels empty their mailboxes themselves, in stream order).
* Policy file and policy-chosen trees in the batched calls.
"""
import os

import numpy as np
import pytest

from oracle import dense, lowprec, tree as otree
from synth import dominant_spd, rhs, seed_for

pytestmark = pytest.mark.gpu

WEIGHTS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2601_08082_gb300",
                       "policy_weights.json")


@pytest.fixture(scope="module")
def env():
    import torch

    import paper_2601_08082_gb300 as hrp
    h = hrp.Handle(0)
    yield hrp, h, torch
    h.close()


def test_bounded_wait_expires_and_the_context_stays_usable(env):
    hrp, h, torch = env
    st, waited = h.wait_selftest(2000)
    assert hrp.STATUS[st] == "HRP_ERR_TIMEOUT"
    assert 2000 <= waited < 1e6, waited
    assert h.check() == 0                       # the status word was cleared
    A = dominant_spd(300, 2.0, seed_for(7, 1))
    At = hrp.colmajor(A).cuda()
    assert h.potrf(hrp.tree_parse("[F16,F32|F64@64]", 64), At) == 0
    L0, _ = dense.cholesky(A)
    assert dense.factor_error(np.tril(hrp.from_colmajor(At)), L0) < 1e-6


def test_solve_with_a_tiny_wait_limit_is_correct_or_reports_nan(env):
    hrp, h, torch = env
    n = 4096
    A = dominant_spd(n, 2.0, seed_for(7, 2))
    L0, _ = dense.cholesky(A)
    B = rhs(n, 1, seed_for(7, 3))
    X0 = dense.potrs(L0, B)
    Lt = hrp.colmajor(L0).cuda()
    try:
        h.set_wait_limit(1)
        for _ in range(3):
            Bt = hrp.colmajor(B).cuda()
            h.potrs(Lt, Bt)
            st = h.check()
            X = hrp.from_colmajor(Bt)
            if st == 0:
                assert np.max(np.abs(X - X0)) <= 1e-12 * np.max(np.abs(X0))
            else:
                assert hrp.STATUS[st] == "HRP_ERR_TIMEOUT"
                assert np.all(np.isnan(X[:64]))        # x_0 depends on every block
    finally:
        h.set_wait_limit(2000000)
    Bt = hrp.colmajor(B).cuda()
    h.potrs(Lt, Bt)
    assert h.check() == 0
    assert np.max(np.abs(hrp.from_colmajor(Bt) - X0)) <= 1e-12 * np.max(np.abs(X0))


def test_fp16_operand_beyond_65504_is_a_range_error(env):
    hrp, h, torch = env
    import torch as _t
    n = 640
    A = dominant_spd(n, 2.0, seed_for(7, 4)) * 1e15            # |l_ij| ~ 1e6 > 65504
    spec, leaf = "[F16,F32|F64@128]", 128
    # the paper's rule on the CPU: alpha > 1 on the FP16 operands, and the factor is fine
    L_emu, info, em = otree.emulate_potrf(A, otree.parse(spec, leaf=leaf))
    assert info == 0 and dense.backward_error(A, L_emu) < 5e-5
    n1 = otree.split(n)
    assert lowprec.quantize_f16(L_emu[n1:, :n1])[1] > 1.0
    # the GPU (alpha = 1 on its FP16 path) refuses it
    At = hrp.colmajor(A).cuda()
    with pytest.raises(hrp.HrpError) as e:
        h.potrf(hrp.tree_parse(spec, leaf), At)
    assert hrp.STATUS[e.value.status] == "HRP_ERR_RANGE"
    assert h.check() == 0
    # an FP32 tree factors it, and hrp_posv falls back to one by itself
    At = hrp.colmajor(A).cuda()
    assert h.potrf(hrp.tree_parse("[F32|F64@128]", leaf), At) == 0
    B = rhs(n, 2, seed_for(7, 5))
    A_t = hrp.colmajor(A).cuda()
    B_t = hrp.colmajor(B).cuda()
    X_t = _t.zeros_like(B_t)
    out = h.posv(hrp.tree_parse(spec, leaf), A_t, B_t, X_t, tol=1e-12)
    assert out["status"] == 0 and out["used_fallback"] == 1
    assert np.max(dense.column_residuals(A, hrp.from_colmajor(X_t), B)) <= 1e-12
    # the same matrix scaled into range is accepted by the FP16 tree
    At = hrp.colmajor(A * 1e-15).cuda()
    assert h.potrf(hrp.tree_parse(spec, leaf), At) == 0


def test_factor_and_solve_replayed_from_one_graph(env):
    hrp, h, torch = env
    sizes = [256, 384, 128, 640, 1000]
    mats = [dominant_spd(n, 2.0, seed_for(7, 10 + i)) for i, n in enumerate(sizes)]
    rhss = [rhs(n, 3, seed_for(7, 20 + i)) for i, n in enumerate(sizes)]
    tree = hrp.tree_parse("[F16,F32|F64@128]", leaf=128)
    A0 = [hrp.colmajor(A).cuda() for A in mats]
    B0 = [hrp.colmajor(B).cuda() for B in rhss]
    As = [A.clone() for A in A0]
    Bs = [B.clone() for B in B0]
    d_info = torch.zeros(len(sizes), dtype=torch.int32, device="cuda")
    h.potrf_batched(tree, As, d_info)              # workspace, outside the capture
    h.potrs_batched(As, Bs)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            h.potrf_batched(tree, As, d_info, stream=s)
            h.potrs_batched(As, Bs, stream=s)
    for rep in range(3):
        for A, a0 in zip(As, A0):
            A.copy_(a0)
        for B, b0 in zip(Bs, B0):
            B.copy_(b0)
        g.replay()
        torch.cuda.synchronize()
        assert d_info.cpu().tolist() == [0] * len(sizes)
        for At, Bt, B in zip(As, Bs, rhss):
            L = np.tril(hrp.from_colmajor(At))
            X_ref = dense.potrs(L, B)
            X = hrp.from_colmajor(Bt)
            assert np.max(np.abs(X - X_ref)) <= 1e-12 * np.max(np.abs(X_ref)), rep
    assert h.check() == 0


def test_policy_file_and_policy_chosen_batched_trees(env):
    hrp, h, torch = env
    import json
    h2 = hrp.Handle(0)
    try:
        h2.policy_load(WEIGHTS)
        w = json.load(open(WEIGHTS))
        h.policy_set(np.array(w["params"], np.float32), np.array(w["mean"], np.float32),
                     np.array(w["scale"], np.float32))
        sizes = [300, 512, 1024]
        mats = [dominant_spd(n, r, seed_for(7, 30 + i)) for i, (n, r) in enumerate(zip(sizes, [8.0, 1.05, 2.0]))]
        for A in mats:
            feat = h2.policy_features(hrp.colmajor(A).cuda())
            t2, k2 = h2.policy_predict_tree(feat)
            t1, k1 = h.policy_predict_tree(feat)
            assert k1 == k2 and hrp.tree_format(t2) == hrp.tree_format(hrp.policy_tree(k2))
        As = [hrp.colmajor(A).cuda() for A in mats]
        Bs = [hrp.colmajor(rhs(n, 2, seed_for(7, 40 + i))).cuda() for i, n in enumerate(sizes)]
        Xs = [torch.zeros_like(B) for B in Bs]
        out = h2.posv_batched(None, As, Bs, Xs, tol=1e-12)
        assert out["status"] == 0
        for A, B, X in zip(mats, Bs, Xs):
            assert np.max(dense.column_residuals(A, hrp.from_colmajor(X), hrp.from_colmajor(B))) <= 1e-12
        d_info = torch.zeros(len(sizes), dtype=torch.int32, device="cuda")
        Ac = [hrp.colmajor(A).cuda() for A in mats]
        h2.potrf_batched([None, hrp.tree_parse("[F64]", 64), None], Ac, d_info)
        torch.cuda.synchronize()
        assert d_info.cpu().tolist() == [0, 0, 0]
        L0, _ = dense.cholesky(mats[1])
        assert np.max(np.abs(np.tril(hrp.from_colmajor(Ac[1])) - L0)) <= 1e-12 * np.max(np.abs(L0))
    finally:
        h2.close()


def test_policy_load_rejects_a_wrong_file(env, tmp_path):
    hrp, h, torch = env
    p = tmp_path / "bad.json"
    p.write_text('{"format": "hrp-policy-v1", "trees": ["[F64]"], "params": [1, 2], "mean": [], "scale": []}')
    with pytest.raises(hrp.HrpError):
        h.policy_load(str(p))
    with pytest.raises(hrp.HrpError):
        h.policy_load(str(tmp_path / "missing.json"))
