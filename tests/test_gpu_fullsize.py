"""Parity at the full sizes `bench.py` times, in the same launch configuration (one
hrp_potrf / hrp_posv call on the whole matrix):

* n = 8192, tree [F16,F16,F16,F16,F32|F64@128], rho = 2 (the bench's second matrix): the
  whole factor against the step-by-step emulator of Alg. 1-3.
* n = 32768, tree [F8,F16,F16,F32|F64@128], the bench's device-drawn matrix: the emulator
  does not finish at this size, so the test checks what the oracle can compute piece by piece
  on the host: the first FP64 leaf block against the plain Cholesky, sampled rows of
  L L^T - A against the backward-error bound, and the refined solution's residual.
"""
import numpy as np
import pytest

from oracle import dense, tree as otree
from synth import dominant_spd, seed_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hrp_mod():
    import torch
    import paper_2601_08082_gb300 as hrp
    assert torch.cuda.is_available()
    return hrp


@pytest.fixture(scope="module")
def handle(hrp_mod):
    h = hrp_mod.Handle(0)
    yield h
    h.close()


def test_bench_tree_at_n8192_matches_emulator(hrp_mod, handle):
    n, spec = 8192, "[F16,F16,F16,F16,F32|F64@128]"
    A = dominant_spd(n, 2.0, seed_for(1, 1))
    At = hrp_mod.colmajor(A).cuda()
    assert handle.potrf(hrp_mod.tree_parse(spec, leaf=128), At) == 0
    L = np.tril(hrp_mod.from_colmajor(At))
    L_emu, info_e, _ = otree.emulate_potrf(A, otree.parse(spec, leaf=128))
    assert info_e == 0
    # FP32 accumulation (GPU) vs exact sums (emulator): the bound of the mixed-tree tests
    assert np.max(np.abs(L - L_emu)) <= 1e-5 * np.max(np.abs(L_emu))
    # same precision semantics: the backward errors agree (a level run in a higher or lower
    # precision than the tree says would move it by orders of magnitude)
    be_gpu, be_emu = dense.backward_error(A, L), dense.backward_error(A, L_emu)
    assert be_gpu <= 5e-5
    assert 0.5 * be_emu <= be_gpu <= 2.0 * be_emu, (be_gpu, be_emu)


def _zero_below_diagonal(S, blk=2048):
    """S (n x n, C order) holds a column-major lower factor, i.e. its transpose: keep the upper
    triangle of S in place (the strict lower part holds the untouched input)."""
    n = S.shape[0]
    for r0 in range(0, n, blk):
        r1 = min(n, r0 + blk)
        S[r0:r1, :r0] = 0.0
        S[r0:r1, r0:r1] = np.triu(S[r0:r1, r0:r1])


def test_fp8_tree_at_n32768_sampled(hrp_mod, handle):
    import torch
    n, nrhs, rho, spec = 32768, 16, 2.0, "[F8,F16,F16,F32|F64@128]"
    # the bench's input: A = (B + B^T)/2, B iid N(0,1), A_ii = 2 sum_{j!=i} |A_ij|
    g = torch.Generator(device="cuda")
    g.manual_seed(2601008082 + 2000)
    Bt = torch.randn((n, n), generator=g, device="cuda", dtype=torch.float64)
    A = Bt + Bt.T
    del Bt
    A.mul_(0.5)
    A.diagonal().zero_()
    A.diagonal().copy_(rho * A.abs().sum(dim=1))
    Bm = torch.randn((nrhs, n), generator=g, device="cuda", dtype=torch.float64)
    tree = hrp_mod.tree_parse(spec, leaf=128)

    Af = A.clone()
    assert handle.potrf(tree, Af) == 0
    rows = [0, 127, 128, 4095, 8191, 16383, 16384, 24575, 32767]
    A_rows = A[rows].cpu().numpy()                      # A symmetric: row i = column i
    S = Af.cpu().numpy()                                # S[j, i] = L[i, j]
    del Af
    # the first diagonal leaf is factored in FP64 from untouched data: the plain Cholesky
    L11, info = dense.cholesky(A[:128, :128].cpu().numpy())
    assert info == 0
    assert np.max(np.abs(np.tril(S[:128, :128].T) - L11)) <= 1e-12 * np.max(np.abs(L11))
    # sampled rows of L L^T against A: row i of L L^T = L[i, :] L^T = S[:, i]^T S
    _zero_below_diagonal(S)
    for r, i in enumerate(rows):
        v = S[:, i] @ S
        rel = np.linalg.norm(v - A_rows[r]) / np.linalg.norm(A_rows[r])
        assert rel <= 5e-5, (i, rel)
    del S

    # refined solve: the residual recomputed on the host from A, X and B
    X = torch.zeros_like(Bm)
    out = handle.posv(tree, A, Bm, X, max_iter=30, tol=1e-12)
    assert out["status"] == 0 and out["used_fallback"] == 0
    Ah = A.cpu().numpy()
    Xh = X.cpu().numpy().T                               # n x nrhs
    Bh = Bm.cpu().numpy().T
    R = Bh - Ah @ Xh
    res = np.linalg.norm(R, axis=0) / np.linalg.norm(Bh, axis=0)
    assert np.max(res) <= 1e-12, res
