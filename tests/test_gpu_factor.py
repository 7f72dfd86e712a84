"""GPU parity of the factorization and solves against the CPU oracle (through the C ABI).

* FP64 tree vs the plain Cholesky: <= 1e-12 relative (max-norm over L).
* Mixed trees vs the step-by-step emulator of Alg. 1-3: the GPU accumulates GEMMs in
  FP32 (TMEM / registers) where the emulator sums exact products in FP64, and its FP32
  leaf TRSM multiplies by the FP32 inverse of the diagonal leaf where the emulator
  substitutes.  Both are FP32 rounding effects of order K * 2^-24 relative to
  sum |x||y| per entry.  The discriminating check (tests/mixed_check.py) projects the GPU
  factor's deviation from the emulator onto the direction in which each mis-levelled tree
  (one level at another precision) would move the factor: the GPU must sit at most 0.25
  of the way there (measured: <= 0.01) for every FP16 alternative that stands above the
  FP32 noise, and must not be closer to the FP64 factor than half the emulator's distance
  (a reduced level run in FP64 fails that).  tests/test_mixed_check_cpu.py shows on the CPU
  that mis-levelled factors fail it.  max|L_gpu - L_emu| <= 1e-5 max|L| stays as a sanity
  bound.
"""
import numpy as np
import pytest

from mixed_check import check_mixed_factor
from residual_check import assert_refined
from oracle import dense, tree as otree
from synth import dominant_spd, paper_spd, rhs, seed_for

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


def _factor(hrp, h, A, spec, leaf, trsm_leaf=0):
    At = hrp.colmajor(A).cuda()
    info = h.potrf(hrp.tree_parse(spec, leaf=leaf, trsm_leaf=trsm_leaf), At)
    return np.tril(hrp.from_colmajor(At)), info, At


@pytest.mark.parametrize("n", [1, 2, 3, 7, 8, 63, 64, 65, 127, 129, 300, 1000, 1024])
def test_fp64_tree_matches_plain_cholesky(hrp_mod, handle, n):
    A = dominant_spd(n, 1.0, seed_for(0, n), shift=1.0)
    L, info, _ = _factor(hrp_mod, handle, A, "[F64]", 64)
    assert info == 0
    L0, _ = dense.cholesky(A)
    assert np.max(np.abs(L - L0)) <= 1e-12 * np.max(np.abs(L0))


@pytest.mark.parametrize("leaf", [16, 100, 128])
def test_fp64_tree_other_leaves(hrp_mod, handle, leaf):
    n = 777
    A = dominant_spd(n, 1.05, seed_for(0, 3))
    L, info, _ = _factor(hrp_mod, handle, A, "[F64]", leaf)
    assert info == 0
    L0, _ = dense.cholesky(A)
    assert np.max(np.abs(L - L0)) <= 1e-12 * np.max(np.abs(L0))


@pytest.mark.parametrize("n", [33, 47, 64, 100, 127, 128])
def test_single_fp64_leaf_on_a_cluster(hrp_mod, handle, n):
    # one leaf of order n (the 8-CTA tile kernel for 32 < n <= 128, ragged last tile)
    A = dominant_spd(n, 1.05, seed_for(0, 40 + n))
    L, info, _ = _factor(hrp_mod, handle, A, "[F64]", 128)
    assert info == 0
    L0, _ = dense.cholesky(A)
    assert np.max(np.abs(L - L0)) <= 1e-12 * np.max(np.abs(L0))


@pytest.mark.parametrize("scale", [1.0, 1e-40, 1e40])
def test_single_fp64_leaf_graded_pivots(hrp_mod, handle, scale):
    # A = G G^T with rows 2i + 1 = row 2i + eps_i h_i (eps_i from 1e-3 to 1): every odd
    # pivot is about eps_i^2 under diagonal entries about 1, so the pivot recurrence's
    # single-precision estimate of d_k cancels and its reciprocal falls back to the seed
    # from d_k itself (51 of the 128 pivots lose more than 4 bits); scaled by 1e-40 or 1e40
    # the pivots leave the single-precision range.  Backward error: |L L^T - A| <=
    # gamma_{n+1} |L| |L^T| <= (n + 1) u max a_ii per entry (Higham, Thm. 10.3), with a
    # factor 4 for the FP64 residual product and the reciprocals' last-bit errors; and no
    # more than 8x the plain Cholesky's residual (a reciprocal off in its last 8 bits would
    # show there first).
    n = 128
    rng = np.random.default_rng(seed_for(0, 42))
    G0 = rng.standard_normal((n, 2 * n)) / np.sqrt(2 * n)
    G = G0.copy()
    G[1::2] = G0[0::2] + (10.0 ** rng.uniform(-3, 0, n // 2))[:, None] * G0[1::2]
    A = (G @ G.T) * scale
    A = 0.5 * (A + A.T)
    bound = 4 * (n + 1) * np.finfo(np.float64).eps * np.max(np.diag(A))
    Lo, info0 = dense.cholesky(A)
    res0 = np.max(np.abs(Lo @ Lo.T - A))
    assert info0 == 0 and res0 <= bound
    L, info, _ = _factor(hrp_mod, handle, A, "[F64]", 128)
    assert info == 0
    res = np.max(np.abs(L @ L.T - A))
    assert res <= bound and res <= 8 * res0


@pytest.mark.parametrize("col", [1, 16, 17, 90, 127])
def test_single_fp64_leaf_reports_failing_column(hrp_mod, handle, col):
    n = 127
    A = dominant_spd(n, 2.0, seed_for(0, 41))
    A[col - 1, col - 1] = -1e3
    _, info0 = dense.cholesky(A)
    _, info, _ = _factor(hrp_mod, handle, A, "[F64]", 128)
    assert info == info0 == col


def test_upper_triangle_untouched(hrp_mod, handle):
    n = 200
    A = dominant_spd(n, 2.0, seed_for(0, 5))
    At = hrp_mod.colmajor(A).cuda()
    handle.potrf(hrp_mod.tree_parse("[F16,F32|F64@64]", leaf=64), At)
    M = hrp_mod.from_colmajor(At)
    iu = np.triu_indices(n, 1)
    assert np.array_equal(M[iu], A[iu])


MIXED = [
    ("[F32]", 128), ("[F16,F32]", 128), ("[F16,F32,F64]", 128), ("[F32,F32,F32,F64]", 128),
    ("[F16,F16,F32|F64@128]", 128), ("[F16,F16,F16,F16,F32|F64@128]", 128), ("[F16,F32|F64@64]", 64),
]


@pytest.mark.parametrize("spec,leaf", MIXED)
@pytest.mark.parametrize("n,rho", [(1000, 1.05), (2048, 2.0), (1300, 8.0)])
def test_mixed_tree_matches_emulator(hrp_mod, handle, spec, leaf, n, rho):
    A = dominant_spd(n, rho, seed_for(1, n))
    L, info, _ = _factor(hrp_mod, handle, A, spec, leaf)
    assert info == 0
    L_emu, info_e, _ = otree.emulate_potrf(A, otree.parse(spec, leaf=leaf))
    assert info_e == 0
    scale = np.max(np.abs(L_emu))
    d_gpu = np.max(np.abs(L - L_emu)) / scale
    assert d_gpu <= 1e-5, d_gpu
    assert dense.backward_error(A, L) <= 5e-5
    rows, gn = check_mixed_factor(L, A, spec, leaf, L_emu=L_emu)
    print(f"{spec} n={n}: |L-L_emu|_F = {gn:.2e}; " + "; ".join(f"{a} |v|={v:.2e} t={t:+.3f}" for a, _, v, t in rows))


def test_large_fp32_level_matches_emulator(hrp_mod, handle):
    # n = 4096 with an FP32 tree: the FP32 products of the outer levels (2048^2 x 2048 and
    # below) are large enough to run on 128 x 128 tiles from the FP32 shadow.  With every
    # level FP32, the GPU's FP32 accumulation over k = 2048 moves entries by as much as the
    # FP32 operand rounding the emulator models (both ~1e-10 relative here), so only the
    # FP32-accumulation bound is asserted, not the "closer to the emulator" ratio.
    n = 4096
    A = dominant_spd(n, 2.0, seed_for(0, 77))
    L, info, _ = _factor(hrp_mod, handle, A, "[F32|F64@128]", 128)
    assert info == 0
    L_emu, info_e, _ = otree.emulate_potrf(A, otree.parse("[F32|F64@128]", leaf=128))
    assert info_e == 0
    assert np.max(np.abs(L - L_emu)) <= 1e-5 * np.max(np.abs(L_emu))
    rows, gn = check_mixed_factor(L, A, "[F32|F64@128]", 128, L_emu=L_emu)
    print(f"[F32|F64@128] n={n}: |L-L_emu|_F = {gn:.2e}; " + "; ".join(f"{a} t={t:+.3f}" for a, _, _, t in rows))


def test_large_fp16_level_matches_emulator(hrp_mod, handle):
    # n = 8192: the outer FP16 products have more 256-column tiles than SMs and run on the
    # persistent tcgen05 kernel (double-buffered TMEM accumulator).  Its result is bitwise the
    # one-tile-per-CTA kernel's (same MMAs in the same K order, same epilogue).  At this size
    # the FP32 accumulation over k = 4096 moves entries by about half the FP16 effect the
    # emulator models (the emulator sums exactly), so the ratio bound is 0.6 here, not 0.1.
    n, spec = 8192, "[F16,F32|F64@128]"
    A = dominant_spd(n, 1.05, seed_for(0, 78))
    L, info, _ = _factor(hrp_mod, handle, A, spec, 128)
    assert info == 0
    L_emu, info_e, _ = otree.emulate_potrf(A, otree.parse(spec, leaf=128))
    assert info_e == 0
    L0, _ = dense.cholesky(A)
    assert np.max(np.abs(L - L_emu)) <= 1e-5 * np.max(np.abs(L_emu))
    assert np.max(np.abs(L - L_emu)) <= 0.6 * np.max(np.abs(L_emu - L0))


@pytest.mark.parametrize("spec,leaf", [("[F16,F64]", 128), ("[F16,F16,F64]", 64), ("[F16,F16,F16,F64]", 128),
                                       ("[F64,F16,F64]", 64)])
@pytest.mark.parametrize("n,rho", [(1000, 1.05), (2048, 2.0)])
def test_fp16_levels_reproduce_emulator_rounding(hrp_mod, handle, spec, leaf, n, rho):
    """With every leaf in FP64 (trsm_compute = FP64, FP64 diagonal) the only reduced
    precision left is the FP16 rounding of the GEMM operands, so GPU and emulator differ
    only by the GPU's FP32 accumulation (~K 2^-24 of the terms): the GPU factor must sit
    on the emulator's, far closer than the FP16 effect itself (emulator vs FP64)."""
    A = dominant_spd(n, rho, seed_for(1, n))
    At = hrp_mod.colmajor(A).cuda()
    info = handle.potrf(hrp_mod.tree_parse(spec, leaf=leaf, trsm_fp64=True), At)
    assert info == 0
    L = np.tril(hrp_mod.from_colmajor(At))
    L_emu, _, _ = otree.emulate_potrf(A, otree.parse(spec, leaf=leaf), leaf_compute="F64")
    L64, _ = dense.cholesky(A)
    d_gpu = np.max(np.abs(L - L_emu))
    d_emu = np.max(np.abs(L_emu - L64))
    assert d_emu > 1e3 * 2.0 ** -52 * np.max(np.abs(L64))     # FP16 did change the factor
    # FP32 accumulation noise relative to the FP16 operand noise: ~ sqrt(K) 2^-24 / 2^-11
    # (about 0.004 at K = 1024); a term rounded at the wrong level would give ~1
    assert d_gpu <= 0.3 * d_emu, (d_gpu, d_emu)
    f_gpu = np.linalg.norm(L - L_emu)
    f_emu = np.linalg.norm(L_emu - L64)
    assert f_gpu <= 0.05 * f_emu, (f_gpu, f_emu)


def test_paper_generator_ladder_on_gpu(hrp_mod, handle):
    n = 1024
    A = paper_spd(n, seed_for(9, 1))
    errs = {}
    for spec in ["[F64]", "[F32,F32,F32,F64]", "[F32]", "[F16,F32]"]:
        L, info, _ = _factor(hrp_mod, handle, A, spec, 128)
        assert info == 0
        errs[spec] = dense.backward_error(A, L)
    assert errs["[F64]"] < 1e-14
    assert errs["[F64]"] < errs["[F32,F32,F32,F64]"] < errs["[F32]"]


@pytest.mark.parametrize("n,nrhs", [(1, 1), (65, 3), (1000, 1), (1100, 16), (640, 20)])
def test_potrs_fp64_matches_oracle(hrp_mod, handle, n, nrhs):
    A = dominant_spd(n, 1.0, seed_for(0, n), shift=1.0)
    L0, _ = dense.cholesky(A)
    B = rhs(n, nrhs, seed_for(0, 100 + n))
    Lt = hrp_mod.colmajor(L0).cuda()
    Bt = hrp_mod.colmajor(B).cuda()
    handle.potrs(Lt, Bt)
    X = hrp_mod.from_colmajor(Bt)
    X0 = dense.potrs(L0, B)
    assert np.max(np.abs(X - X0)) <= 1e-12 * np.max(np.abs(X0))


@pytest.mark.parametrize("nrhs", [1, 3, 16])
def test_potrs_columns_of_any_magnitude(hrp_mod, handle, nrhs):
    """The solve forms its products in pairs of binary32 values scaled by powers of two per
    group of entries: right-hand sides whose columns lie near the ends of the FP64 range
    (2^-900 .. 2^900, far outside binary32's) are solved as accurately as unit ones, column
    by column, against the oracle's FP64 solve."""
    n = 1000
    A = dominant_spd(n, 1.0, seed_for(0, 77), shift=1.0)
    L0, _ = dense.cholesky(A)
    B = rhs(n, nrhs, seed_for(0, 78))
    exps = [(-900, 0, 900)[c % 3] for c in range(nrhs)]
    B = B * np.array([2.0 ** e for e in exps])[None, :]
    Lt = hrp_mod.colmajor(L0).cuda()
    Bt = hrp_mod.colmajor(B).cuda()
    handle.potrs(Lt, Bt)
    X = hrp_mod.from_colmajor(Bt)
    X0 = dense.potrs(L0, B)
    for c in range(nrhs):
        assert np.all(np.isfinite(X[:, c]))
        assert np.max(np.abs(X[:, c] - X0[:, c])) <= 1e-12 * np.max(np.abs(X0[:, c])), (c, exps[c])


def test_not_spd_reports_first_failing_column(hrp_mod, handle):
    n = 300
    A = dominant_spd(n, 2.0, seed_for(0, 9))
    A[200, 200] = -5.0
    _, info0 = dense.cholesky(A)
    for spec, leaf in [("[F64]", 64), ("[F16,F32|F64@64]", 64)]:
        _, info, _ = _factor(hrp_mod, handle, A, spec, leaf)
        assert info == info0 == 201
    A = dominant_spd(n, 2.0, seed_for(0, 9))
    A[37, 37] = np.nan
    _, info, _ = _factor(hrp_mod, handle, A, "[F64]", 64)
    assert info == 38


def test_invalid_arguments(hrp_mod, handle):
    import torch
    t = hrp_mod.tree_parse("[F64]", leaf=64)
    A = torch.zeros((8, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(hrp_mod.HrpError):
        handle.potrf(t, A, n=9)            # lda (8) < n
    assert handle.last_arg() == -5
    bad = hrp_mod.tree_parse("[F64]", leaf=64)
    bad.leaf = 0
    with pytest.raises(hrp_mod.HrpError):
        handle.potrf(bad, A)
    assert handle.last_arg() == -2


def test_empty_matrix(hrp_mod, handle):
    import torch
    A = torch.zeros((1, 1), dtype=torch.float64, device="cuda")
    assert handle.potrf(hrp_mod.tree_parse("[F16,F32]", 128), A, n=0) == 0


def test_gpu_backward_error_matches_cpu(hrp_mod, handle):
    n = 700
    A = dominant_spd(n, 1.05, seed_for(1, 11))
    L, info, At = _factor(hrp_mod, handle, A, "[F16,F32]", 128)
    assert info == 0
    A_t = hrp_mod.colmajor(A).cuda()
    be_gpu = handle.backward_error(A_t, At)
    be_cpu = dense.backward_error(A, L)
    assert abs(be_gpu - be_cpu) <= 1e-6 * be_cpu + 1e-15


@pytest.mark.parametrize("spec", ["[F16,F16,F32|F64@128]", "[F64]"])
def test_posv_refines_to_tolerance(hrp_mod, handle, spec):
    import torch
    n, nrhs = 1500, 4
    A = dominant_spd(n, 2.0, seed_for(2, 1))
    B = rhs(n, nrhs, seed_for(2, 2))
    A_t = hrp_mod.colmajor(A).cuda()
    B_t = hrp_mod.colmajor(B).cuda()
    X_t = torch.zeros_like(B_t)
    A_before = A_t.clone()
    out = handle.posv(hrp_mod.tree_parse(spec, 128), A_t, B_t, X_t, max_iter=30, tol=1e-12)
    assert out["status"] == 0 and out["info"] == 0
    assert torch.equal(A_t, A_before)                    # A is not modified
    X = hrp_mod.from_colmajor(X_t)
    res = dense.column_residuals(A, X, B)
    assert np.max(res) <= 1e-12
    assert abs(out["resid"] - np.max(res)) <= 1e-13 + 0.1 * np.max(res)


def test_posv_falls_back_when_the_mixed_tree_fails(hrp_mod, handle):
    """Pure FP16 off-diagonals on a barely positive definite matrix lose definiteness;
    hrp_posv must refactor with the FP32/FP64 tree and still converge."""
    import torch
    n = 600
    L = np.tril(np.random.default_rng(4).standard_normal((n, n)) * 0.3)
    np.fill_diagonal(L, 1e-3)
    A = L @ L.T + 1e-9 * np.eye(n)
    B = rhs(n, 1, seed_for(2, 3))
    _, info16, _ = otree.emulate_potrf(A, otree.parse("[F16,F16,F16]", leaf=64))
    if info16 == 0:
        pytest.skip("matrix did not break the FP16 tree in the emulator")
    A_t = hrp_mod.colmajor(A).cuda()
    B_t = hrp_mod.colmajor(B).cuda()
    X_t = torch.zeros_like(B_t)
    out = handle.posv(hrp_mod.tree_parse("[F16,F16,F16]", 64), A_t, B_t, X_t, max_iter=5, tol=1e-30)
    assert out["used_fallback"] == 1


# ---------------------------------------------------------------------------------------
# FP8 E4M3 outermost level (per-128x128 power-of-two tile scales)
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("spec", ["[F8,F16,F32|F64@128]", "[F8,F32|F64@128]"])
@pytest.mark.parametrize("n,rho", [(1024, 2.0), (2048, 1.05)])
def test_fp8_tree_matches_emulator(hrp_mod, handle, spec, n, rho):
    """E4M3 rounding moves an operand by up to 2^-4 of itself, so a rounding decision the
    GPU and the emulator take differently (their FP32/FP64 accumulations differ before
    the operand is quantized) changes one term by ~6%; such flips are rare and diluted
    over K terms, so the bound is 1e-4 max|L| (1e-5 for the FP16 trees)."""
    A = dominant_spd(n, rho, seed_for(3, n))
    L, info, _ = _factor(hrp_mod, handle, A, spec, 128)
    assert info == 0
    L_emu, info_e, em = otree.emulate_potrf(A, otree.parse(spec, leaf=128))
    assert info_e == 0 and any(c[0] == "F8" for c in em.gemm_calls)
    scale = np.max(np.abs(L_emu))
    d_gpu = np.max(np.abs(L - L_emu)) / scale
    assert d_gpu <= 1e-4, d_gpu
    be_gpu, be_emu = dense.backward_error(A, L), dense.backward_error(A, L_emu)
    assert abs(be_gpu - be_emu) <= 0.05 * be_emu


@pytest.mark.parametrize("spec", ["[F8,F64]", "[F8,F16,F64]"])
def test_fp8_levels_reproduce_emulator_rounding(hrp_mod, handle, spec):
    """With every leaf in FP64 only the E4M3 (and FP16) operand rounding remains: the GPU
    factor must sit on the emulator's, far inside the size of the E4M3 effect."""
    n = 1024
    A = dominant_spd(n, 1.05, seed_for(3, 77))
    At = hrp_mod.colmajor(A).cuda()
    assert handle.potrf(hrp_mod.tree_parse(spec, leaf=128, trsm_fp64=True), At) == 0
    L = np.tril(hrp_mod.from_colmajor(At))
    L_emu, _, _ = otree.emulate_potrf(A, otree.parse(spec, leaf=128), leaf_compute="F64")
    L64, _ = dense.cholesky(A)
    f_gpu = np.linalg.norm(L - L_emu)
    f_emu = np.linalg.norm(L_emu - L64)
    assert f_emu > 1e-8 * np.linalg.norm(L64)
    assert f_gpu <= 0.02 * f_emu, (f_gpu, f_emu)


@pytest.mark.parametrize("spec,n", [("[F8,F16,F32|F64@128]", 2048), ("[F8,F32|F64@128]", 1024),
                                    ("[F8,F16,F16,F32|F64@128]", 4096)])
def test_fp8_block_scaled_equals_fp16_storage(hrp_mod, handle, spec, n):
    """The block-scaled E4M3 MMAs (UE8M0 scale per tile) and the FP16-stored E4M3 values on the
    FP16 GEMM form the same exact products of the same quantized operands; only the FP32
    accumulation inside the tensor core may differ, and with it, rarely, a later rounding
    decision of the quantizer."""
    A = dominant_spd(n, 2.0, seed_for(3, 300 + n))
    L8, info8 = _factor_mode(hrp_mod, A, spec, fp16_storage=False)
    L16, info16 = _factor_mode(hrp_mod, A, spec, fp16_storage=True)
    assert info8 == info16 == 0
    scale = np.max(np.abs(L16))
    d = np.abs(np.tril(L8 - L16)) / scale
    assert np.median(d[np.tril_indices(n)]) <= 1e-8 and d.max() <= 1e-4, (np.median(d), d.max())


def _factor_mode(hrp_mod, A, spec, fp16_storage):
    h = hrp_mod.Handle(0)
    try:
        h.set_f8_gemm(fp16_storage)
        At = hrp_mod.colmajor(A).cuda()
        info = h.potrf(hrp_mod.tree_parse(spec, leaf=128), At)
        assert h.check() == 0
        return np.tril(hrp_mod.from_colmajor(At)), info
    finally:
        h.close()


def test_fp8_requires_power_of_two_blocks(hrp_mod, handle):
    A = dominant_spd(1000, 2.0, seed_for(3, 5))
    At = hrp_mod.colmajor(A).cuda()
    with pytest.raises(hrp_mod.HrpError) as e:
        handle.potrf(hrp_mod.tree_parse("[F8,F32|F64@128]", leaf=128), At)
    assert e.value.status == 7


def test_posv_with_fp8_tree_refines(hrp_mod, handle):
    import torch
    n, nrhs = 2048, 16
    A = dominant_spd(n, 2.0, seed_for(3, 9))
    B = rhs(n, nrhs, seed_for(3, 10))
    A_t = hrp_mod.colmajor(A).cuda()
    B_t = hrp_mod.colmajor(B).cuda()
    X_t = torch.zeros_like(B_t)
    out = handle.posv(hrp_mod.tree_parse("[F8,F16,F16,F32|F64@128]", 128), A_t, B_t, X_t, tol=1e-12)
    assert out["status"] == 0 and out["used_fallback"] == 0
    X = hrp_mod.from_colmajor(X_t)
    assert np.max(dense.column_residuals(A, X, B)) <= 1e-12


# ---------------------------------------------------------------------------------------
# batched factorization / solve (many independent systems, one stream pool, graph-capturable)
# ---------------------------------------------------------------------------------------
def test_batched_equals_one_by_one(hrp_mod, handle):
    """Stream-pool mode: every system runs the single factorization's kernels in the same
    order, so the factors are bitwise those of hrp_potrf."""
    import torch
    handle.set_batched_mode(False)
    sizes = [64, 200, 128, 513, 96, 1000, 1, 300, 777, 65]
    mats = [dominant_spd(n, 1.5, seed_for(4, i), shift=1.0) for i, n in enumerate(sizes)]
    tree = hrp_mod.tree_parse("[F16,F32|F64@128]", leaf=128)
    As = [hrp_mod.colmajor(A).cuda() for A in mats]
    d_info = torch.full((len(sizes),), -1, dtype=torch.int32, device="cuda")
    handle.potrf_batched(tree, As, d_info)
    torch.cuda.synchronize()
    assert d_info.cpu().tolist() == [0] * len(sizes)
    for A, At in zip(mats, As):
        single = hrp_mod.colmajor(A).cuda()
        assert handle.potrf(tree, single) == 0
        assert torch.equal(torch.tril(single.T), torch.tril(At.T))     # same kernels, same order
    Bs = [hrp_mod.colmajor(rhs(n, 4, seed_for(4, 100 + i))).cuda() for i, n in enumerate(sizes)]
    B_single = [B.clone() for B in Bs]
    handle.potrs_batched(As, Bs)
    torch.cuda.synchronize()
    for At, B, Bs1, A in zip(As, Bs, B_single, mats):
        handle.potrs(At, Bs1)
        assert torch.equal(B, Bs1)
        L = np.tril(hrp_mod.from_colmajor(At))
        X_ref = dense.potrs(L, rhs(A.shape[0], 4, seed_for(4, 100 + sizes.index(A.shape[0]))))
        X = hrp_mod.from_colmajor(B)
        assert np.max(np.abs(X - X_ref)) <= 1e-12 * np.max(np.abs(X_ref))
    handle.set_batched_mode(False)


@pytest.mark.parametrize("persistent", [True, False])
def test_batched_reports_per_system_info(hrp_mod, handle, persistent):
    import torch
    handle.set_batched_mode(persistent)
    sizes = [100, 150, 80]
    mats = [dominant_spd(n, 2.0, seed_for(4, 50 + i)) for i, n in enumerate(sizes)]
    mats[1][40, 40] = -1.0
    _, info1 = dense.cholesky(mats[1])
    As = [hrp_mod.colmajor(A).cuda() for A in mats]
    d_info = torch.zeros(len(sizes), dtype=torch.int32, device="cuda")
    handle.potrf_batched(hrp_mod.tree_parse("[F64]", leaf=64), As, d_info)
    torch.cuda.synchronize()
    handle.set_batched_mode(False)
    assert d_info.cpu().tolist() == [0, info1, 0] and info1 == 41


def test_batched_graph_capture_replays(hrp_mod, handle):
    import torch
    sizes = [256, 384, 128, 640]
    mats = [dominant_spd(n, 2.0, seed_for(4, 70 + i)) for i, n in enumerate(sizes)]
    tree = hrp_mod.tree_parse("[F16,F32|F64@128]", leaf=128)
    A0 = [hrp_mod.colmajor(A).cuda() for A in mats]
    As = [A.clone() for A in A0]
    d_info = torch.zeros(len(sizes), dtype=torch.int32, device="cuda")
    handle.potrf_batched(tree, As, d_info)          # allocates the workspace (outside capture)
    torch.cuda.synchronize()
    ref = [A.clone() for A in As]
    for A, a0 in zip(As, A0):
        A.copy_(a0)
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            handle.potrf_batched(tree, As, d_info, stream=s)
    for rep in range(2):
        for A, a0 in zip(As, A0):
            A.copy_(a0)
        g.replay()
        torch.cuda.synchronize()
        for A, R in zip(As, ref):
            assert torch.equal(torch.tril(A.T), torch.tril(R.T))


def test_posv_batched_refines_every_system(hrp_mod, handle):
    import torch
    from synth import rbf_spd
    sizes = [64, 300, 129, 700, 512]
    mats = [rbf_spd(n, seed_for(4, 200 + i)) for i, n in enumerate(sizes)]
    As = [hrp_mod.colmajor(A).cuda() for A in mats]
    Bs = [hrp_mod.colmajor(rhs(n, 4, seed_for(4, 300 + i))).cuda() for i, n in enumerate(sizes)]
    Xs = [torch.zeros_like(B) for B in Bs]
    keep = [A.clone() for A in As]
    out = handle.posv_batched(hrp_mod.tree_parse("[F16,F32|F64@128]", 128), As, Bs, Xs, tol=1e-12)
    assert out["status"] == 0 and out["info"] == [0] * len(sizes)
    for A, K in zip(As, keep):
        assert torch.equal(A, K)                           # inputs untouched
    for i, A in enumerate(mats):
        X = hrp_mod.from_colmajor(Xs[i])
        B = hrp_mod.from_colmajor(Bs[i])
        assert out["resid"][i] <= 1e-12
        assert_refined(A, X, B, 1e-12, reported=out["resid"][i])


# ---------------------------------------------------------------------------------------
# persistent batched launch (batched mode 1): many uneven systems in one launch
# ---------------------------------------------------------------------------------------
def _uneven_sizes(count, lo, hi, seed):
    return [int(x) for x in np.random.default_rng(seed).integers(lo, hi + 1, count)]


def test_persistent_batched_fp64_tree_matches_cholesky(hrp_mod, handle):
    import torch
    handle.set_batched_mode(True)
    sizes = _uneven_sizes(40, 1, 600, seed_for(4, 400))
    mats = [dominant_spd(n, 1.2, seed_for(4, 410 + i), shift=1.0) for i, n in enumerate(sizes)]
    As = [hrp_mod.colmajor(A).cuda() for A in mats]
    d_info = torch.full((len(sizes),), -7, dtype=torch.int32, device="cuda")
    handle.potrf_batched(hrp_mod.tree_parse("[F64]", leaf=64), As, d_info)
    torch.cuda.synchronize()
    assert handle.launch_count() == 1
    assert d_info.cpu().tolist() == [0] * len(sizes)
    for A, At in zip(mats, As):
        L0, _ = dense.cholesky(A)
        L = np.tril(hrp_mod.from_colmajor(At))
        assert np.max(np.abs(L - L0)) <= 1e-12 * np.max(np.abs(L0))
    handle.set_batched_mode(False)


def test_persistent_batched_mixed_tree_matches_emulator(hrp_mod, handle):
    """[F16,F32|F64@128] over 36 uneven systems: every factor within the FP32 noise of the
    emulator's (max-norm 1e-5 of max|L|, backward error within 2x of the emulator's), and the
    projection check against mis-levelled trees on the largest systems."""
    import torch
    handle.set_batched_mode(True)
    spec = "[F16,F32|F64@128]"
    sizes = _uneven_sizes(36, 64, 900, seed_for(4, 500)) + [1100, 1300]
    mats = [dominant_spd(n, 1.05, seed_for(4, 510 + i)) for i, n in enumerate(sizes)]
    As = [hrp_mod.colmajor(A).cuda() for A in mats]
    d_info = torch.full((len(sizes),), -7, dtype=torch.int32, device="cuda")
    handle.potrf_batched(hrp_mod.tree_parse(spec, leaf=128), As, d_info)
    torch.cuda.synchronize()
    assert d_info.cpu().tolist() == [0] * len(sizes)
    for n, A, At in zip(sizes, mats, As):
        L = np.tril(hrp_mod.from_colmajor(At))
        L_emu, info, _ = otree.emulate_potrf(A, otree.parse(spec, leaf=128))
        assert info == 0
        assert np.max(np.abs(L - L_emu)) <= 1e-5 * np.max(np.abs(L_emu)), n
        be, be_emu = dense.backward_error(A, L), dense.backward_error(A, L_emu)
        assert be <= 2 * be_emu + 1e-15, (n, be, be_emu)
        if n >= 1100:
            check_mixed_factor(L, A, spec, 128, L_emu=L_emu)
    handle.set_batched_mode(False)


def test_persistent_batched_posv_and_graph_replay(hrp_mod, handle):
    import torch
    from synth import rbf_spd
    handle.set_batched_mode(True)
    sizes = _uneven_sizes(32, 64, 700, seed_for(4, 600))
    mats = [rbf_spd(n, seed_for(4, 610 + i)) for i, n in enumerate(sizes)]
    As = [hrp_mod.colmajor(A).cuda() for A in mats]
    Bs = [hrp_mod.colmajor(rhs(n, 4, seed_for(4, 650 + i))).cuda() for i, n in enumerate(sizes)]
    Xs = [torch.zeros_like(B) for B in Bs]
    out = handle.posv_batched(hrp_mod.tree_parse("[F16,F32|F64@128]", 128), As, Bs, Xs, tol=1e-12)
    assert out["status"] == 0 and out["info"] == [0] * len(sizes)
    assert max(out["resid"]) <= 1e-12
    # the FP64 residual of these RBF systems (kappa up to ~1e5) is at its evaluation floor:
    # the exact residual, within the bound on the GPU's own evaluation error
    for A, B, X in zip(mats, Bs, Xs):
        assert_refined(A, hrp_mod.from_colmajor(X), hrp_mod.from_colmajor(B), 1e-12)
    # one persistent launch captured in a graph and replayed: the same factors each time
    tree = hrp_mod.tree_parse("[F16,F32|F64@128]", leaf=128)
    A0 = [A.clone() for A in As]
    W = [A.clone() for A in As]
    d_info = torch.zeros(len(sizes), dtype=torch.int32, device="cuda")
    handle.potrf_batched(tree, W, d_info)
    torch.cuda.synchronize()
    ref = [w.clone() for w in W]
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            handle.potrf_batched(tree, W, d_info, stream=s)
    for rep in range(2):
        for w, a0 in zip(W, A0):
            w.copy_(a0)
        g.replay()
        torch.cuda.synchronize()
        for w, r in zip(W, ref):
            assert torch.equal(w, r), rep
    handle.set_batched_mode(False)
