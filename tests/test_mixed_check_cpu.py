"""The mixed-tree parity check (tests/mixed_check.py) rejects mis-levelled factors and
accepts factors that differ from the emulator only by FP32 arithmetic.

No GPU: the "correct" candidate is the emulator with every reduced-precision GEMM
accumulated in float32, 16 exact products at a time, each partial sum truncated toward
zero (a pessimistic stand-in for the tensor cores' FP32 accumulator); the wrong ones
are the same model run on a mis-levelled tree, or with operands rounded at the wrong level.
"""
import numpy as np
import pytest

from mixed_check import check_mixed_factor, level_alternatives, mislevel_projections
from oracle import dense, tree as otree
from synth import dominant_spd, seed_for


class Acc32(otree.Emulator):
    def _gemm(self, p, r0, m, c0, nd, k0, k, lower=False):
        if m == 0 or nd == 0 or k == 0:
            return
        if p == "F64":
            return super()._gemm(p, r0, m, c0, nd, k0, k, lower)
        X, Y, scale = self._operands(p, r0, m, c0, nd, k0, k)
        acc = np.zeros((m, nd), np.float32)
        for q in range(0, k, 16):
            s = acc.astype(np.float64) + X[:, q:q + 16] @ Y[:, q:q + 16].T
            f = s.astype(np.float32)
            over = np.abs(f.astype(np.float64)) > np.abs(s)
            f[over] = np.nextafter(f[over], np.float32(0))
            acc = f
        prod = scale * acc.astype(np.float64)
        D = self.M[r0:r0 + m, c0:c0 + nd]
        if lower:
            mask = np.arange(r0, r0 + m)[:, None] >= np.arange(c0, c0 + nd)[None, :]
            D -= np.where(mask, prod, 0.0)
        else:
            D -= prod


def _acc32(A, spec, leaf, cls=Acc32):
    em = cls(A, otree.parse(spec, leaf=leaf))
    em.potrf(0, em.n, 0)
    return np.tril(em.M)


def test_level_alternatives():
    assert level_alternatives("[F16,F32|F64@128]") == [
        ("[F32,F32|F64@128]", True), ("[F16,F16|F64@128]", True), ("[F16,F64|F64@128]", False),
        ("[F16,F32|F32@128]", False)]
    assert level_alternatives("[F8,F64]") == [("[F16,F64]", True), ("[F8,F32]", False)]


SPECS = [("[F16,F16,F32|F64@128]", 128), ("[F16,F32|F64@64]", 64), ("[F16,F32,F64]", 128),
         ("[F16,F16,F16,F16,F32|F64@128]", 128)]


@pytest.mark.parametrize("spec,leaf", SPECS)
def test_fp32_accumulation_passes_and_mislevelled_trees_fail(spec, leaf):
    n = 1000
    A = dominant_spd(n, 1.05, seed_for(1, n))
    check_mixed_factor(_acc32(A, spec, leaf), A, spec, leaf)
    L_emu, _, _ = otree.emulate_potrf(A, otree.parse(spec, leaf=leaf))
    for alt, low in level_alternatives(spec):
        if not low:
            continue
        L_bad = _acc32(A, alt, leaf)
        rows, gn = mislevel_projections(L_bad, A, spec, leaf, L_emu=L_emu)
        if not any(a == alt for a, _, _, _ in rows):
            continue                                   # level not reached at this n
        with pytest.raises(AssertionError):
            check_mixed_factor(L_bad, A, spec, leaf, L_emu=L_emu)


def test_operands_rounded_at_the_wrong_level_fail():
    """The GEMMs of the F32 nodes fed FP16 operands (a shallower level's rounding)."""
    spec, leaf, n = "[F16,F32|F64@128]", 128, 1000
    A = dominant_spd(n, 1.05, seed_for(1, n))

    class Wrong(Acc32):
        def _gemm(self, p, r0, m, c0, nd, k0, k, lower=False):
            super()._gemm("F16" if p == "F32" else p, r0, m, c0, nd, k0, k, lower)

    with pytest.raises(AssertionError):
        check_mixed_factor(_acc32(A, spec, leaf, Wrong), A, spec, leaf)


@pytest.mark.parametrize("spec", ["[F32]", "[F32,F32,F32,F64]"])
def test_fp32_levels_run_in_fp64_fail(spec):
    n = 1000
    A = dominant_spd(n, 2.0, seed_for(1, n))
    check_mixed_factor(_acc32(A, spec, 128), A, spec, 128)
    L64, _ = dense.cholesky(A)
    with pytest.raises(AssertionError):
        check_mixed_factor(L64, A, spec, 128)
