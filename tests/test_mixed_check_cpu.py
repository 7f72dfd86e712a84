"""The mixed-tree parity check (tests/mixed_check.py) rejects a mis-levelled factor and
accepts a factor that differs from the emulator only by FP32 accumulation.

No GPU: the "correct" candidate is the emulator with every reduced-precision GEMM
accumulated in float32, 16 exact products at a time, each partial sum truncated toward
zero (a pessimistic stand-in for the tensor cores' FP32 accumulator); the wrong
candidates are planted on the CPU.
"""
import numpy as np
import pytest

from mixed_check import fp32_effect_ratio, level_alternatives, mislevel_ratio
from oracle import dense, tree as otree
from synth import dominant_spd, seed_for

MISLEVEL_BOUND = 0.3      # the GPU test's bound on mislevel_ratio
FP32_EFFECT_RANGE = (0.5, 2.0)


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


def _acc32(A, spec, leaf):
    em = Acc32(A, otree.parse(spec, leaf=leaf))
    em.potrf(0, em.n, 0)
    return np.tril(em.M)


def test_level_alternatives():
    assert level_alternatives("[F16,F32|F64@128]") == ["[F32,F32|F64@128]", "[F16,F16|F64@128]"]
    assert level_alternatives("[F8,F64]") == ["[F16,F64]", "[F8,F32]"]


@pytest.mark.parametrize("spec,leaf", [("[F16,F16,F32|F64@128]", 128), ("[F16,F32|F64@64]", 64),
                                       ("[F16,F32,F64]", 128)])
def test_fp32_accumulation_passes_and_a_mislevelled_tree_fails(spec, leaf):
    n = 1000
    A = dominant_spd(n, 1.05, seed_for(1, n))
    r_ok, _, _ = mislevel_ratio(_acc32(A, spec, leaf), A, spec, leaf)
    assert r_ok <= MISLEVEL_BOUND, r_ok
    for alt in level_alternatives(spec):
        L_alt, info, _ = otree.emulate_potrf(A, otree.parse(alt, leaf=leaf))
        r_bad, d_bad, _ = mislevel_ratio(L_alt, A, spec, leaf)
        if d_bad > 0:
            assert r_bad >= 1.0 > MISLEVEL_BOUND


def test_operands_rounded_at_the_wrong_level_fail():
    """A GEMM of a deeper F32 node fed FP16 operands (the shallower level's rounding)."""
    spec, leaf, n = "[F16,F32|F64@128]", 128, 1000
    A = dominant_spd(n, 1.05, seed_for(1, n))

    class Wrong(otree.Emulator):
        def _gemm(self, p, r0, m, c0, nd, k0, k, lower=False):
            super()._gemm("F16" if p == "F32" else p, r0, m, c0, nd, k0, k, lower)

    em = Wrong(A, otree.parse(spec, leaf=leaf))
    em.potrf(0, em.n, 0)
    r, _, _ = mislevel_ratio(np.tril(em.M), A, spec, leaf)
    assert r > MISLEVEL_BOUND


@pytest.mark.parametrize("spec", ["[F32]", "[F32,F32,F32,F64]"])
def test_fp32_levels_run_in_fp64_fail_the_effect_bound(spec):
    n = 1000
    A = dominant_spd(n, 2.0, seed_for(1, n))
    L_emu, _, _ = otree.emulate_potrf(A, otree.parse(spec, leaf=128))
    lo, hi = FP32_EFFECT_RANGE
    assert lo <= fp32_effect_ratio(_acc32(A, spec, 128), A, L_emu) <= hi
    L64, _ = dense.cholesky(A)
    assert fp32_effect_ratio(L64, A, L_emu) < lo
