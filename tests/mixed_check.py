"""Discriminating parity check of a mixed-precision factor against the tree emulator.

A mixed tree is an approximation (Sec. 3.3): its factor differs from the FP64 factor by
the roundings the tree prescribes.  The GPU reproduces the emulator's operand roundings
exactly but accumulates its reduced-precision GEMMs in FP32 where the emulator sums in
float64, and its FP32 leaf solve multiplies by an FP32 inverse where the emulator
substitutes.  Those differences are FP32-sized, so a correct GPU factor sits on the
emulator's factor much more closely than the factor of any tree that assigns one level a
different precision ("mis-levelled").  The check here measures exactly that:

    ratio = ||L - L_emu(tree)||_F / min_alt ||L_emu(alt) - L_emu(tree)||_F

over the alternatives that change one level of the list (F16 <-> F32, F64 -> F32,
F8 -> F16) and that the recursion at this n actually reaches (an alternative whose
factor equals the tree's is not realized and is skipped).  A plausible implementation
error -- a level run at the wrong precision, a GEMM whose operands are rounded at
another level, a missing rounding -- moves L by at least one of these distances.
"""
from __future__ import annotations

import numpy as np

from oracle import dense, tree as otree

SWAP = {"F16": "F32", "F32": "F16", "F64": "F32", "F8": "F16"}


def level_alternatives(spec: str) -> list[str]:
    t = otree.parse(spec)
    out = []
    for i, lv in enumerate(t.levels):
        levels = list(t.levels)
        levels[i] = SWAP[lv]
        inner = f"|{t.inner}@{t.inner_size}" if t.inner else ""
        out.append("[" + ",".join(levels) + inner + "]")
    return out


def mislevel_ratio(L: np.ndarray, A: np.ndarray, spec: str, leaf: int, leaf_compute=None, L_emu=None):
    """(ratio, distance to the emulator, smallest realized mis-level distance)."""
    if L_emu is None:
        L_emu, info, _ = otree.emulate_potrf(A, otree.parse(spec, leaf=leaf), leaf_compute=leaf_compute)
        assert info == 0
    d = np.linalg.norm(np.tril(L) - L_emu)
    dmin = np.inf
    floor = 1e-14 * np.linalg.norm(L_emu)
    for alt in level_alternatives(spec):
        La, info, _ = otree.emulate_potrf(A, otree.parse(alt, leaf=leaf), leaf_compute=leaf_compute)
        if info:
            continue
        da = np.linalg.norm(La - L_emu)
        if da > floor:
            dmin = min(dmin, da)
    return d / dmin, d, dmin


def fp32_effect_ratio(L: np.ndarray, A: np.ndarray, L_emu: np.ndarray) -> float:
    """||L - L64||_F / ||L_emu - L64||_F: a factor computed with a reduced level run in
    FP64 would come out much closer to the FP64 factor than the emulator is."""
    L64, _ = dense.cholesky(A)
    return np.linalg.norm(np.tril(L) - L64) / np.linalg.norm(L_emu - L64)
