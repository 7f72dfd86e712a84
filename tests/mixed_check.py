"""Discriminating parity check of a mixed-precision factor against the tree emulator.

A mixed tree is an approximation (Sec. 3.3): its factor differs from the FP64 factor by
the roundings the tree prescribes.  The GPU reproduces the emulator's operand roundings
(FP16 / E4M3 / FP32 of the same values), but it accumulates its GEMMs in FP32 where the
emulator sums in float64, runs its FP32 leaf Cholesky right-looking, and solves FP32
leaves through an FP32 inverse.  Those deviations are FP32 noise, unrelated to the
rounding decisions that distinguish one precision tree from another.

For each alternative tree that assigns one level (or the inner region) another precision,
v = L_emu(alt) - L_emu(tree) is the direction in which that mistake would move the factor,
and with g = L - L_emu(tree),

    t = <g, v> / <v, v>

is how far along that direction the candidate factor sits: 0 for the right tree, 1 for
the mis-levelled one.  Measured on GB300, a correct factor gives |t| <= 0.01 for every
alternative that changes an FP16 / E4M3 level, whenever |v| is at least half of |g| (an
alternative whose whole effect is smaller than the FP32 noise cannot be told apart and is
not used).  Alternatives that only trade FP32 for FP64 move the factor along the FP32
rounding the GPU shares in part with the emulator (t = 0.3-0.9 for a correct factor);
for them the check is that the factor is not closer to the FP64 factor than half the
emulator's distance, which a reduced level run in FP64 throughout fails.
"""
from __future__ import annotations

import numpy as np

from oracle import dense, tree as otree

T_MAX = 0.25            # |t| bound for the FP16 / E4M3 alternatives
NOISE_FLOOR = 0.5       # an alternative is used when |v| >= NOISE_FLOOR |g|
FP64_DISTANCE_MIN = 0.5


def level_alternatives(spec: str) -> list[tuple[str, bool]]:
    """(alternative spec, whether it changes an FP16 / E4M3 rounding) per level swap."""
    t = otree.parse(spec)
    inner = f"|{t.inner}@{t.inner_size}" if t.inner else ""
    swaps = {"F16": ["F32"], "F32": ["F16", "F64"], "F64": ["F32"], "F8": ["F16"]}
    out = []
    for i, lv in enumerate(t.levels):
        for sw in swaps[lv]:
            levels = list(t.levels)
            levels[i] = sw
            out.append(("[" + ",".join(levels) + inner + "]", "F16" in (lv, sw) or "F8" in (lv, sw)))
    if t.inner:
        other = "F32" if t.inner == "F64" else "F64"
        out.append(("[" + ",".join(t.levels) + f"|{other}@{t.inner_size}]", False))
    return out


def mislevel_projections(L: np.ndarray, A: np.ndarray, spec: str, leaf: int, leaf_compute=None, L_emu=None):
    """[(alt, low-precision alternative?, |v|, t)] for the realized alternatives, and |g|."""
    if L_emu is None:
        L_emu, info, _ = otree.emulate_potrf(A, otree.parse(spec, leaf=leaf), leaf_compute=leaf_compute)
        assert info == 0
    g = np.tril(L) - L_emu
    floor = (1e-14 * np.linalg.norm(L_emu)) ** 2
    rows = []
    for alt, low in level_alternatives(spec):
        La, info, _ = otree.emulate_potrf(A, otree.parse(alt, leaf=leaf), leaf_compute=leaf_compute)
        if info:
            continue
        v = La - L_emu
        vv = float(np.sum(v * v))
        if vv <= floor:
            continue                                  # the recursion never reaches that level
        rows.append((alt, low, np.sqrt(vv), float(np.sum(g * v)) / vv))
    return rows, float(np.linalg.norm(g))


def check_mixed_factor(L, A, spec, leaf, L_emu=None, leaf_compute=None):
    """Raise AssertionError unless L carries the tree's precisions (see the module text).
    Returns the projections for reporting."""
    if L_emu is None:
        L_emu, info, _ = otree.emulate_potrf(A, otree.parse(spec, leaf=leaf), leaf_compute=leaf_compute)
        assert info == 0
    rows, gn = mislevel_projections(L, A, spec, leaf, leaf_compute=leaf_compute, L_emu=L_emu)
    used = [(alt, vn, t) for alt, low, vn, t in rows if low and vn >= NOISE_FLOOR * gn]
    if any(low for _, low, _, _ in rows):
        assert used, f"{spec}: every FP16 alternative is below the FP32 noise ({rows}, |g|={gn:.2e})"
    for alt, vn, t in used:
        assert abs(t) <= T_MAX, f"{spec}: the factor sits t={t:.3f} of the way to {alt} (|v|={vn:.2e}, |g|={gn:.2e})"
    if any(not low for _, low, _, _ in rows):
        L64, _ = dense.cholesky(A)
        r = np.linalg.norm(np.tril(L) - L64) / np.linalg.norm(L_emu - L64)
        assert r >= FP64_DISTANCE_MIN, f"{spec}: the factor is {r:.3f}x the emulator's distance from FP64"
    return rows, gn
