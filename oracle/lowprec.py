"""Rounding to the reduced precisions used by the precision tree, and block scaling.

Sec. 3.3 assigns FP16 (and, in the large FP8 configuration, FP8 E4M3) to
the off-diagonal GEMM operands; Sec. 3.4 rescales each operand block into the
format's range before the low-precision product and scales the result back.

  * FP32: IEEE-754 binary32, round to nearest even (numpy's float64->float32 cast).
  * FP16: IEEE-754 binary16, round to nearest even, overflow to +-inf
    (numpy's float64->float16 cast converts directly from double, one rounding).
  * E4M3: OCP 8-bit floating point, "E4M3FN": 1 sign, 4 exponent bits (bias 7),
    3 mantissa bits; no infinities; the all-ones code is NaN; largest finite
    value 448 = 1.75 * 2^8; smallest normal 2^-6; subnormals k * 2^-9, k = 1..7.
    Written here from that definition (numpy has no FP8 type); saturating
    ("satfinite") rounding clamps finite overflow to +-448.

  * TF32: binary32's exponent range with 10 explicit mantissa bits (11 significant bits),
    the tensor-core input format of the FP32 levels when they run on tensor cores; round to
    nearest even, written here from that definition.
  * TF32 split (Ootomo and Yokota, 2022, error-corrected single-precision GEMM on tensor
    cores; the remedy for FP32 diagonal regions named by the paper's Sec. 5): an FP32
    operand x becomes hi = tf32(x) and lo = tf32(x - hi); the product a b is taken as
    hi_a hi_b + (hi_a lo_b + lo_a hi_b), dropping lo_a lo_b.  |x - hi - lo| <= 2^-22 |x|.

Scaling rules
  * FP16 (Sec. 3.4): alpha = max(1, ||B||_inf / R_max) with R_max = 65504 and
    ||B||_inf read as the largest |b_ij| of the operand block; the block is
    computed on as B / alpha and the product is multiplied back by alpha.
  * E4M3: one power-of-two scale per 128 x 128 tile, s = 2^ceil(log2(amax/448))
    (two-sided, so that small tiles are scaled up out of the subnormal range);
    s = 1 for an all-zero tile.
"""
from __future__ import annotations

import numpy as np

F16_MAX = 65504.0
E4M3_MAX = 448.0


def round_f32(x: np.ndarray) -> np.ndarray:
    return np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float64)


def round_tf32(x: np.ndarray) -> np.ndarray:
    """Round to TF32 (11 significant bits, binary32's exponent range), nearest even."""
    x = np.asarray(x, dtype=np.float64)
    ax = np.abs(x)
    _, ex = np.frexp(ax)                      # ax = f * 2^ex, f in [0.5, 1)
    e = np.maximum(ex - 1, -126)              # binade exponent (binary32's subnormal binade)
    quantum = np.exp2((e - 10).astype(np.float64))
    r = np.rint(ax / quantum) * quantum       # power-of-two divide: exact; rint: ties to even
    r = np.where(ax == 0.0, 0.0, r)
    out = np.copysign(r, x)
    return np.where(np.isfinite(x), out, x)


def split_tf32(x: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """(hi, lo) of the FP32 rounding of x: hi = tf32(x32), lo = tf32(x32 - hi)."""
    x32 = round_f32(x)
    hi = round_tf32(x32)
    return hi, round_tf32(x32 - hi)           # x32 - hi is exact in binary32


def gemm_tf32x3(X: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """X Y^T from the TF32 splits of X and Y: hi hi^T + (hi lo^T + lo hi^T), summed in float64."""
    hx, lx = split_tf32(X)
    hy, ly = split_tf32(Y)
    return hx @ hy.T + (hx @ ly.T + lx @ hy.T)


def round_f16(x: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        return np.asarray(x, dtype=np.float64).astype(np.float16).astype(np.float64)


def decode_f16(code: np.ndarray) -> np.ndarray:
    """Value of binary16 bit patterns, from the format definition (pins ``round_f16``)."""
    code = np.asarray(code, dtype=np.int64)
    s = np.where(code >> 15 & 1, -1.0, 1.0)
    e = (code >> 10) & 0x1F
    m = (code & 0x3FF).astype(np.float64)
    val = np.where(e == 0, m * 2.0 ** -24, (1.0 + m / 1024.0) * np.exp2(e.astype(np.float64) - 15.0))
    val = np.where(e == 31, np.where(m == 0, np.inf, np.nan), val)
    return s * val


def decode_e4m3(code: np.ndarray) -> np.ndarray:
    """Value of E4M3FN bit patterns, from the format definition."""
    code = np.asarray(code, dtype=np.int64)
    s = np.where(code >> 7 & 1, -1.0, 1.0)
    e = (code >> 3) & 0xF
    m = (code & 0x7).astype(np.float64)
    val = np.where(e == 0, m * 2.0 ** -9, (1.0 + m / 8.0) * np.exp2(e.astype(np.float64) - 7.0))
    val = np.where((e == 15) & (m == 7), np.nan, val)
    return s * val


def round_e4m3(x: np.ndarray, satfinite: bool = True) -> np.ndarray:
    """Round float64 values to E4M3FN, nearest even, directly from double (one rounding)."""
    x = np.asarray(x, dtype=np.float64)
    ax = np.abs(x)
    _, ex = np.frexp(ax)                      # ax = f * 2^ex, f in [0.5, 1)
    e = np.maximum(ex - 1, -6)                # binade exponent, subnormal binade clamps at -6
    quantum = np.exp2((e - 3).astype(np.float64))
    r = np.rint(ax / quantum) * quantum       # ax / quantum is exact (power-of-two divide)
    if satfinite:
        r = np.minimum(r, E4M3_MAX)
    else:
        # beyond the largest finite value the FN format has no infinity: values that do not
        # round to 448 become NaN
        r = np.where(ax >= 464.0, np.nan, r)
    r = np.where(ax == 0.0, 0.0, r)
    out = np.copysign(r, x)
    return np.where(np.isnan(x), np.nan, out)


def f16_alpha(block: np.ndarray) -> float:
    """Sec. 3.4 scaling factor alpha = max(1, amax / R_max) for an FP16 operand block."""
    if block.size == 0:
        return 1.0
    amax = float(np.max(np.abs(block)))
    return max(1.0, amax / F16_MAX)


def quantize_f16(block: np.ndarray) -> tuple[np.ndarray, float]:
    """(round_f16(B / alpha), alpha) for one FP16 GEMM operand block."""
    alpha = f16_alpha(block)
    if alpha == 1.0:
        return round_f16(block), 1.0
    return round_f16(block / alpha), alpha


def e4m3_tile_scale(amax: float) -> float:
    """Power-of-two scale s = 2^ceil(log2(amax / 448)) of one E4M3 tile (1 for a zero tile)."""
    if amax == 0.0 or not np.isfinite(amax):
        return 1.0
    ratio = amax / E4M3_MAX
    f, ex = np.frexp(ratio)                   # ratio = f * 2^ex, f in [0.5, 1)
    k = ex - 1 if f == 0.5 else ex            # ceil(log2(ratio))
    return float(np.ldexp(1.0, int(k)))


def quantize_e4m3_tiles(M: np.ndarray, r0: int, c0: int, rows: int, cols: int,
                        tile: int = 128) -> tuple[np.ndarray, np.ndarray]:
    """E4M3 codes-as-values and per-element scales for M[r0:r0+rows, c0:c0+cols].

    Tiles are the cells of the global ``tile`` x ``tile`` grid of M (so one element
    always has one scale, whichever operand block it is read through); the amax of
    a tile is taken over the part of the tile inside the lower triangle of the
    factor, i.e. over M's entries with row >= col.
    Returns (q, s) with q = round_e4m3(x / s) and s the element's tile scale.
    """
    sub = M[r0:r0 + rows, c0:c0 + cols]
    scale = np.empty_like(sub)
    for ti in range(r0 // tile, (r0 + rows - 1) // tile + 1 if rows else r0 // tile):
        for tj in range(c0 // tile, (c0 + cols - 1) // tile + 1 if cols else c0 // tile):
            gr0, gr1 = ti * tile, min((ti + 1) * tile, M.shape[0])
            gc0, gc1 = tj * tile, min((tj + 1) * tile, M.shape[1])
            t = M[gr0:gr1, gc0:gc1]
            ii = np.arange(gr0, gr1)[:, None]
            jj = np.arange(gc0, gc1)[None, :]
            amax = float(np.max(np.where(ii >= jj, np.abs(t), 0.0))) if t.size else 0.0
            s = e4m3_tile_scale(amax)
            lr0, lr1 = max(gr0, r0) - r0, min(gr1, r0 + rows) - r0
            lc0, lc1 = max(gc0, c0) - c0, min(gc1, c0 + cols) - c0
            scale[lr0:lr1, lc0:lc1] = s
    return round_e4m3(sub / scale), scale
