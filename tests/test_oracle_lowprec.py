"""Pins of the reduced-precision rounding and the block-scaling rules (oracle/lowprec.py).

FP16 rounding is numpy's cast; it is checked exhaustively against a decoder written
from the binary16 definition.  E4M3 rounding is written in the oracle from the OCP
definition; it is checked exhaustively against its own decoder, against PyTorch's
float8_e4m3fn cast (an independent implementation) and against hand-worked cases.
"""
import os

import numpy as np
import pytest
import torch

from oracle import lowprec

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_f16_every_code_round_trips_and_midpoints_go_to_even():
    codes = np.arange(0, 0x7C00)                       # positive finite codes
    vals = lowprec.decode_f16(codes)
    assert np.all(np.diff(vals) > 0)
    assert np.array_equal(lowprec.round_f16(vals), vals)
    assert np.array_equal(lowprec.round_f16(-vals), -vals)
    mids = 0.5 * (vals[:-1] + vals[1:])                # exact in float64
    got = lowprec.round_f16(mids)
    even = np.where(codes[:-1] % 2 == 0, vals[:-1], vals[1:])
    assert np.array_equal(got, even)
    # just off the midpoint goes to the nearer neighbour
    assert np.array_equal(lowprec.round_f16(np.nextafter(mids, 0)), vals[:-1])
    assert np.array_equal(lowprec.round_f16(np.nextafter(mids, np.inf)), vals[1:])
    assert lowprec.round_f16(np.array([65520.0]))[0] == np.inf


def test_e4m3_every_code_round_trips_and_midpoints_go_to_even():
    codes = np.arange(0, 0x7F)                          # positive finite codes (0x7F is NaN)
    vals = lowprec.decode_e4m3(codes)
    assert vals[-1] == 448.0 and vals[1] == 2.0 ** -9 and vals[8] == 2.0 ** -6
    assert np.all(np.diff(vals) > 0)
    assert np.array_equal(lowprec.round_e4m3(vals), vals)
    assert np.array_equal(lowprec.round_e4m3(-vals), -vals)
    mids = 0.5 * (vals[:-1] + vals[1:])
    even = np.where(codes[:-1] % 2 == 0, vals[:-1], vals[1:])
    assert np.array_equal(lowprec.round_e4m3(mids), even)
    assert np.array_equal(lowprec.round_e4m3(np.nextafter(mids, 0)), vals[:-1])
    assert np.array_equal(lowprec.round_e4m3(np.nextafter(mids, np.inf)), vals[1:])
    assert np.isnan(lowprec.decode_e4m3(np.array([0x7F]))[0])


def test_e4m3_matches_torch_cast():
    rng = np.random.default_rng(5)
    x = np.concatenate([
        rng.standard_normal(20000) * 10.0 ** rng.uniform(-4, 2.5, 20000),
        0.5 * (lowprec.decode_e4m3(np.arange(0, 0x7E)) + lowprec.decode_e4m3(np.arange(1, 0x7F))),
    ])
    x = x[np.abs(x) < 464.0]                            # torch's cast is not saturating
    ref = torch.from_numpy(x).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert np.array_equal(lowprec.round_e4m3(x, satfinite=False), ref)
    assert np.array_equal(lowprec.round_e4m3(x), ref)
    assert lowprec.round_e4m3(np.array([1e6, -500.0])).tolist() == [448.0, -448.0]


def _cases():
    out = []
    with open(os.path.join(GOLD, "rounding_cases.txt")) as f:
        for line in f:
            if not line.strip() or line.startswith("#"):
                continue
            fmt, x, y, _why = [t.strip() for t in line.split("|")]
            out.append((fmt, float(x), float(y)))
    return out


@pytest.mark.parametrize("fmt,x,y", _cases())
def test_hand_worked_rounding_cases(fmt, x, y):
    f = lowprec.round_f16 if fmt == "f16" else lowprec.round_e4m3
    assert f(np.array([x]))[0] == y


def test_f16_alpha_rule():
    B = np.array([[1.0, -3.0], [2.0, 0.5]])
    assert lowprec.f16_alpha(B) == 1.0
    q, a = lowprec.quantize_f16(B)
    assert a == 1.0 and np.array_equal(q, B)
    B = np.array([[1.0, -131008.0], [2.0, 0.5]])        # amax = 2 * 65504
    assert lowprec.f16_alpha(B) == 2.0
    q, a = lowprec.quantize_f16(B)
    assert a == 2.0 and np.array_equal(q * a, B)        # every entry halves exactly
    B = np.array([[1e6]])
    q, a = lowprec.quantize_f16(B)
    assert a == 1e6 / 65504 and q[0, 0] == 65504.0


def test_e4m3_tile_scale_rule():
    for amax in [1e-9, 3.7e-3, 0.5, 1.0, 448.0, 449.0, 1e5]:
        s = lowprec.e4m3_tile_scale(amax)
        m, _ = np.frexp(s)
        assert m == 0.5                                  # power of two
        assert amax / s <= 448.0 < 2 * amax / s          # the smallest such power of two
    assert lowprec.e4m3_tile_scale(448.0) == 1.0
    assert lowprec.e4m3_tile_scale(0.0) == 1.0


def test_e4m3_tiles_use_the_global_grid():
    M = np.zeros((256, 256))
    M[130, 5] = 1.0                                      # tile (1, 0)
    M[200, 140] = 96.0                                   # tile (1, 1); 96/0.25 = 384 is an E4M3 value
    q, s = lowprec.quantize_e4m3_tiles(M, 128, 0, 128, 256, tile=128)
    assert s[2, 5] == lowprec.e4m3_tile_scale(1.0)
    assert s[72, 140] == lowprec.e4m3_tile_scale(96.0)
    assert q[2, 5] * s[2, 5] == 1.0 and q[72, 140] * s[72, 140] == 96.0
    # a sub-block read through an offset sees the same scales
    q2, s2 = lowprec.quantize_e4m3_tiles(M, 160, 100, 64, 100, tile=128)
    assert s2[40, 40] == s[72, 140] and s2[0, 0] == s[32, 100]


# ---------------------------------------------------------------------------------------
# TF32 rounding and the error-corrected TF32 split (FP32 levels on tensor cores)
# ---------------------------------------------------------------------------------------
def _tf32_by_bits(x32: np.ndarray) -> np.ndarray:
    """Round-to-nearest-even on the binary32 bit pattern: keep 10 of the 23 mantissa bits."""
    b = x32.astype(np.float32).view(np.uint32).astype(np.uint64)
    b = b + 0x0FFF + ((b >> 13) & 1)
    b = b & 0xFFFFE000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def test_tf32_rounding_matches_the_bit_pattern_rule():
    rng = np.random.default_rng(11)
    x = (rng.standard_normal(200000) * np.exp2(rng.integers(-120, 120, 200000))).astype(np.float32)
    assert np.array_equal(lowprec.round_tf32(x.astype(np.float64)), _tf32_by_bits(x))
    # exact midpoints: low 13 bits = 0x1000, bit 13 even and odd
    base = (rng.integers(0x00800000, 0x7E000000, 4000).astype(np.uint32) & np.uint32(0xFFFFE000))
    mids = (base | np.uint32(0x1000)).view(np.float32)
    got = lowprec.round_tf32(mids.astype(np.float64))
    assert np.array_equal(got, _tf32_by_bits(mids))
    even = np.where((base >> 13) & 1, (base + np.uint32(0x2000)).view(np.float32), base.view(np.float32))
    assert np.array_equal(got, even.astype(np.float64))


def test_tf32_values_round_trip():
    e = np.arange(1, 255, dtype=np.uint32)
    m = np.arange(0, 1024, dtype=np.uint32)
    codes = ((e[:, None] << 23) | (m[None, :] << 13)).ravel()
    v = codes.view(np.float32).astype(np.float64)
    assert np.array_equal(lowprec.round_tf32(v), v)
    assert np.array_equal(lowprec.round_tf32(-v), -v)


def test_tf32_split_reconstructs_to_22_bits():
    rng = np.random.default_rng(12)
    x = rng.standard_normal(100000) * np.exp2(rng.integers(-60, 60, 100000))
    hi, lo = lowprec.split_tf32(x)
    x32 = lowprec.round_f32(x)
    assert np.array_equal(lowprec.round_tf32(hi), hi) and np.array_equal(lowprec.round_tf32(lo), lo)
    assert np.all(np.abs(x32 - hi - lo) <= 2.0 ** -22 * np.abs(x32))
    assert np.all(np.abs(lo) <= 2.0 ** -11 * np.abs(hi))
    # a value with at most 11 significant bits has no low part
    small = np.round(rng.uniform(-1024, 1024, 1000)) * np.exp2(rng.integers(-30, 30, 1000))
    assert not lowprec.split_tf32(small)[1].any()


def test_tf32x3_product_is_exact_on_small_integers():
    rng = np.random.default_rng(13)
    X = rng.integers(-1000, 1001, (40, 300)).astype(np.float64)
    Y = rng.integers(-1000, 1001, (30, 300)).astype(np.float64)
    assert np.array_equal(lowprec.gemm_tf32x3(X, Y), X @ Y.T)


def test_tf32x3_error_bound_and_the_correction_terms():
    """|x y - (hx hy + hx ly + lx hy)| <= 3 2^-22 |x y| per term (la lb dropped, two
    representation errors of 2^-22): the split product stays inside 3.01 2^-22 |X||Y|^T of the
    exact product of the FP32 operands.  Dropping the correction terms (plain TF32) or
    either one of them leaves that bound."""
    rng = np.random.default_rng(14)
    X = lowprec.round_f32(rng.standard_normal((64, 512)))
    Y = lowprec.round_f32(rng.standard_normal((48, 512)))
    exact = X @ Y.T
    bound = 3.01 * 2.0 ** -22 * (np.abs(X) @ np.abs(Y).T)
    assert np.all(np.abs(lowprec.gemm_tf32x3(X, Y) - exact) <= bound)
    hx, lx = lowprec.split_tf32(X)
    hy, ly = lowprec.split_tf32(Y)
    for wrong in (hx @ hy.T, hx @ hy.T + hx @ ly.T, hx @ hy.T + lx @ hy.T, hx @ hy.T + hx @ ly.T - lx @ hy.T):
        assert np.any(np.abs(wrong - exact) > bound)
