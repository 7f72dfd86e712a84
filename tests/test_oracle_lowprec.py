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
