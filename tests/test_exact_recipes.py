"""The integer-operation recipes the kernels use to keep conversions off the
binary64 pipe (csrc/mt_internal.cuh), replayed on their bit patterns:
widen_exact equals the binary32 -> binary64 conversion for every class of
value (normals, subnormals, zeros, infinities, NaNs); i2d_exact equals the
int -> binary64 conversion; rcp_ge1 (a binary32 reciprocal of the leading
24 bits, then two Newton steps with fused multiply-adds) stays within one
unit in the last place of 1/r over the row sums' range."""
import math
import struct
from fractions import Fraction

import numpy as np


def widen_exact(f32_bits: int) -> float:
    u = f32_bits
    ex = u & 0x7F800000
    if ex not in (0, 0x7F800000):  # normal: the high and low words directly
        hi = (u & 0x80000000) | (((u & 0x7FFFFFFF) >> 3) + (896 << 20))
        lo = (u << 29) & 0xFFFFFFFF
        return struct.unpack("<d", struct.pack("<Q", (hi << 32) | lo))[0]
    e, m = (u >> 23) & 0xFF, u & 0x7FFFFF
    if e == 0xFF:
        E, F = 0x7FF, m << 29
    elif e:
        E, F = e + 896, m << 29
    elif m:
        p = m.bit_length() - 1
        E, F = p + 874, (m << (52 - p)) & ((1 << 52) - 1)
    else:
        E, F = 0, 0
    return struct.unpack("<d", struct.pack("<Q", ((u >> 31) << 63) | (E << 52) | F))[0]


def i2d_exact(v: int) -> float:
    if v == 0:
        return 0.0
    a = -v if v < 0 else v
    p = a.bit_length() - 1
    m = (a << (52 - p)) & ((1 << 52) - 1)
    bits = ((1 if v < 0 else 0) << 63) | ((p + 1023) << 52) | m
    return struct.unpack("<d", struct.pack("<Q", bits))[0]


def _fma(a, b, c):
    return float(Fraction(a) * Fraction(b) + Fraction(c))  # one rounding


def rcp_ge1(r: float) -> float:
    u = struct.unpack("<Q", struct.pack("<d", r))[0]
    e = (u >> 52) & 0x7FF
    rf_bits = ((e - 1023 + 127) << 23) | ((u >> 29) & 0x7FFFFF)
    rf = np.frombuffer(struct.pack("<I", rf_bits), dtype=np.float32)[0]
    y0 = np.float32(1.0) / rf  # binary32 reciprocal, rounded to nearest
    y = widen_exact(struct.unpack("<I", struct.pack("<f", float(y0)))[0])
    y = _fma(y, _fma(-r, y, 1.0), y)
    return _fma(y, _fma(-r, y, 1.0), y)


def test_widen_exact_is_the_conversion():
    rng = np.random.default_rng(3)
    bits = list(rng.integers(0, 2 ** 32, 50000, dtype=np.uint64)) + [
        0, 0x80000000, 1, 0x80000001, 0x007FFFFF, 0x00800000, 0x7F7FFFFF, 0x7F800000,
        0xFF800000, 0x7FC00000, 0x3F800000, 0x00400000]
    for b in bits:
        b = int(b)
        f = np.frombuffer(struct.pack("<I", b), dtype=np.float32)[0]
        w, r = widen_exact(b), float(f)
        if math.isnan(r):
            assert math.isnan(w)
        else:
            assert w == r and math.copysign(1.0, w) == math.copysign(1.0, r), hex(b)


def test_i2d_exact_is_the_conversion():
    rng = np.random.default_rng(4)
    vals = [0, 1, -1, 2 ** 30 - 1, -(2 ** 30), 2 ** 31 - 1, -(2 ** 31)]
    vals += [int(v) for v in rng.integers(-(2 ** 31), 2 ** 31, 50000)]
    for v in vals:
        assert i2d_exact(v) == float(v), v


def test_rcp_ge1_within_one_ulp():
    rng = np.random.default_rng(5)
    rs = np.concatenate([[1.0, 1.5, 2.0, 3.0, 1.0 + 2.0 ** -52, 2.0 - 2.0 ** -52],
                         1.0 + rng.exponential(3.0, 3000), 10.0 ** rng.uniform(0, 6, 1000)])
    worst = 0.0
    for r in rs:
        got = rcp_ge1(float(r))
        exact = 1 / Fraction(float(r))
        err = abs(Fraction(got) - exact) / Fraction(math.ulp(float(exact)))
        worst = max(worst, float(err))
    assert worst <= 1.0, worst
