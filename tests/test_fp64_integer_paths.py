"""Host check of the FP64 form's integer replacements of exact double
operations (hd_device.cuh: exact_from_i53, scale_2m53, nonneg_bits,
below_pos_bits), emulated bit for bit in Python and compared with the double
operations they replace, on edge and random values."""
import math
import struct

import numpy as np


def bits(x):
    return struct.unpack("<q", struct.pack("<d", x))[0]


def from_bits(b):
    return struct.unpack("<d", struct.pack("<q", b))[0]


def clz64(a):
    return 64 - a.bit_length()


def exact_from_i53(v):
    s = 1 << 63 if v < 0 else 0
    a = -v if v < 0 else v
    lz = clz64(a)
    mant = (a << (lz - 11)) & ((1 << 52) - 1)
    u = s | ((1023 + 63 - lz) << 52) | mant
    return from_bits(u - (1 << 64) if u >= 1 << 63 else u)


def scale_2m53(x):
    b = bits(x)
    return x if ((b >> 52) & 0x7FF) == 0 else from_bits(b - (53 << 52))


def nonneg_bits(x):
    b = bits(x)
    return b >= 0 or b == -(1 << 63)


def below_pos_bits(x, y):
    return bits(x) < bits(y)


def test_exact_from_i53_matches_conversion():
    edge = [1, -1, 2, 3, -3, 2 ** 52 - 1, 2 ** 52, 2 ** 52 + 1, 2 ** 53 - 1, -(2 ** 53 - 1), 12345, -98765]
    rng = np.random.default_rng(0)
    rand = [int(v) | 1 for v in rng.integers(-(2 ** 53) + 1, 2 ** 53 - 1, 20000)]
    for v in edge + rand:
        assert exact_from_i53(v) == float(v), v


def test_scale_matches_multiply():
    rng = np.random.default_rng(1)
    # the domain: 0, or |x| >= 2^-900 (delta is 0 or at least 2^-900 and |v| >= 1)
    xs = [1.0, -1.0, 0.1 * (2 ** 53 - 1), -0.25, 2.0 ** -900, -(2.0 ** -900), 0.0, -0.0]
    xs += list(rng.uniform(-1e3, 1e3, 20000)) + list(rng.uniform(-1e-250, 1e-250, 2000))
    for x in xs:
        got, want = scale_2m53(x), x * 2.0 ** -53
        assert got == want and math.copysign(1, got) == math.copysign(1, want), x


def test_bit_comparisons_match_double_comparisons():
    rng = np.random.default_rng(2)
    w = 2.0008917450904846
    xs = [0.0, -0.0, w, math.nextafter(w, 0), math.nextafter(w, 10), -w, 1e-300, -1e-300, 5e-324, -5e-324]
    xs += list(rng.uniform(-3, 5, 20000))
    for x in xs:
        assert nonneg_bits(x) == (x >= 0.0), x
        assert below_pos_bits(x, w) == (x < w), x
