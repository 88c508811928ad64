"""Exactness arguments of the split-precision forms, checked on the host.

Both forms split fixed-point values into six signed 8-bit digits at bit
positions 61 - 8k (k = 1..6) and sum the digit products of one level
l = i + k over K terms in FP32 on the tensor cores. A level is exact if its
largest possible magnitude is below 2^24 (FP32 significand); the tcgen05
form also reads the second product's levels with the add-magic-number
conversion, which is exact below 2^22. These tests recompute the bounds from
the digit ranges and check the balanced-digit identity the tcgen05 form uses
(digit k = byte of Z + C at bit 61 - 8k, minus 128) on random values,
including the extremes. No GPU is involved."""

import numpy as np

S = 6            # digits per operand
LEVELS = 7       # kept levels, 0-based l = i + k <= 6
OFFSET = sum(1 << (68 - 8 * k) for k in range(1, 7)) + (1 << 12)


def level_bound(first_a, first_b, K):
    """Largest |sum over K terms of the level's digit products| when operand
    a's first digit is at most first_a (others 128), likewise b."""
    worst = 0
    for lv in range(LEVELS):
        s = 0
        for i in range(S):
            k = lv - i
            if 0 <= k < S:
                s += (first_a if i == 0 else 128) * (first_b if k == 0 else 128)
        worst = max(worst, s * K)
    return worst


def test_first_product_levels_exact_in_fp32():
    # Z (first digit <= 256) against V' (<= 2^60: first digit <= 128), K = window rows <= 96
    assert level_bound(128, 256, 96) < 2 ** 24
    assert level_bound(128, 256, 64) < 2 ** 24  # b = 32: 63 rows padded to 64


def test_second_product_levels_below_magic_range():
    # U' and W both scaled to <= 2^60 (first digits <= 128), K = 32 reflectors
    assert level_bound(128, 128, 32) < 2 ** 22
    # with first digits up to 256 on both sides (scale 2^61) a level could
    # reach the edge of the range exactly: why the operands are kept at 2^60
    assert level_bound(256, 256, 32) == 2 ** 22


def balanced_digits(x):
    """Digits d_1..d_6 of x (|x| <= 2^61) read from the offset form, as the
    tcgen05 kernel does, and the remainder."""
    y = x + OFFSET
    d = [(y >> 53) - 128]
    for k in range(2, 7):
        d.append(((y >> (61 - 8 * k)) & 0xFF) - 128)
    rem = x - sum(dk << (61 - 8 * k) for k, dk in enumerate(d, start=1))
    return d, rem


def test_balanced_digit_identity_and_ranges():
    rng = np.random.default_rng(5)
    vals = [0, 1, -1, 2 ** 61, -(2 ** 61), 2 ** 60, -(2 ** 60), 2 ** 61 - 1, 2 ** 12, -(2 ** 12), 2 ** 12 - 1]
    vals += [int(v) for v in rng.integers(-(2 ** 61), 2 ** 61, size=2000, dtype=np.int64)]
    vals += [int(v) >> int(s) for v, s in zip(rng.integers(-(2 ** 61), 2 ** 61, size=500, dtype=np.int64),
                                               rng.integers(0, 60, size=500))]
    for x in vals:
        d, rem = balanced_digits(x)
        assert -(2 ** 12) <= rem < 2 ** 12, (x, rem)           # half a unit of the last digit
        assert -256 <= d[0] <= 256, (x, d)
        assert all(-128 <= dk <= 127 for dk in d[1:]), (x, d)
        if abs(x) <= 2 ** 60:
            assert -128 <= d[0] <= 128, (x, d)               # operands scaled to 2^60
        for dk in d:                                          # every digit is exact in BF16
            f = np.float32(dk)
            assert (f.view(np.uint32) & 0xFFFF) == 0 and float(f) == dk


def test_fp32_magic_conversions():
    # integer-valued floats below 2^22: x + 1.5 * 2^23 keeps unit spacing
    for v in [0, 1, -1, 2 ** 22 - 1, -(2 ** 22), 12345, -777777]:
        f = np.float32(v)
        t = (f + np.float32(12582912.0)).view(np.int32) - 0x4B400000
        assert t == v
    # the digit-to-float form: byte e in the mantissa of 2^23, minus 2^23 + 128
    for e in range(256):
        f = np.array([0x4B000000 | e], dtype=np.uint32).view(np.float32)[0] - np.float32(8388736.0)
        assert float(f) == e - 128
