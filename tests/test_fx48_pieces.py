"""The k-means++ seeding's fixed-point weights on the FMA pipe (CPU emulation).

The seeding draws a centre with probability proportional to D^2 by exact
fixed-point sums of fx48(d) = floor(d 2^48) (the oracle's definition).  The
cluster seeding kernel forms fx48(d) for 0 <= d < 2^10 from three binary32
round-toward-zero fused multiply-adds onto 2^23 and two exact remainders:

    y1 = rz(d 2^13 + 2^23),         h = y1 - 2^23
    r1 = d - h 2^-13                (exact)
    y2 = rz(r1 2^36 + 2^23),        m = y2 - 2^23
    r2 = r1 - m 2^-36               (exact)
    y3 = rz(r2 2^48 + 2^23),        l = y3 - 2^23
    fx48(d) = h 2^35 + m 2^12 + l

Here every step is evaluated in exact rational arithmetic and rounded to
binary32 the way the instruction rounds, and the identity is checked on
values spread over every exponent the range holds, subnormals and the
boundaries included; the bit-pattern sums with their biases removed are
checked against the plain integer sum.
"""
from fractions import Fraction

import numpy as np

F = Fraction


def to_f32_rz(x: Fraction) -> Fraction:
    """Round a non-negative rational toward zero to binary32 (no overflow here)."""
    if x == 0:
        return F(0)
    e = x.numerator.bit_length() - x.denominator.bit_length()
    while F(2) ** e > x:
        e -= 1
    while F(2) ** (e + 1) <= x:
        e += 1
    ulp = F(2) ** max(e - 23, -149)
    return (x // ulp) * ulp


def to_f32_rn(x: Fraction) -> Fraction:
    v = float(np.float32(float(x)))
    assert F(v) == x, "a remainder the kernel takes as exact is not"
    return x


def pieces(d: float):
    dq = F(float(np.float32(d)))
    two23 = F(2) ** 23
    y1 = to_f32_rz(dq * F(2) ** 13 + two23)
    h = y1 - two23
    r1 = to_f32_rn(dq - h * F(2) ** -13)
    y2 = to_f32_rz(r1 * F(2) ** 36 + two23)
    m = y2 - two23
    r2 = to_f32_rn(r1 - m * F(2) ** -36)
    y3 = to_f32_rz(r2 * F(2) ** 48 + two23)
    l = y3 - two23
    for v in (h, m, l):
        assert v.denominator == 1 and 0 <= v < two23
    return int(h), int(m), int(l), dq


def bits(v: int) -> int:
    return 0x4B000000 + v    # binary32 pattern of 2^23 + v, 0 <= v < 2^23


def test_pieces_equal_the_fixed_point_definition():
    rng = np.random.default_rng(0)
    vals = [0.0, 2.0 ** -149, 2.0 ** -126, 2.0 ** -48, 2.0 ** -36, 2.0 ** -13, 1.0, 1023.9999, 2.0 ** 10 * (1 - 2 ** -24)]
    vals += list(2.0 ** rng.uniform(-149, 10, 3000))
    vals += list(rng.uniform(0, 1024, 1000))
    for d in vals:
        h, m, l, dq = pieces(d)
        assert h * 2 ** 35 + m * 2 ** 12 + l == (dq * F(2) ** 48) // 1


def test_biased_sums_recover_the_integer_sum():
    rng = np.random.default_rng(1)
    for _ in range(200):
        ds = np.float32(2.0 ** rng.uniform(-60, 10, 36))
        ds[rng.random(36) < 0.2] = 0.0          # padding points add fx48(0)
        ah = am = al = 0
        want = 0
        for d in ds:
            h, m, l, dq = pieces(float(d))
            ah, am, al = (ah + bits(h)) % 2 ** 32, (am + bits(m)) % 2 ** 32, (al + bits(l)) % 2 ** 32
            want += int((dq * F(2) ** 48) // 1)
        bias = (36 * 0x4B000000) % 2 ** 32
        got = ((ah - bias) % 2 ** 32 << 35) + ((am - bias) % 2 ** 32 << 12) + (al - bias) % 2 ** 32
        assert got == want and got < 2 ** 64
