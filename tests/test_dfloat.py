"""The FP64 table march carries everything that only feeds the fields in double-float pairs
(csrc/dfloat.h) and moves values between doubles and pairs with integer operations, so that the
FP64 unit does only the two deciding operations of a segment. Those conversions are replayed here
operation by operation (IEEE single precision, bit patterns as integers) and checked against exact
rationals: a double split into a pair (head = its leading 24 bits, tail = the rest rounded), its
mantissa split, and a pair rounded back to a double by adding the tail as an integer count of the
head's last place. That lands within one unit of the last place of the exact sum, also where a
positive tail carries to the next power of two; where the renormalised head is a power of two and
the tail negative, the sum lies in the binade below, whose last place is half as large, so half the
tail is lost: at most 2^-26 of the value, the bound the kernel states."""
import math
import struct
from fractions import Fraction

import numpy as np


def f32(x) -> float:
    return struct.unpack("<f", struct.pack("<f", float(x)))[0]


def fbits(x: float) -> int:
    return struct.unpack("<I", struct.pack("<f", x))[0]


def bits_f(u: int) -> float:
    return struct.unpack("<f", struct.pack("<I", u & 0xFFFFFFFF))[0]


def dbits(x: float) -> int:
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def bits_d(b: int) -> float:
    return struct.unpack("<d", struct.pack("<Q", b & 0xFFFFFFFFFFFFFFFF))[0]


def add(a, b):
    return f32(Fraction(a) + Fraction(b))            # exact sum rounded once (float() rounds to nearest)


def mul(a, b):
    return f32(Fraction(a) * Fraction(b))


def u2f(v: int) -> float:
    return f32(v)


def f2i_rn(x: float) -> int:
    return int(round(x))                               # ties to even, as cvt.rni


def df_of(x: float):
    b = dbits(x)
    hw, lw = b >> 32, b & 0xFFFFFFFF
    e = hw >> 20
    if e < 897:
        return 0.0, 0.0
    h = bits_f(((e - 896) << 23) | ((hw & 0xFFFFF) << 3) | (lw >> 29))
    lo = mul(u2f(lw & 0x1FFFFFFF), bits_f((e - 948) << 23)) if e >= 949 else 0.0
    return h, lo


def df_of_len(x: float):
    b = dbits(x)
    hw, lw = b >> 32, b & 0xFFFFFFFF
    e = hw >> 20
    return (bits_f(((e - 896) << 23) | ((hw & 0xFFFFF) << 3) | (lw >> 29)),
            mul(u2f(lw & 0x1FFFFFFF), bits_f((e - 948) << 23)))


def df_mant(x: float):
    b = dbits(x)
    hw, lw = b >> 32, b & 0xFFFFFFFF
    ex = (hw >> 20) - 1023
    h = bits_f(0x3F800000 | ((hw & 0xFFFFF) << 3) | (lw >> 29))
    return (h, mul(u2f(lw & 0x1FFFFFFF), 2.0 ** -52)), ex


def fast_two_sum(a, b):
    s = add(a, b)
    return s, add(b, -add(s, -a))


def df_to_double_pos(h: float, lo: float, e2: int):
    """The integer path; None where the kernel takes its FP64 fallback."""
    nh, nl = fast_two_sum(h, lo)
    u = fbits(nh)
    eh = (u >> 23) - 127
    if eh < -75 or eh > 126 or (u >> 31):
        return None
    hi = ((u >> 3) + ((896 + e2) << 20)) & 0xFFFFFFFF
    b = (hi << 32) | ((u << 29) & 0xFFFFFFFF)
    units = f2i_rn(mul(nl, bits_f((179 - eh) << 23)))
    return bits_d(b + units)


def ulp(x: float) -> Fraction:
    return Fraction(2) ** (math.frexp(x)[1] - 53)


def val(h, lo, e2=0):
    return (Fraction(h) + Fraction(lo)) * Fraction(2) ** e2


def test_double_to_pair():
    rng = np.random.default_rng(5)
    xs = [float(v) for v in 10.0 ** rng.uniform(-20, 30, 2000)] + [1.0, 2.0 ** -74, 2.0 ** 126, 1.7320508075688772]
    for x in xs:
        h, lo = df_of(x)
        # the head is x truncated to 24 significant bits, the pair within 2^-48 of x
        assert dbits(float(h)) == dbits(x) & ~((1 << 29) - 1), x
        assert abs(val(h, lo) - Fraction(x)) <= Fraction(x) * Fraction(1, 2 ** 48), x
        assert df_of_len(x) == (h, lo), x
    # below 2^-74 the head alone, below 2^-126 nothing
    h, lo = df_of(3.0 * 2.0 ** -80)
    assert lo == 0.0 and abs(Fraction(h) - Fraction(3.0 * 2.0 ** -80)) <= Fraction(3.0 * 2.0 ** -80) / 2 ** 23
    assert df_of(2.0 ** -127) == (0.0, 0.0)


def test_mantissa_split():
    rng = np.random.default_rng(6)
    for x in [float(v) for v in 10.0 ** rng.uniform(-30, 30, 2000)]:
        (h, lo), ex = df_mant(x)
        assert 1.0 <= h < 2.0
        assert abs(val(h, lo) * Fraction(2) ** ex - Fraction(x)) <= Fraction(x) / 2 ** 48, x


def test_pair_to_double():
    rng = np.random.default_rng(7)
    cases = []
    for _ in range(3000):
        h = f32(float(rng.uniform(1, 2)) * 2.0 ** int(rng.integers(-60, 60)))
        lo = f32(h * float(rng.uniform(-1, 1)) * 2.0 ** -22)       # unnormalised, as a product leaves it
        cases.append((h, lo, int(rng.integers(-200, 200))))
    # sums that cross a power of two: the head exactly 2^k with a negative tail (a borrow out of the
    # binade), or just below 2^k with a positive tail (a carry into the next)
    for k in range(-40, 41, 7):
        for t in (-2.0 ** -30, -2.0 ** -25, -2.0 ** -24, 2.0 ** -26):
            cases.append((2.0 ** k, f32(t * 2.0 ** k), 3))
        below = f32(np.nextafter(np.float32(2.0 ** k), np.float32(0)))
        cases.append((below, f32(2.0 ** (k - 24)), -5))
        cases.append((below, f32(2.0 ** (k - 23)), 0))
    corner = 0
    for h, lo, e2 in cases:
        got = df_to_double_pos(h, lo, e2)
        assert got is not None
        exact = val(h, lo, e2)
        nh, nl = fast_two_sum(h, lo)
        if fbits(nh) & 0x7FFFFF == 0 and nl < 0:
            # the borrow into the binade below: half the tail is lost, nothing more
            corner += 1
            err = abs(Fraction(got) - exact)
            assert err <= abs(Fraction(nl)) * Fraction(2) ** e2 / 2 + ulp(got), (h, lo, e2)
            assert err <= Fraction(nh) * Fraction(2) ** e2 / 2 ** 26, (h, lo, e2)
        else:
            assert abs(Fraction(got) - exact) <= ulp(got), (h, lo, e2)
    assert corner >= 20


def widen_scaled(x: float, e2: int) -> float:
    """Float to double times 2^e2 by re-biasing the exponent and shifting the mantissa."""
    u = fbits(x)
    mag = u & 0x7FFFFFFF
    if (mag - 0x00800000) & 0xFFFFFFFF < 0x7F000000:
        hi = (((mag >> 3) + ((896 + e2) << 20)) | (u & 0x80000000)) & 0xFFFFFFFF
        return bits_d((hi << 32) | ((u << 29) & 0xFFFFFFFF))
    if mag == 0:
        return 0.0
    return bits_d(dbits(float(x)) + e2 * (1 << 52))


def test_float_widening_is_exact():
    # the FP32 march widens each deposit for its FP64 atomic by the same bit operations (e2 = 0), and
    # the double-float fallback rounds its two widened parts: the result must be x 2^e2 exactly, for
    # normal and subnormal floats of either sign
    rng = np.random.default_rng(8)
    xs = [f32(float(v) * s) for v, s in zip(10.0 ** rng.uniform(-37, 38, 3000), rng.choice([-1.0, 1.0], 3000))]
    xs += [bits_f(v) for v in (1, 7, 0x007FFFFF, 0x00800000, 0x7F7FFFFF, 0x80000001, 0x80800000)]
    for x in xs:
        for e2 in (-300, -64, 0, 64, 300):
            assert Fraction(widen_scaled(x, e2)) == Fraction(x) * Fraction(2) ** e2, (x, e2)
    assert widen_scaled(0.0, 17) == 0.0
