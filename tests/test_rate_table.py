"""The FP64 table march evaluates the Eq. 1 factor g(y) = (1 - e^{-y}) / y below y = 2
in double-float arithmetic from a Taylor table (csrc/rate_table.h). The table must be the
one its generator derives, and the evaluation, replayed here operation by operation in
IEEE single precision (fused multiply-adds rounded once), must stay within 1e-14 of g
relative, checked against 40-digit arithmetic (the tail additions of a double-float sum
round at about 2^-48 of the value each), so that the march's deposits keep their 1e-12
agreement with the FP64 oracle with room to spare."""
import math
import os
import re
import struct
import sys
from fractions import Fraction

import numpy as np
import pytest

mp = pytest.importorskip("mpmath")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2512_12466_gb300", "csrc")


def header_rows():
    src = open(os.path.join(CSRC, "rate_table.h")).read()
    body = src[src.index("kRateTable[512 * 8] = {") + len("kRateTable[512 * 8] = {"):src.index("};")]
    vals = [float.fromhex(v) for v in re.findall(r"-?0x[0-9a-fA-F.]+p[-+]?\d+", body)]
    assert len(vals) == 512 * 8
    return [vals[8 * j:8 * j + 8] for j in range(512)]


def round32(q: Fraction) -> float:
    """q rounded to the nearest float32 (ties to even), for normal results."""
    if q == 0:
        return 0.0
    sign = -1 if q < 0 else 1
    q = abs(q)
    e = math.floor(math.log2(q.numerator) - math.log2(q.denominator))
    while Fraction(2) ** e > q:
        e -= 1
    while Fraction(2) ** (e + 1) <= q:
        e += 1
    scale = Fraction(2) ** (23 - e)
    m = q * scale
    fl = math.floor(m)
    rem = m - fl
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and fl % 2 == 1):
        fl += 1
    return sign * float(Fraction(fl) / scale)


def add(a, b):
    return round32(Fraction(a) + Fraction(b))


def mul(a, b):
    return round32(Fraction(a) * Fraction(b))


def fma(a, b, c):
    return round32(Fraction(a) * Fraction(b) + Fraction(c))


def fast_two_sum(a, b):
    s = add(a, b)
    return s, add(b, -add(s, -a))


def two_sum(a, b):
    s = add(a, b)
    bb = add(s, -a)
    return s, add(add(a, -add(s, -bb)), add(b, -bb))


def df_of(y: float):
    """The double y split as the kernel does: head = leading 24 bits, tail = the rest rounded."""
    b = struct.unpack("<q", struct.pack("<d", y))[0]
    h = struct.unpack("<d", struct.pack("<q", b & ~((1 << 29) - 1)))[0]
    return h, round32(Fraction(y) - Fraction(h))


def rate_factor(rows, y: float):
    xh, xl = df_of(y)
    j = min(int(mul(xh, 256.0)), 511)
    c0h, c0l, c1h, c1l, c2h, c2l, c3, c4 = rows[j]
    y0 = mul(add(float(j), 0.5), 0.00390625) if j else 0.0
    rh, rl = two_sum(add(xh, -y0), xl)
    t = fma(c4, rh, c3)
    uh, ul = fast_two_sum(c2h, fma(rh, t, fma(rl, t, c2l)))
    p = mul(rh, uh)
    pe = fma(rl, uh, fma(rh, ul, fma(rh, uh, -p)))
    vh, vl = fast_two_sum(c1h, p)
    vl = add(vl, add(pe, c1l))
    p = mul(rh, vh)
    pe = fma(rl, vh, fma(rh, vl, fma(rh, vh, -p)))
    gh, gl = fast_two_sum(c0h, p)
    gl = add(gl, add(pe, c0l))
    return Fraction(gh) + Fraction(gl)


def g_exact(y):
    y = mp.mpf(y)
    return -mp.expm1(-y) / y if y != 0 else mp.mpf(1)


def test_table_is_the_generators():
    sys.path.insert(0, CSRC)
    import gen_rate_table as G
    assert header_rows() == G.rows()


def test_double_float_evaluation_accuracy():
    mp.mp.dps = 40
    rows = header_rows()
    rng = np.random.default_rng(12)
    # every interval at its ends and middle, plus random points and tiny arguments
    ys = []
    for j in range(512):
        y0 = j / 256
        ys += [y0, y0 + 1 / 512, np.nextafter(y0 + 1 / 256, 0.0)]
    ys += list(rng.uniform(0, 2, 400)) + [1e-30, 1e-15, 3e-9, 1e-4]
    worst = 0.0
    for y in ys:
        y = float(y)
        if y >= 2.0:
            continue
        got = rate_factor(rows, y)
        ex = g_exact(y)
        worst = max(worst, float(abs((mp.mpf(got.numerator) / got.denominator - ex) / ex)))
    assert worst < 1e-14, worst


def test_closed_forms():
    rows = header_rows()
    # g(0) = 1 exactly (row 0: c0 = 1), g(1) = 1 - 1/e, and g(y) = 1 - y/2 + y^2/6 near 0
    assert rate_factor(rows, 0.0) == 1
    assert abs(float(rate_factor(rows, 1.0)) - float(1 - mp.exp(-1))) < 5e-15
    y = 1e-6
    assert abs(float(rate_factor(rows, y)) - (1 - y / 2 + y * y / 6)) < 5e-16
