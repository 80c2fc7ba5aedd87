"""The FP64 table march evaluates the Eq. 1 factor g(y) = (1 - e^{-y}) / y below y = 2
in double-float arithmetic from a Taylor table (csrc/rate_table.h). The table must be the
one its generator derives, and the evaluation, replayed here operation by operation in
IEEE single precision (fused multiply-adds rounded once), must stay within 1e-14 of g
relative, checked against 40-digit arithmetic (the tail additions of a double-float sum
round at about 2^-48 of the value each), so that the march's deposits keep their 1e-12
agreement with the FP64 oracle with room to spare. The Eqs. 5-8 shares of each segment's
rate (f from the geometry table's code, Eq. 8's (1 - f) w kap / kap') are replayed the
same way against exact rationals."""
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
    y0 = fma(float(j), 0.00390625, 0.001953125) if j else 0.0
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


# ---- the Eqs. 5-8 shares of a segment's rate, as the FP64 table march evaluates them

def df_mul(a, b):
    p = mul(a[0], b[0])
    e = fma(a[0], b[1], fma(a[0], b[0], -p))
    return p, fma(a[1], b[0], e)


def df_mant(x: float):
    """A positive double as a double-float mantissa in [1, 2) and its exponent, as the kernel splits it."""
    ex = math.frexp(x)[1] - 1
    h, l = df_of(math.ldexp(x, -ex))
    return (h, l), ex


def f_of_code(code: int):
    """The kernel's double-float f from a table entry's 53-bit code (bits of f less those of 1/2, plus 1)."""
    m = code - 1
    h = struct.unpack("<f", struct.pack("<I", 0x3F000000 + (m >> 29)))[0]
    return h, mul(float(m & 0x1FFFFFFF), 2.0 ** -53)


def frcp(x):
    return round32(1 / Fraction(x))


def val(a):
    return Fraction(a[0]) + Fraction(a[1])


def test_share_f_from_the_table_code():
    # the entry stores f in [1/2, 1] as its bit pattern less that of 1/2, plus 1; the kernel reads
    # it back as a double-float directly, which must be the head/tail split of that double
    base = struct.unpack("<q", struct.pack("<d", 0.5))[0] - 1
    rng = np.random.default_rng(31)
    fs = [0.5, 1.0, np.nextafter(1.0, 0.0), np.nextafter(0.5, 1.0)] + list(rng.uniform(0.5, 1.0, 300))
    for f in fs:
        code = struct.unpack("<q", struct.pack("<d", float(f)))[0] - base
        assert f_of_code(code) == df_of(float(f)), f


def test_secondary_share_double_float():
    """Eq. 8's share (1 - f) w kap / kap' of a segment whose rate is w = u ds (u = Q g, the
    budget times the Eq. 1 factor), in the kernel's two forms: from the absorbed photons u dtau
    over kap' (gray rate) and from the ratio of the mantissas of kap and kap' (the blackbody rate
    and segments thinner than 2^-74). Against exact rationals, over f up to just below 1, where
    1 - f must be renormalised to keep its precision, and kap' from 1e-3 to 1e3 of kap."""
    rng = np.random.default_rng(77)
    worst = {"ux": 0.0, "ratio": 0.0}
    for _ in range(1500):
        u = (round32(Fraction(float(rng.uniform(1, 2) * 2.0 ** 60))), round32(Fraction(float(rng.uniform(-1, 1) * 2.0 ** 36))))
        kap = float(rng.uniform(1e-3, 3) * 10 ** rng.uniform(-8, 0))
        kn = float(kap * 10 ** rng.uniform(-3, 3))
        ds = float(rng.uniform(0.01, 1.7))
        dtau = kap * ds                          # IEEE FP64, as the kernel's deciding product
        f = float(1 - 10 ** rng.uniform(-15, -0.31))
        fd = df_of(f)
        om = fast_two_sum(add(1.0, -fd[0]), -fd[1])
        mn, en = df_mant(kn)
        exact = (1 - val(fd)) * val(u) * Fraction(dtau) / Fraction(kn)
        if exact == 0:
            continue
        # gray: (1 - f) ux / kap', ux = u dtau
        ux = df_mul(u, df_of(dtau))
        # the hardware's approximate reciprocal, taken anywhere within 2^-22 of 1 / x, then one
        # Newton step and the residual as the tail
        r = round32(Fraction(1) / Fraction(mn[0]) * (1 + Fraction(float(rng.uniform(-1, 1))) / 2 ** 22))
        r = fma(r, fma(-mn[0], r, 1.0), r)
        inv = (r, mul(fma(-mn[1], r, fma(-mn[0], r, 1.0)), r))
        got = val(df_mul(df_mul(om, ux), inv)) / Fraction(2) ** en
        worst["ux"] = max(worst["ux"], abs(float((got - exact) / exact)))
        # ratio form: (1 - f) w (m_kap / m_kap') 2^(e_kap - e_kap')
        w = df_mul(u, df_of(ds))
        mk, ek = df_mant(kap)
        r0 = frcp(mn[0])
        q0 = mul(mk[0], r0)
        p = mul(mn[0], q0)
        pe = fma(mn[0], q0, -p)
        rho = fma(-q0, mn[1], add(add(add(mk[0], -p), -pe), mk[1]))
        got = val(df_mul(df_mul(om, w), (q0, mul(rho, r0)))) * Fraction(2) ** (ek - en)
        exact_w = (1 - val(fd)) * val(u) * Fraction(ds) * Fraction(kap) / Fraction(kn)
        worst["ratio"] = max(worst["ratio"], abs(float((got - exact_w) / exact_w)))
    # double-float products round at about 2^-45 each; the deposit is then rounded to double
    assert worst["ux"] < 2e-13 and worst["ratio"] < 2e-13, worst
