"""Taylor table of the Eq. 1 factor g(y) = (1 - e^{-y}) / y for the FP64 table march's
double-float arithmetic; writes ``rate_table.h`` next to this script.

On [0, 2) the factor is expanded about y0 in each of 512 intervals of width 1/256: the left end
y0 = 0 for the first interval and the midpoint y0 = (j + 1/2) / 256 for the others, so that
|y - y0| <= 1/512 (below 1/256 on the first) and y - y0 is exact in float arithmetic (Sterbenz:
y / y0 lies in [2/3, 4/3] for j >= 1). The expansion g(y0 + r) = sum_k c_k(y0) r^k runs to degree 4;
its coefficients c_k(y0) = sum_{n >= k} C(n, k) (-1)^n y0^(n - k) / (n + 1)!, the k-th derivative of
the power series g(y) = sum_n (-y)^n / (n + 1)! divided by k!, are summed in 50-digit arithmetic.
c_0..c_2 are stored as double-float pairs (head = the value rounded to float, tail = the rest
rounded to float, about 48 bits together), c_3 and c_4 as floats: c_3 r^3 is below 3e-9, so float
precision there costs under 1e-15 of g, and the truncation after r^4 is below 2e-15 relative
(|c_5| r^5 < 2^-6 2^-45 for j >= 1, 2^-40 / 720 for j = 0).

Each row: {c0 head, c0 tail, c1 head, c1 tail, c2 head, c2 tail, c3, c4}, written as C99
hexadecimal float literals, so the header holds the exact float values.

    python paper_2512_12466_gb300/csrc/gen_rate_table.py
"""
import os
import struct

import mpmath as mp

INTERVALS = 512          # over [0, 2), width 1/256
STEP = mp.mpf(1) / 256
DEGREE = 4
HERE = os.path.dirname(os.path.abspath(__file__))


def f32(x) -> float:
    """x rounded to the nearest float (through double; the tail absorbs the double rounding)."""
    return struct.unpack("<f", struct.pack("<f", float(x)))[0]


def coefficient(k: int, y0) -> mp.mpf:
    """c_k(y0) = g^(k)(y0) / k! from the power series of g about 0."""
    s = mp.mpf(0)
    n = k
    while True:
        term = mp.binomial(n, k) * (-1) ** n * y0 ** (n - k) / mp.factorial(n + 1)
        s += term
        if n > k + 8 and abs(term) < mp.mpf(10) ** -45:
            return s
        n += 1


def centre(j: int):
    """Expansion point of interval j: its left end for j = 0, its midpoint otherwise."""
    return mp.mpf(0) if j == 0 else (j + mp.mpf(1) / 2) * STEP


def rows():
    mp.mp.dps = 50
    out = []
    for j in range(INTERVALS):
        c = [coefficient(k, centre(j)) for k in range(DEGREE + 1)]
        row = []
        for k in range(3):
            h = f32(c[k])
            row += [h, f32(c[k] - mp.mpf(h))]
        row += [f32(c[3]), f32(c[4])]
        out.append(row)
    return out


def write(path=os.path.join(HERE, "rate_table.h")):
    lines = [
        "// Generated by gen_rate_table.py: Taylor coefficients of g(y) = (1 - e^{-y}) / y about",
        "// y0 = 0 (j = 0) and y0 = (j + 1/2) / 256 (j = 1..511), the Eq. 1 rate factor of the FP64",
        "// table march. Row j: {c0 head, c0 tail, c1 head, c1 tail, c2 head, c2 tail, c3, c4}.",
        "#pragma once",
        "",
        "namespace nyx {",
        f"constexpr int kRateIntervals = {INTERVALS};",
        "constexpr int kRateCoefs = 8;",
        f"__device__ const float kRateTable[{INTERVALS} * 8] = {{",
    ]
    for r in rows():
        lines.append("    " + ", ".join(v.hex() if v != 0 else "0x0p+0" for v in r) + ",")
    lines += ["};", "}  // namespace nyx", ""]
    with open(path, "w") as f:
        f.write("\n".join(lines))


if __name__ == "__main__":
    write()
