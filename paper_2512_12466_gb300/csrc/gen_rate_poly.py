"""Coefficients of the FP64 march's Eq. 1 factor g(y) = (1 - e^{-y}) / y on 0 <= y < 2.

Writes the polynomial in t = y - 1 (t in [-1, 1)) that march.cu evaluates by Horner's rule:
a Chebyshev interpolant of degree DEGREE (mpmath.chebyfit, i.e. interpolation at Chebyshev
nodes, Trefethen, Approximation Theory and Approximation Practice, ch. 4-8), its coefficients
rounded to double. Prints the C initialiser and the largest relative error of the rounded
polynomial, evaluated with fused multiply-adds, over a fine grid of [0, 2).

    python paper_2512_12466_gb300/csrc/gen_rate_poly.py
"""
from fractions import Fraction

import mpmath as mp

DEGREE = 13


def g(y):
    return -mp.expm1(-y) / y if y != 0 else mp.mpf(1)


def coefficients(degree=DEGREE):
    mp.mp.dps = 50
    poly, err = mp.chebyfit(lambda t: g(1 + t), [-1, 1], degree + 1, error=True)
    return [float(c) for c in poly], float(err)       # highest degree first


def horner_fma(coef, y):
    """Horner's rule in t = y - 1 with every step a correctly rounded fused multiply-add."""
    t = float(Fraction(y) - 1)
    p = coef[0]
    for c in coef[1:]:
        p = float(Fraction(p) * Fraction(t) + Fraction(c))
    return p


def max_rel_error(coef, points=4000):
    mp.mp.dps = 40
    worst = 0.0
    for i in range(points):
        y = 2.0 * i / points
        y = y if y > 0 else 1e-300
        exact = g(mp.mpf(y))
        worst = max(worst, float(abs((mp.mpf(horner_fma(coef, y)) - exact) / exact)))
    return worst


if __name__ == "__main__":
    coef, err = coefficients()
    print("// highest degree first; interpolation error %.2e (absolute)" % err)
    for c in coef:
        print("    %s," % repr(c))
    print("// max relative error of the rounded polynomial on [0, 2): %.2e" % max_rel_error(coef))
