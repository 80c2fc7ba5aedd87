"""The FP64 march's Eq. 1 factor g(y) = (1 - e^{-y}) / y below y = 2 is a
polynomial whose constants are written in march.cu: they must be the ones the
generator script derives, and the polynomial, evaluated as the kernel does
(Horner's rule in y - 1 with fused multiply-adds), must stay within 3e-16 of g
relative (checked against 40-digit arithmetic), so that the FP64 march's
deposits keep their 1e-12 agreement with the oracle with room to spare."""
import os
import re
import sys

import pytest

mp = pytest.importorskip("mpmath")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2512_12466_gb300", "csrc")


def kernel_coefficients():
    src = open(os.path.join(CSRC, "march.cu")).read()
    body = src[src.index("const double t = dtau - 1.0;"):src.index("a = P * (dtau * g);")]
    first = re.search(r"double g = ([-+0-9.e]+);", body).group(1)
    rest = re.findall(r"g = fma\(g, t, ([-+0-9.e]+)\);", body)
    return [float(first)] + [float(c) for c in rest]


def test_constants_are_the_generators():
    sys.path.insert(0, CSRC)
    import gen_rate_poly as G
    coef, err = G.coefficients()
    assert kernel_coefficients() == coef
    assert err < 1e-16


def test_polynomial_accuracy():
    sys.path.insert(0, CSRC)
    import gen_rate_poly as G
    assert G.max_rel_error(kernel_coefficients(), points=1500) < 3e-16
    # the expansion near 0 and the value at 1 (closed forms)
    c = kernel_coefficients()
    assert abs(G.horner_fma(c, 1e-12) - (1.0 - 0.5e-12)) < 2e-16      # g(y) = 1 - y/2 + O(y^2)
    assert abs(G.horner_fma(c, 1.0) - float(1 - mp.exp(-1))) < 2e-16
