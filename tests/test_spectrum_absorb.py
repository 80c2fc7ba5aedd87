"""A segment's absorbed fraction Phi(tau) - Phi(tau + dtau) under the blackbody
rate (Eq. 1 over frequency, Sec. 2.5), as the FP64 march computes it
(rt_spectrum_absorb runs the same function on the host), against the defining
integral <exp(-tau s) (1 - exp(-dtau s))>, taken here by adaptive quadrature with
expm1 so that thin segments keep their precision. No GPU.

The march takes the difference from cubic pieces in tau as a mean slope, so the
error of a segment is relative to the segment itself: thin segments, segments
that just cross a node, segments that cross many pieces and the series below
2^-20 all hold the same relative bar.
"""
import math

import numpy as np
import pytest

import paper_2512_12466_gb300 as nyx

H_NU0_ERG = 13.598 * 1.602176634e-12
K_B = 1.380649e-16
T_BB = 1e5


def absorbed(t_bb, tau, dtau):
    from scipy.integrate import quad
    theta = H_NU0_ERG / (K_B * t_bb)
    w = lambda y: y ** 2 * math.exp(-theta * y) / -math.expm1(-theta * y)
    f = lambda y: w(y) * math.exp(-tau * y ** -3.0) * -math.expm1(-dtau * y ** -3.0)
    norm = quad(w, 1, np.inf, epsabs=0, epsrel=1e-13, limit=400)[0]
    return quad(f, 1, np.inf, epsabs=0, epsrel=1e-13, limit=400)[0] / norm


def node(e, i, per):
    """The i-th node of octave e at `per` pieces per octave."""
    return math.ldexp(1.0 + i / per, e)


@pytest.fixture(scope="module")
def lib():
    try:
        return nyx.lib()
    except ImportError as e:
        pytest.skip(str(e))


CASES = [
    # thin segments, far below any piece width
    (0.3, 1e-12), (2.7, 1e-10), (40.0, 1e-9), (1e-5, 1e-13),
    # within one piece
    (0.05, 1e-4), (6.0, 1e-2),
    # just across one node, below and above tau = 1 and across tau = 1 itself
    (node(-3, 7, 32) - 1e-12, 2e-12), (node(2, 9, 128) - 1e-11, 3e-11), (1.0 - 1e-12, 3e-12),
    # across several pieces, and from the ray's start
    (0.2, 0.5), (3.0, 7.0), (0.0, 2.0), (0.0, 1e3), (0.5, 80.0), (0.99, 0.05), (0.999, 2e-3),
    # the series below 2^-20, and out of it
    (0.0, 1e-8), (2e-7, 3e-7), (9e-7, 1e-7), (2.0 ** -20 - 1e-15, 1e-14),
]


@pytest.mark.parametrize("tau,dtau", CASES)
def test_segment_matches_definition(lib, tau, dtau):
    got = nyx.rt_spectrum_absorb(T_BB, tau, dtau)
    ref = absorbed(T_BB, tau, dtau)
    assert abs(got - ref) <= 2e-7 * ref, (tau, dtau, got, ref)


def test_segments_add_up_along_a_ray(lib):
    """A chain of segments of mixed lengths loses what Phi says it loses between its ends."""
    rng = np.random.default_rng(11)
    tau = 0.0
    total = 0.0
    for _ in range(400):
        dtau = float(10 ** rng.uniform(-9, -0.5))
        total += nyx.rt_spectrum_absorb(T_BB, tau, dtau)
        tau += dtau
    phi_end = nyx.rt_spectrum_eval(T_BB, tau)[0]
    assert abs(total - (1.0 - phi_end)) <= 1e-12 * (1.0 - phi_end)


def test_rejects_out_of_range(lib):
    for t_bb, tau, dtau in ((1e5, -1.0, 0.1), (1e5, 1.0, 0.0), (1e5, 2e4, 0.1), (0.0, 1.0, 0.1), (1e5, 1.0, 2e4)):
        with pytest.raises(nyx.NyxError):
            nyx.rt_spectrum_absorb(t_bb, tau, dtau)
