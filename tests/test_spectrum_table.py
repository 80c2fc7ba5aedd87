"""The library's blackbody spectrum table (RT_SPECTRUM_BLACKBODY, Eq. 1 over
frequency) against the defining integrals, on the host (no GPU).

Phi(tau) = <exp(-tau s)> and Psi(tau) = <s exp(-tau s)> over the photon-number
spectrum y^2 / (exp(theta y) - 1) above the threshold (y = nu / nu_0,
s = y^-3, theta = h nu_0 / k T), computed here by adaptive quadrature; the
library builds cubic pieces in tau by its own quadrature (Hermite cubics of the
node values and slopes, 32 per octave below tau = 1 and 128 above, a three-term
series below 2^-20) and reads them back between nodes. The bar, 2e-11 absolute,
sits four times above the worst error measured (5e-12, at 2e4 K).
"""
import math

import numpy as np
import pytest

import paper_2512_12466_gb300 as nyx

H_NU0_ERG = 13.598 * 1.602176634e-12
K_B = 1.380649e-16


def moment(t_bb, tau, p):
    from scipy.integrate import quad
    theta = H_NU0_ERG / (K_B * t_bb)
    f = lambda y, q, t: (y ** 2 * math.exp(-theta * y) / -math.expm1(-theta * y)) * y ** (-3.0 * q) * math.exp(-t * y ** -3.0)
    norm = quad(f, 1, np.inf, args=(0, 0.0), epsabs=0, epsrel=1e-13, limit=400)[0]
    return quad(f, 1, np.inf, args=(p, tau), epsabs=0, epsrel=1e-13, limit=400)[0] / norm


@pytest.fixture(scope="module")
def lib():
    try:
        return nyx.lib()
    except ImportError as e:
        pytest.skip(str(e))


@pytest.mark.parametrize("t_bb", [2e4, 1e5])
def test_table_matches_definition(lib, t_bb):
    rng = np.random.default_rng(3)
    # below, at and above the series' end (2^-20), the change of resolution (1) and the last node (2^14 > 1e4)
    edges = [2.0 ** -20 * (1 - 1e-12), 2.0 ** -20, 2.0 ** -20 * (1 + 1e-9), 1 - 1e-12, 1.0, 1 + 1e-9]
    taus = [0.0, 3e-9, 1e-8, 1e-6, 1e-3] + edges + list(10 ** rng.uniform(-8, 4, size=25)) + [30.0, 100.0, 1e3, 1e4]
    for tau in taus:
        phi, psi = nyx.rt_spectrum_eval(t_bb, tau)
        assert abs(phi - moment(t_bb, tau, 0)) < 2e-11, tau
        assert abs(psi - moment(t_bb, tau, 1)) < 2e-11, tau
    assert nyx.rt_spectrum_eval(t_bb, 0.0)[0] == 1.0


def test_table_rejects_out_of_range(lib):
    for t_bb, tau in ((1e5, -1.0), (1e5, 2e4), (0.0, 1.0), (-5.0, 1.0)):
        with pytest.raises(nyx.NyxError):
            nyx.rt_spectrum_eval(t_bb, tau)
