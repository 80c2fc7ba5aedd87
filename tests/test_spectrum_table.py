"""The library's blackbody spectrum table (RT_SPECTRUM_BLACKBODY, Eq. 1 over
frequency) against the defining integrals, on the host (no GPU).

Phi(tau) = <exp(-tau s)> and Psi(tau) = <s exp(-tau s)> over the photon-number
spectrum y^2 / (exp(theta y) - 1) above the threshold (y = nu / nu_0,
s = y^-3, theta = h nu_0 / k T), computed here by adaptive quadrature; the
library builds its table by its own quadrature and reads it back by cubic
interpolation in ln tau, also between grid points and below the first one.
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
    taus = [0.0, 3e-9, 1e-8, 1e-6, 1e-3] + list(10 ** rng.uniform(-8, 2, size=25)) + [30.0, 100.0, 1e3]
    for tau in taus:
        phi, psi = nyx.rt_spectrum_eval(t_bb, tau)
        assert abs(phi - moment(t_bb, tau, 0)) < 2e-9, tau
        assert abs(psi - moment(t_bb, tau, 1)) < 2e-9, tau
    assert nyx.rt_spectrum_eval(t_bb, 0.0)[0] == 1.0


def test_table_rejects_out_of_range(lib):
    for t_bb, tau in ((1e5, -1.0), (1e5, 2e4), (0.0, 1.0), (-5.0, 1.0)):
        with pytest.raises(nyx.NyxError):
            nyx.rt_spectrum_eval(t_bb, tau)
