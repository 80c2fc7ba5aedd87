"""The seeded synthetic inputs follow the recipes they state: a Gaussian random
field with P(k) ~ k^-2, mean-preserving lognormal densities, sources in the
densest 1% of cells, Ndot ~ Ndot^-2 on [1e50, 1e53], the workload shapes, and
reproducibility from the seed alone."""
import numpy as np
import pytest

from paper_2512_12466_gb300 import inputs as I


def test_gaussian_field_spectrum_slope():
    """Shell-averaged |FFT|^2 of the field falls as k^-2 (fitted slope within 0.15) over the
    modes away from the box scale and the grid scale, with zero mean and unit variance."""
    n = 64
    g = I.gaussian_random_field(n, seed=11)
    assert abs(g.mean()) < 1e-12 and abs(g.std() - 1) < 1e-12
    p = np.abs(np.fft.rfftn(g)) ** 2
    kz = np.fft.fftfreq(n) * n
    kx = np.fft.rfftfreq(n) * n
    kk = np.sqrt(kz[:, None, None] ** 2 + kz[None, :, None] ** 2 + kx[None, None, :] ** 2)
    bins = np.arange(4, 24)
    pk = [p[(kk >= b) & (kk < b + 1)].mean() for b in bins]
    slope = np.polyfit(np.log(bins + 0.5), np.log(pk), 1)[0]
    assert abs(slope + 2) < 0.15, slope


def test_lognormal_mean_exact_and_width():
    v = I.lognormal(48, 2e-4, 1.0, seed=12)
    assert abs(v.mean() / 2e-4 - 1) < 1e-12
    assert (v > 0).all()
    assert abs(np.log(v).std() - 1.0) < 1e-9        # log of the field is the unit-variance field


def test_sources_in_densest_percent():
    n_h = I.lognormal(40, 1.0, 1.0, seed=13)
    cells = I.place_sources(n_h, 500, seed=14)
    thresh = np.sort(n_h.ravel())[-int(round(0.01 * n_h.size))]
    vals = n_h[cells[:, 2], cells[:, 1], cells[:, 0]]
    assert (vals >= thresh).all()
    assert len(np.unique(cells, axis=0)) < 500      # drawn with replacement: duplicates occur


def test_power_law_ndot_distribution():
    """Inverse-CDF draws of p(x) ~ x^-2 on [a, b]: F(x) = (1/a - 1/x) / (1/a - 1/b); the
    empirical CDF agrees within 0.01 at five points, and every draw lies in [a, b]."""
    a, b = 1e50, 1e53
    x = I.power_law_ndot(200000, seed=15)
    assert x.min() >= a and x.max() <= b
    for q in (2e50, 5e50, 1e51, 1e52, 5e52):
        cdf = (1 / a - 1 / q) / (1 / a - 1 / b)
        assert abs((x <= q).mean() - cdf) < 0.01


def test_workload_shapes_and_reproducibility():
    w = I.config2("thin")
    assert w.n == 128 and w.n_h.shape == (128, 128, 128) and len(w.ndot) == 1024
    assert abs(w.box_cm - 20.0 / I.HUBBLE_H * I.MPC_CM) < 1e-6 * w.box_cm
    assert abs(w.n_h.mean() / 2e-4 - 1) < 1e-12
    assert np.allclose(1 - w.x_ion, 1e-4)
    w2 = I.config2("thin")
    assert np.array_equal(w.n_h, w2.n_h) and np.array_equal(w.cells, w2.cells) and np.array_equal(w.ndot, w2.ndot)
    wn = I.config2("neutral")
    assert (wn.x_ion == 0).all() and np.array_equal(wn.cells, w.cells)


def test_patchy_ionized_fraction():
    """x = clip(v, 0, 1) with v a mean-1 lognormal of sigma_ln 1.5: the fully ionized fraction
    is P(ln v >= 0) = P(Z >= 0.75) = 0.2266 for ln v ~ N(-1.125, 1.5^2), up to the sample."""
    w = I.cosmo_box(64, 10.0, 1.5, 16, config=4, x_mode="patchy")
    assert abs((w.x_ion == 1).mean() - 0.2266) < 0.03
    assert w.x_ion.min() >= 0 and w.x_ion.max() <= 1


def test_batch_mix_recipe():
    ws = I.batch_solves(64, config=3, x_mode="neutral")
    assert len(ws) == 64
    assert {w.n for w in ws} <= {32, 64, 96, 128}
    assert all(1 <= len(w.ndot) <= 4096 for w in ws)
    dx = {w.box_cm / w.n for w in ws}
    assert max(dx) / min(dx) - 1 < 1e-12                # one cell size across the mix


def test_poisson_arrivals_rate():
    t = I.poisson_arrivals(200.0, 20000, seed=16)
    assert np.all(np.diff(t) > 0)
    assert abs(len(t) / t[-1] / 200.0 - 1) < 0.03


@pytest.mark.parametrize("config,stream,solve,expect", [(2, 1, 0, 2001), (4, 3, 0, 4003), (3, 4, 5, 3504)])
def test_seed_scheme(config, stream, solve, expect):
    assert I.seed_for(config, stream, solve) == expect
