"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed
forms (Stromgren radius and I-front, optically thin 1/r^2, opaque source
cell, split-count powers of 4), exact invariants (photon ledger, deposited =
absorbed, linearity in sources, symmetry), an independent brute-force tracer
with exact rational geometry, textbook chemistry limits, and brute-force
graph components for source merging.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import brute_trace as bt
import oracle
from paper_2512_12466_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def relerr(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


# ------------------------------------------------------------------ hashing / HEALPix

def test_mix64_splitmix_vector():
    # splitmix64 seeded with 0: first state 0x9e3779b97f4a7c15, first output 0xe220a8397b1dcdaf.
    assert oracle.mix64(0x9E3779B97F4A7C15) == 0xE220A8397B1DCDAF


def test_healpix_level0_centres():
    """12 base pixels: z = 2/3 (faces 0-3), 0 (4-7), -2/3 (8-11); phi as in Gorski et al."""
    for p in range(12):
        v = oracle.pix2vec(0, p)
        row, col = divmod(p, 4)
        z = [2.0 / 3.0, 0.0, -2.0 / 3.0][row]
        phi = (math.pi / 4 + col * math.pi / 2) if row != 1 else col * math.pi / 2
        s = math.sqrt(1 - z * z)
        np.testing.assert_allclose(v, [s * math.cos(phi), s * math.sin(phi), z], atol=1e-15)


@pytest.mark.parametrize("level", [1, 2, 3, 4])
def test_healpix_structure(level):
    nside = 2 ** level
    npix = 12 * nside * nside
    vs = np.array([oracle.pix2vec(level, p) for p in range(npix)])
    np.testing.assert_allclose(np.linalg.norm(vs, axis=1), 1.0, atol=2e-16)
    # rings: 4 nside - 1 distinct z; polar ring i has 4i pixels, belt rings 4 nside
    zs, counts = np.unique(np.round(vs[:, 2], 12), return_counts=True)
    assert len(zs) == 4 * nside - 1
    expect = {}
    for i in range(1, 4 * nside):
        if i < nside:
            z, c = 1 - i * i / (3 * nside * nside), 4 * i
        elif i > 3 * nside:
            j = 4 * nside - i
            z, c = -(1 - j * j / (3 * nside * nside)), 4 * j
        else:
            z, c = (2 * nside - i) * 2 / (3 * nside), 4 * nside
        expect[round(z, 12)] = c
    assert dict(zip(zs.tolist(), counts.tolist())) == expect
    # nested children 4p..4p+3 lie around the parent (within the parent's pixel radius)
    parents = np.array([oracle.pix2vec(level - 1, p) for p in range(npix // 4)])
    ang_parent = math.sqrt(4 * math.pi / (npix // 4))
    for p in range(npix // 4):
        for q in range(4):
            cosang = float(np.dot(parents[p], vs[4 * p + q]))
            assert math.acos(min(1.0, cosang)) < ang_parent
    # the set of quantised directions is symmetric under z -> -z and 90 deg about z
    q = {tuple(oracle.direction(level, p)[0]) for p in range(npix)}
    assert {(x, y, -z) for x, y, z in q} == q
    assert {(-y, x, z) for x, y, z in q} == q


def test_two_healpix_implementations_agree():
    for level in range(6):
        for p in range(12 * 4 ** level):
            assert list(oracle.direction(level, p)[0]) == bt.quantise(bt.healpix_nest_vec(level, p))


# ------------------------------------------------------------------ split criterion (Eq. 4)

@pytest.mark.parametrize("n_min", [1.0, 2.0, 4.0, 8.0])
def test_split_radius_matches_eq4(n_min):
    """Omega_c / Omega(l) = N_min exactly at R_l (Omega_c = 1/R^2, Omega(l) = 4pi/(12 4^l))."""
    rq = oracle.split_rq(n_min)
    for lvl in range(8):
        r = rq * 2.0 ** (lvl - 24)
        ratio = (1.0 / r ** 2) / (4 * math.pi / (12 * 4 ** lvl))
        assert abs(ratio / n_min - 1) < 1e-6


def test_default_level_max_never_binds():
    for n, nmin in [(64, 4.0), (128, 4.0), (256, 2.0)]:
        lm = oracle.default_level_max(n, nmin)
        rq = oracle.split_rq(nmin)
        assert rq * 2.0 ** (lm - 1 - 24) >= math.sqrt(3) * n
        assert rq * 2.0 ** (lm - 2 - 24) < math.sqrt(3) * n


# ------------------------------------------------------------------ brute force (P5)

@pytest.mark.parametrize("seed,mode,n_th_frac,xmode", [
    (5, 0, 0.01, "mixed"), (6, 3, 0.01, "mixed"), (7, 3, 0.8, "mixed"), (8, 2, 0.8, "mixed"),
    (9, 1, 0.01, "thin"), (10, 3, 0.5, "patchy"), (11, 4, 0.01, "thin"), (12, 5, 0.5, "mixed")])
def test_oracle_matches_brute_force(seed, mode, n_th_frac, xmode):
    n = 6 if seed % 2 else 8
    w = I.random_small(n, 3, seed=seed, x_mode=xmode, box_cm=n * 3e21)
    # the catalog both sides trace: lexicographically sorted, duplicates summed
    uc, inv = np.unique(w.cells, axis=0, return_inverse=True)
    w.ndot = np.bincount(inv.reshape(-1), weights=w.ndot)
    w.cells = uc.astype(np.int32)
    n_th = n_th_frac * float(w.n_h.mean())
    g, vis, cnt = bt.trace(w.n_h, w.x_ion, w.cells, w.ndot, w.box_cm, overlap_mode=mode, n_th=n_th)
    r = oracle.run_workload(w, record=400000, overlap_mode=mode, n_th_cm3=n_th)
    v = r["visits"]
    assert v["total"] == len(vis)
    ov = sorted(zip(v["ray"].tolist(), v["seq"].tolist(), v["cell"].tolist()))
    bv = sorted((a, b, c) for a, b, c, _ in vis)
    assert ov == bv
    ds_o = dict(((a, b), d) for a, b, d in zip(v["ray"].tolist(), v["seq"].tolist(), v["ds"].tolist()))
    for a, b, c, d in vis:
        assert abs(ds_o[(a, b)] - d) <= 4e-16 * max(1.0, abs(d))
    assert relerr(r["gamma"].reshape(-1), g.reshape(-1)) < 1e-12
    st = r["stats"]
    assert sum(st["secondary"]) == sum(cnt["secondary"].values())
    for lvl, c in cnt["rays"].items():
        assert st["rays"][lvl] == c
    for lvl, c in cnt["splits"].items():
        assert st["splits"][lvl] == c


# ------------------------------------------------------------------ periodic boundaries (Sec. 2.5.1)

@pytest.mark.parametrize("seed,mode,xmode", [(21, 0, "thin"), (22, 3, "mixed"), (23, 1, "patchy"), (24, 2, "mixed"),
                                             (25, 4, "thin"), (26, 5, "mixed")])
def test_periodic_oracle_matches_brute_force(seed, mode, xmode):
    """Periodic boundaries: cells wrap, rays stop at travel distance sqrt(3) n
    (and do not split there); the brute force lists the same segments from
    exact crossing times in the unwrapped frame."""
    n = 5 if seed % 2 else 4
    w = I.random_small(n, 2, seed=seed, x_mode=xmode, box_cm=n * 3e21)
    uc, inv = np.unique(w.cells, axis=0, return_inverse=True)
    w.ndot = np.bincount(inv.reshape(-1), weights=w.ndot)
    w.cells = uc.astype(np.int32)
    n_th = 0.3 * float(w.n_h.mean())
    g, vis, cnt = bt.trace(w.n_h, w.x_ion, w.cells, w.ndot, w.box_cm, overlap_mode=mode, n_th=n_th, periodic=True)
    r = oracle.run_workload(w, record=2000000, overlap_mode=mode, n_th_cm3=n_th, periodic=1)
    v = r["visits"]
    assert v["total"] == len(vis)
    ov = sorted(zip(v["ray"].tolist(), v["seq"].tolist(), v["cell"].tolist()))
    bv = sorted((a, b, c) for a, b, c, _ in vis)
    assert ov == bv
    assert relerr(r["gamma"].reshape(-1), g.reshape(-1)) < 1e-12
    st = r["stats"]
    assert sum(st["secondary"]) == sum(cnt["secondary"].values())
    for lvl, c in cnt["rays"].items():
        assert st["rays"][lvl] == c
    for lvl, c in cnt["splits"].items():
        assert st["splits"][lvl] == c


@pytest.mark.parametrize("prec", [0, 1])
def test_periodic_translation_invariance(prec):
    """On a periodic grid, moving the source by v and rolling the fields by v
    rolls Gamma by v exactly: every ray sees the same cells relative to its
    source, in the same order, so even the floating-point sums are equal."""
    n = 12
    w = I.random_small(n, 1, seed=31, x_mode="mixed", box_cm=n * 3e21)
    v = (5, -3, 7)
    c = np.array([[3, 9, 1]], np.int32)
    cv = ((c + np.array(v)) % n).astype(np.int32)
    roll = lambda a: np.roll(a, shift=(v[2], v[1], v[0]), axis=(0, 1, 2))   # arrays are [z, y, x]
    kw = dict(n_th_cm3=0.3 * float(w.n_h.mean()), periodic=1, precision=prec, overlap_mode=3)
    a = oracle.run(w.n_h, w.x_ion, c, w.ndot[:1], w.box_cm, **kw)
    b = oracle.run(roll(w.n_h), roll(w.x_ion), cv, w.ndot[:1], w.box_cm, **kw)
    assert sum(a["stats"]["segments"]) > 10000
    assert np.array_equal(roll(a["gamma"]), b["gamma"])
    for k in ("rays", "splits", "segments", "secondary", "escaped", "dropped_tau"):
        assert a["stats"][k] == b["stats"][k]


def test_periodic_thin_path_sum():
    """Thin periodic medium: every root-to-leaf chain of rays covers exactly
    the travel distance sqrt(3) n, so sum(Gamma) = Ndot sigma sqrt(3) n / dx^2
    (up to direction quantisation, 2e-6); rays end there, none escapes earlier."""
    n = 16
    n_h = np.full((n, n, n), 2e-4)
    x = np.ones((n, n, n))
    box = n * 7.117e23
    ndot = np.array([1e52])
    r = oracle.run(n_h, x, np.array([[3, 11, 6]], np.int32), ndot, box, overlap_mode=0, periodic=1)
    st = r["stats"]
    rs = oracle.periodic_rs(n)
    rq = oracle.split_rq(4.0)
    last = next(l for l in range(20) if (rq << l) >= rs)
    for lvl in range(last + 1):
        assert st["rays"][lvl] == 12 * 4 ** lvl
        assert st["escaped"][lvl] == (12 * 4 ** lvl if lvl == last else 0)
    dx = box / n
    expect = ndot[0] * 6.3e-18 * (rs * 2.0 ** -24) / dx ** 2
    assert abs(r["gamma"].sum() / expect - 1) < 2e-6
    assert abs(st["absorbed_ph"]) == 0 and abs(st["escaped_ph"] / st["emitted_ph"] - 1) < 1e-12


@pytest.mark.parametrize("prec", [0, 1])
def test_periodic_photon_ledger(prec):
    w = I.random_small(20, 5, seed=41, x_mode="mixed", box_cm=20 * 3e21)
    r = oracle.run_workload(w, precision=prec, periodic=1, overlap_mode=3)
    st = r["stats"]
    e = st["emitted_ph"]
    tol = 1e-12 if prec == 0 else 1e-6
    assert abs(st["absorbed_ph"] + st["escaped_ph"] + st["dropped_ph"] - e) / e < tol
    assert abs(st["deposited_ph"] - st["absorbed_ph"]) / e < tol


# ------------------------------------------------------------------ closed forms

def test_opaque_source_cell_closed_form():
    """Neutral dense gas: every level-0 ray is spent in the source cell, so
    Gamma_src = Ndot / (n_HI V) and nothing else is touched (P1)."""
    w = I.cosmo_box(32, 20.0 * 32 / 128, 1.0, 5, config=2, x_mode="neutral")
    r = oracle.run_workload(w)
    st = r["stats"]
    assert st["rays"][0] == 12 * st["n_src_emit"] and st["segments"][0] == 12 * st["n_src_emit"]
    assert sum(st["splits"]) == 0 and st["dropped_tau"][0] == 12 * st["n_src_emit"]
    vol = w.dx_cm ** 3
    g = r["gamma"]
    expect = np.zeros_like(g)
    for (ix, iy, iz), nd in zip(r["emit_cells"], r["emit_ndot"]):
        expect[iz, iy, ix] += nd / (w.n_h[iz, iy, ix] * vol)
    assert relerr(g, expect) < 1e-14


def _thin_uniform(n=64, level_max=5):
    n_h = np.full((n, n, n), 2e-4)
    x = np.ones((n, n, n))                    # n_HI = 0: optically thin limit
    c = n // 2 - 1                            # origin 31.5: 31.5 cells to the nearest face
    return n_h, x, np.array([[c, c, c]], np.int32), np.array([1e52]), n * 7.117e23, level_max


def test_thin_limit_split_counts_and_path_sum():
    """Infinite thin medium: 12*4^l rays per level (P7) and
    sum(Gamma) = Ndot sigma R_L / dx^2 up to direction quantisation (P2)."""
    n_h, x, cells, ndot, box, lm = _thin_uniform()
    r = oracle.run(n_h, x, cells, ndot, box, level_max=lm, overlap_mode=0)
    st = r["stats"]
    for lvl in range(lm + 1):
        assert st["rays"][lvl] == 12 * 4 ** lvl
        assert st["escaped"][lvl] == 0
    for lvl in range(lm):
        assert st["splits"][lvl] == 12 * 4 ** lvl
    assert st["dropped_level"][lm] == 12 * 4 ** lm
    dx = box / n_h.shape[0]
    r_l = oracle.split_rq(4.0) * 2.0 ** (lm - 24)
    expect = ndot[0] * 6.3e-18 * r_l / dx ** 2
    assert abs(r["gamma"].sum() / expect - 1) < 2e-6


def test_thin_limit_inverse_square():
    """Shell-averaged Gamma r^2 = Ndot sigma / (4 pi dx^2) in a thin medium (P2)."""
    n_h, x, cells, ndot, box, lm = _thin_uniform(level_max=5)
    r = oracle.run(n_h, x, cells, ndot, box, level_max=lm, overlap_mode=0)
    n = n_h.shape[0]
    dx = box / n
    o = cells[0] + 0.5
    zz, yy, xx = np.meshgrid(*(np.arange(n) + 0.5,) * 3, indexing="ij")
    rr = np.sqrt((xx - o[0]) ** 2 + (yy - o[1]) ** 2 + (zz - o[2]) ** 2)
    norm = ndot[0] * 6.3e-18 / (4 * math.pi * dx ** 2)
    for r0 in range(4, 14):
        m = (rr >= r0) & (rr < r0 + 1)
        ratio = (r["gamma"][m] * rr[m] ** 2).mean() / norm
        assert abs(ratio - 1) < 0.02, (r0, ratio)


def test_stromgren_front_test_a():
    """Table 1 Test A, one 0.1 Myr step with the C2-Ray iteration: the I-front
    radius matches r_I(t) = r_s (1 - exp(-t/t_rec))^(1/3) to 1 cell (P3)."""
    g = json.load(open(os.path.join(GOLDEN, "table1_stromgren.json")))
    a = g["tests"]["A"]
    alpha = g["alpha_B_cm3_s"]
    w = I.stromgren_test_a(64)
    assert np.all(w.n_h == a["n_H_cm3"]) and w.ndot[0] == a["Ndot_s"]
    assert abs(w.box_cm / (a["L_box_Mpc"] * I.MPC_CM) - 1) < 1e-12
    t = 0.1 * I.MYR_S
    r = oracle.run_workload(w, chem_iterate=1, dt_s=t, alpha_B=alpha, clumping=a["C"])
    dx = w.dx_cm
    rs = (3 * a["Ndot_s"] / (4 * math.pi * alpha * a["C"] * a["n_H_cm3"] ** 2)) ** (1 / 3)
    trec = 1 / (a["C"] * alpha * a["n_H_cm3"])
    assert abs(rs / (5.393 * I.KPC_CM) - 1) < 1e-3           # 5.393 kpc
    assert abs(trec / I.MYR_S - 122.35) < 0.01
    r_i = rs * (1 - math.exp(-t / trec)) ** (1 / 3) / dx
    r_n = (3 * r["x"].sum() / (4 * math.pi)) ** (1 / 3)
    assert abs(r_n - r_i) < 1.0, (r_n, r_i)
    st = r["stats"]
    assert st["chem_residual"] < 1e-6 and st["chem_iters"] < 100
    # photon budget: ionizations <= photons emitted, and close to it (t << t_rec)
    ionized = (r["x"].sum() * a["n_H_cm3"]) * dx ** 3
    assert ionized <= a["Ndot_s"] * t * (1 + 1e-9)
    assert ionized > 0.99 * a["Ndot_s"] * t


def _front_evolution(w, steps_myr, alpha, clump, **kw):
    """Coupled Gamma <-> x over several steps (each iterated to convergence or
    the cap); equal-volume front radius in cells after each step."""
    x = w.x_ion.copy()
    out, t = [], 0.0
    for dt in steps_myr:
        r = oracle.run(w.n_h, x, w.cells, w.ndot, w.box_cm, chem_iterate=1, dt_s=dt * I.MYR_S, alpha_B=alpha,
                       clumping=clump, n_min_ray=4.0, tau_max=30.0, **kw)
        x = r["x"]
        t += dt
        out.append((t, (3 * x.sum() / (4 * math.pi)) ** (1 / 3), r["stats"]))
    return out


@pytest.mark.parametrize("test,n,steps,tol", [
    ("A", 64, [1.0, 9.0, 20.0], 0.05),          # to 30 Myr (the front reaches the half-box at 31.8 Myr)
    ("B", 48, [10.0, 40.0, 150.0], 0.05),       # clumping 5: past t_rec = 131 Myr, towards r_s = 0.563 Mpc
    ("C", 48, [10.0, 50.0], 0.05),              # r_s = 9.66 Mpc lies beyond the box; front at 60 Myr
])
def test_stromgren_front_growth(test, n, steps, tol):
    """Table 1 Tests A-C over several coupled steps: the equal-volume I-front
    radius follows r_I(t) = r_s (1 - exp(-t / t_rec))^(1/3) within 5% (P3, f2),
    with r_s and t_rec from the Table 1 parameters."""
    g = json.load(open(os.path.join(GOLDEN, "table1_stromgren.json")))
    a = g["tests"][test]
    alpha = g["alpha_B_cm3_s"]
    w = I.stromgren_test(test, n)
    assert w.n_h.flat[0] == a["n_H_cm3"] and w.ndot[0] == a["Ndot_s"] and w.params["clumping"] == a["C"]
    rs = (3 * a["Ndot_s"] / (4 * math.pi * alpha * a["C"] * a["n_H_cm3"] ** 2)) ** (1 / 3)
    trec = 1 / (a["C"] * alpha * a["n_H_cm3"])
    dx = w.box_cm / n
    for t, r_n, st in _front_evolution(w, steps, alpha, a["C"]):
        r_i = rs * (1 - math.exp(-t * I.MYR_S / trec)) ** (1 / 3) / dx
        assert r_i < n / 2                                  # the analytic front is still inside the box
        assert abs(r_n / r_i - 1) < tol, (test, t, r_n, r_i)
        assert st["chem_iters"] >= 1


@pytest.mark.parametrize("prec", [0, 1])
def test_naive_threshold_identities(prec):
    """The naive threshold (mode 5) keeps the Eq. 5 share and drops the Eq. 6
    deposit into neighbours with n'_H < n_th. On a periodic grid (every
    neighbour in the grid) with n_HI > 0 everywhere: with n_th = 0 every
    neighbour is eligible and modes 2, 3 and 5 give the same Gamma bit for bit;
    with n_th above every n_H none is, and mode 5 equals Eq. 5 alone (mode 1)
    while the conservative threshold equals no correction (mode 0)."""
    w = I.random_small(14, 3, seed=51, x_mode="thin", box_cm=14 * 7e20)
    assert (w.x_ion < 1).all()
    run = lambda mode, nth: oracle.run_workload(w, overlap_mode=mode, n_th_cm3=nth, periodic=1, precision=prec)
    g = {m: run(m, 0.0)["gamma"] for m in (2, 3, 5)}
    assert np.array_equal(g[2], g[3]) and np.array_equal(g[3], g[5])
    big = 10 * float(w.n_h.max())
    r5, r1, r3, r0 = run(5, big), run(1, big), run(3, big), run(0, big)
    assert np.array_equal(r5["gamma"], r1["gamma"]) and np.array_equal(r3["gamma"], r0["gamma"])
    assert sum(r5["stats"]["secondary"]) == 0 and not np.array_equal(r5["gamma"], r3["gamma"])


def test_naive_threshold_loses_photons():
    """With some neighbours below n_th, the naive threshold deposits fewer photons
    than are absorbed (the loss the paper reports), while the conservative
    threshold (Eqs. 7-8) deposits all of them."""
    w = I.random_small(24, 6, seed=52, x_mode="patchy", box_cm=24 * 2e21)
    nth = 0.8 * float(w.n_h.mean())
    s5 = oracle.run_workload(w, overlap_mode=5, n_th_cm3=nth)["stats"]
    s3 = oracle.run_workload(w, overlap_mode=3, n_th_cm3=nth)["stats"]
    assert s5["deposited_ph"] < s5["absorbed_ph"] * (1 - 1e-4)
    assert abs(s3["deposited_ph"] / s3["absorbed_ph"] - 1) < 1e-12
    for st in (s5, s3):
        e = st["emitted_ph"]
        assert abs(st["absorbed_ph"] + st["escaped_ph"] + st["dropped_ph"] - e) / e < 1e-12


# ------------------------------------------------------------------ frequency-integrated Eq. 1 (f3)

def _bb_moment(t_bb, tau, power):
    """Defining integral of the blackbody photon spectrum above threshold with
    sigma_nu / sigma_0 = y^-3: int y^2 / (e^{theta y} - 1) y^{-3 power} e^{-tau y^-3} dy
    over [1, inf), by adaptive quadrature (scipy), normalised by power 0 at tau 0."""
    from scipy.integrate import quad
    theta = oracle.H_NU0_ERG / (oracle.K_B_ERG_K * t_bb)
    f = lambda y, p, t: (y ** 2 * math.exp(-theta * y) / -math.expm1(-theta * y)) * y ** (-3.0 * p) * math.exp(-t * y ** -3.0)
    norm = quad(f, 1, np.inf, args=(0, 0.0), epsabs=0, epsrel=1e-13, limit=400)[0]
    return quad(f, 1, np.inf, args=(power, tau), epsabs=0, epsrel=1e-13, limit=400)[0] / norm


@pytest.mark.parametrize("t_bb", [3e4, 1e5])
def test_spectrum_quadrature_matches_definition(t_bb):
    """The oracle's frequency nodes reproduce the surviving fraction Phi(tau) and
    the thin rate Psi(tau) (Eq. 1 integrated over a blackbody photon spectrum with
    sigma ~ nu^-3) from the defining integrals, to 1e-9 of Phi(0) = 1."""
    s, w = oracle.spectrum_nodes(t_bb)
    assert abs(w.sum() - 1) < 1e-14 and (s <= 1).all() and (s > 0).all()
    for tau in (0.0, 0.03, 0.5, 2.0, 8.0, 30.0):
        phi = float((w * np.exp(-tau * s)).sum())
        psi = float((w * s * np.exp(-tau * s)).sum())
        assert abs(phi - _bb_moment(t_bb, tau, 0)) < 1e-9
        assert abs(psi - _bb_moment(t_bb, tau, 1)) < 1e-9


@pytest.mark.parametrize("prec", [0, 1])
def test_spectrum_one_node_at_threshold_is_gray(prec):
    """A spectrum with all photons at the threshold (one node, sigma = sigma_0)
    makes Eq. 1 the gray rate: the same Gamma to rounding, the same bookkeeping."""
    w = I.random_small(16, 4, seed=62, x_mode="mixed", box_cm=16 * 3e21)
    kw = dict(overlap_mode=3, n_th_cm3=0.3 * float(w.n_h.mean()), precision=prec)
    g = oracle.run_workload(w, **kw)
    f = oracle.run_workload(w, spectrum=1, q_nodes=(np.array([1.0]), np.array([1.0])), **kw)
    for k in ("rays", "splits", "segments", "secondary", "escaped", "dropped_tau"):
        assert g["stats"][k] == f["stats"][k]
    assert relerr(f["gamma"], g["gamma"]) < (1e-13 if prec == 0 else 1e-5)
    e = g["stats"]["emitted_ph"]
    for k in ("absorbed_ph", "escaped_ph", "dropped_ph"):
        assert abs(f["stats"][k] - g["stats"][k]) <= (1e-13 if prec == 0 else 1e-6) * e


def test_spectrum_thin_path_sum():
    """Thin medium with the blackbody spectrum: every photon's share of the rate
    is weighted by its cross-section, so sum(Gamma) = Ndot sigma_0 <sigma/sigma_0> R_L / dx^2,
    <sigma/sigma_0> = Psi(0) from the defining integral (direction quantisation: 2e-6)."""
    n_h, x, cells, ndot, box, lm = _thin_uniform()
    r = oracle.run(n_h, x, cells, ndot, box, level_max=lm, overlap_mode=0, spectrum=1, t_bb_K=1e5)
    dx = box / n_h.shape[0]
    r_l = oracle.split_rq(4.0) * 2.0 ** (lm - 24)
    expect = ndot[0] * 6.3e-18 * _bb_moment(1e5, 0.0, 1) * r_l / dx ** 2
    assert abs(r["gamma"].sum() / expect - 1) < 2e-6


@pytest.mark.parametrize("prec", [0, 1])
def test_spectrum_photon_ledger(prec):
    """emitted = absorbed + escaped + dropped, deposited = absorbed (conservative
    correction), with the remaining photons of a ray B Phi(tau)."""
    w = I.random_small(20, 5, seed=63, x_mode="patchy", box_cm=20 * 2e21)
    st = oracle.run_workload(w, spectrum=1, precision=prec, overlap_mode=3)["stats"]
    e = st["emitted_ph"]
    tol = 1e-12 if prec == 0 else 1e-6
    assert abs(st["absorbed_ph"] + st["escaped_ph"] + st["dropped_ph"] - e) / e < tol
    assert abs(st["deposited_ph"] - st["absorbed_ph"]) / e < tol
    assert st["dropped_ph"] > 0            # hard photons outlive tau_max at the threshold


# ------------------------------------------------------------------ invariants

@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_photon_ledger(prec, mode):
    """emitted = absorbed + escaped + dropped; deposited (sum Gamma n_HI V) =
    absorbed for the photon-conserving modes; mode 1 (Eq. 5 alone) loses."""
    w = I.random_small(24, 6, seed=21 + mode, x_mode="patchy", box_cm=24 * 7e22)
    r = oracle.run_workload(w, precision=prec, overlap_mode=mode, n_th_cm3=0.5 * float(w.n_h.mean()))
    st = r["stats"]
    e = st["emitted_ph"]
    tol = 1e-12 if prec == 0 else 1e-6
    assert abs(st["absorbed_ph"] + st["escaped_ph"] + st["dropped_ph"] - e) / e < tol
    assert st["emitted_ph"] == pytest.approx(float(np.sum(r["emit_ndot"])), rel=1e-15)
    if mode in (0, 2, 3):
        assert abs(st["deposited_ph"] - st["absorbed_ph"]) / e < tol
    else:
        assert st["deposited_ph"] < st["absorbed_ph"] * (1 - 1e-6)


def test_linearity_in_sources():
    """At fixed x, Gamma of the union of two source sets is the sum (P6)."""
    w = I.random_small(16, 6, seed=31, x_mode="mixed", box_cm=16 * 5e22)
    # distinct cells so dedup does not merge across the two sets
    cells = np.array([[1, 2, 3], [10, 4, 7], [15, 15, 0], [5, 5, 5], [8, 1, 13], [3, 12, 9]], np.int32)
    a = oracle.run(w.n_h, w.x_ion, cells[:3], w.ndot[:3], w.box_cm)
    b = oracle.run(w.n_h, w.x_ion, cells[3:], w.ndot[3:], w.box_cm)
    ab = oracle.run(w.n_h, w.x_ion, cells, w.ndot, w.box_cm)
    assert relerr(ab["gamma"], a["gamma"] + b["gamma"]) < 1e-13
    # duplicates are exactly a summed source
    dup = oracle.run(w.n_h, w.x_ion, np.array([[5, 5, 5], [5, 5, 5]], np.int32), np.array([2e50, 3e50]),
                     w.box_cm)
    one = oracle.run(w.n_h, w.x_ion, np.array([[5, 5, 5]], np.int32), np.array([5e50]), w.box_cm)
    assert dup["stats"]["n_src_emit"] == 1
    assert relerr(dup["gamma"], one["gamma"]) < 1e-15


def test_symmetry_centred_source():
    """Odd grid, source at the centre cell, uniform gas: Gamma is invariant
    under z -> -z, x -> -x and 90 degree rotations about z (P8)."""
    n = 21
    c = n // 2
    n_h = np.full((n, n, n), 1e-3)
    x = np.full((n, n, n), 0.9)
    r = oracle.run(n_h, x, np.array([[c, c, c]], np.int32), np.array([5e48]), n * 3.182e20,
                   overlap_mode=0)
    g = r["gamma"]
    assert relerr(g[::-1, :, :], g) < 1e-12
    assert relerr(g[:, :, ::-1], g) < 1e-12
    assert relerr(np.rot90(g, 1, axes=(1, 2)), g) < 1e-12


def test_fp32_physics_close_to_fp64():
    w = I.random_small(24, 5, seed=41, x_mode="patchy", box_cm=24 * 7e22)
    r64 = oracle.run_workload(w, precision=0)
    r32 = oracle.run_workload(w, precision=1)
    assert relerr(r32["gamma"], r64["gamma"]) < 1e-5
    assert relerr(r32["heat"], r64["heat"]) < 1e-5


def test_level_max_drops_budget():
    w = I.random_small(16, 2, seed=51, x_mode="thin", box_cm=16 * 7e20)
    r = oracle.run_workload(w, level_max=2)
    st = r["stats"]
    assert sum(st["rays"][3:]) == 0 and st["dropped_level"][2] > 0
    e = st["emitted_ph"]
    assert abs(st["absorbed_ph"] + st["escaped_ph"] + st["dropped_ph"] - e) / e < 1e-12


def test_invalid_inputs_rejected():
    n = 8
    n_h = np.full((n, n, n), 1e-3)
    x = np.zeros((n, n, n))
    with pytest.raises(ValueError):
        oracle.run(n_h, x, np.array([[8, 0, 0]], np.int32), np.array([1e50]), 1e22)
    with pytest.raises(ValueError):
        oracle.run(n_h, x, np.array([[0, 0, 0]], np.int32), np.array([-1.0]), 1e22)
    bad = n_h.copy()
    bad[0, 0, 0] = np.nan
    with pytest.raises(ValueError):
        oracle.run(bad, x, np.array([[0, 0, 0]], np.int32), np.array([1e50]), 1e22)


# ------------------------------------------------------------------ chemistry (Eq. 3, C2-Ray average)

def test_chem_pure_photoionization():
    """n_e = 0 (first iterate from a neutral start): x(t) = 1 - (1 - x0) e^{-Gamma t}."""
    g = np.array([1e-12, 3e-14, 0.0])
    x0 = np.array([0.0, 0.2, 0.3])
    xa, xe, _ = oracle.chem_update(np.full(3, 1e-3), x0, np.zeros(3), g, 3e12, 2.59e-13)
    np.testing.assert_allclose(xe[:2], 1 - (1 - x0[:2]) * np.exp(-g[:2] * 3e12), rtol=1e-13)
    assert xe[2] == 0.3 and xa[2] == 0.3


def test_chem_pure_recombination():
    """Gamma = 0, fixed n_e: x(t) = x0 exp(-n_e C alpha t)."""
    n_h = np.full(2, 1e-2)
    x0 = np.array([0.9, 0.5])
    xa_prev = np.array([0.7, 0.4])
    xa, xe, _ = oracle.chem_update(n_h, x0, xa_prev, np.zeros(2), 1e13, 2.59e-13, clump=2.0)
    rate = xa_prev * n_h * 2.0 * 2.59e-13
    np.testing.assert_allclose(xe, x0 * np.exp(-rate * 1e13), rtol=1e-13)


def test_chem_time_average_is_mean_of_trajectory():
    """<x> returned equals (1/dt) integral of x(t) for the constant-rate solution."""
    n_h = np.full(3, 1e-3)
    x0 = np.array([0.1, 0.6, 0.95])
    xprev = np.array([0.3, 0.5, 0.9])
    gam = np.array([2e-14, 1e-15, 5e-13])
    dt = 4e13
    xa, xe, _ = oracle.chem_update(n_h, x0, xprev, gam, dt, 2.59e-13, C_H=1e-12, clump=1.5)
    ne = xprev * n_h
    ion = gam + ne * 1e-12
    rec = ne * 1.5 * 2.59e-13
    xeq = ion / (ion + rec)
    ts = np.linspace(0, dt, 20001)
    traj = xeq[:, None] + (x0 - xeq)[:, None] * np.exp(-(ion + rec)[:, None] * ts[None, :])
    avg = np.trapezoid(traj, ts, axis=1) / dt
    np.testing.assert_allclose(xa, avg, rtol=1e-8)
    np.testing.assert_allclose(xe, traj[:, -1], rtol=1e-13)


def test_chem_matches_ode_integration():
    """Eq. 3 at constant rates, dx/dt = (Gamma + n_e C_H)(1 - x) - n_e C alpha_B x with n_e the
    previous <x> n_H, integrated by classical fourth-order Runge-Kutta in 40000 steps: the
    oracle's x(t + dt) and time average <x> (its closed form) agree to 1e-10."""
    rng = np.random.default_rng(33)
    n_h = 10 ** rng.uniform(-4, -2, 6)
    x0 = rng.uniform(0, 1, 6)
    xprev = rng.uniform(0, 1, 6)
    gam = 10 ** rng.uniform(-16, -12, 6)
    dt, alpha, c_h, clump = 3e13, 2.59e-13, 3e-13, 2.0
    xa, xe, _ = oracle.chem_update(n_h, x0, xprev, gam, dt, alpha, C_H=c_h, clump=clump)
    ne = xprev * n_h
    f = lambda x: (gam + ne * c_h) * (1 - x) - ne * clump * alpha * x
    steps = 40000
    h = dt / steps
    x = x0.copy()
    integral = np.zeros_like(x)
    for _ in range(steps):
        k1 = f(x)
        k2 = f(x + 0.5 * h * k1)
        k3 = f(x + 0.5 * h * k2)
        k4 = f(x + h * k3)
        # Simpson's rule over the step with the Runge-Kutta midpoint estimate
        integral += h / 6 * (x + 4 * (x + 0.5 * h * (k1 + k2) / 2) + (x + h * (k1 + 2 * k2 + 2 * k3 + k4) / 6))
        x = x + h * (k1 + 2 * k2 + 2 * k3 + k4) / 6
    np.testing.assert_allclose(xe, x, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(xa, integral / dt, rtol=1e-8, atol=1e-10)


# ------------------------------------------------------------------ sources: dedup, radius, merge (Alg. 3)

def test_dedup_sorted_and_summed():
    cells = np.array([[3, 1, 2], [0, 5, 5], [3, 1, 2], [0, 5, 4], [3, 1, 2]], np.int32)
    nd = np.array([1.0, 2.0, 4.0, 8.0, 16.0])
    c, n = oracle.sources_dedup(cells, nd)
    assert c.tolist() == [[0, 5, 4], [0, 5, 5], [3, 1, 2]]
    assert n.tolist() == [8.0, 2.0, 21.0]


def test_max_radius_cases():
    n = 48
    x = np.zeros((n, n, n))
    assert oracle.max_radius(x, [24, 24, 24]) == 0.0                    # neutral source cell
    x[:] = 1.0
    assert oracle.max_radius(x, [24, 24, 24], rmax=16.0) == 16.0         # fully ionized: R_max
    # ionized ball of radius 9 around the source (cell centres)
    zz, yy, xx = np.meshgrid(*(np.arange(n),) * 3, indexing="ij")
    d = np.sqrt((xx - 24) ** 2 + (yy - 24) ** 2 + (zz - 24) ** 2)
    x = (d <= 9.0).astype(float)
    rad = oracle.max_radius(x, [24, 24, 24], dr=2.0, rmax=16.0)
    assert rad == 8.0


def _components(nsrc, edges):
    adj = {i: set() for i in range(nsrc)}
    for a, b in edges:
        adj[a].add(b)
        adj[b].add(a)
    seen, comps = set(), []
    for s in range(nsrc):
        if s in seen:
            continue
        stack, comp = [s], set()
        while stack:
            u = stack.pop()
            if u in comp:
                continue
            comp.add(u)
            stack.extend(adj[u] - comp)
        seen |= comp
        comps.append(comp)
    return comps


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_merge_components_match_dfs(seed):
    rng = np.random.default_rng(seed)
    n = 40
    x = np.clip(I.lognormal(n, 1.0, 1.5, seed + 100), 0, 1)
    cells = rng.integers(0, n, size=(60, 3)).astype(np.int32)
    c, nd = oracle.sources_dedup(cells, rng.uniform(1e50, 1e52, size=60))
    mc, mn, rad, lab = oracle.merge_sources(x, c, nd, rmax=8.0)
    edges = []
    for a, b in itertools.combinations(range(len(nd)), 2):
        if rad[a] > 0 and rad[b] > 0:
            d2 = float(np.sum((c[a].astype(np.int64) - c[b]) ** 2))
            if d2 <= (rad[a] + rad[b]) ** 2 + 1e-6:
                edges.append((a, b))
    comps = _components(len(nd), edges)
    groups = {}
    for i, l in enumerate(lab):
        groups.setdefault(int(l), set()).add(i)
    assert sorted(map(sorted, groups.values())) == sorted(map(sorted, comps))
    assert len(mn) == len(comps)
    assert abs(mn.sum() / nd.sum() - 1) < 1e-14
    member_cells = {tuple(v) for v in c.tolist()}
    assert all(tuple(v) in member_cells for v in mc.tolist())
    keys = [tuple(v) for v in mc.tolist()]
    assert keys == sorted(keys)


@pytest.mark.parametrize("cell", [[2, 30, 41], [45, 3, 20], [0, 47, 1]])
def test_max_radius_periodic_equals_translated(cell):
    """Alg. 3 under periodic (minimum-image) geometry: shell samples wrap. A
    source near the faces of a periodic grid has the radius of the same
    configuration translated so that no shell leaves the grid, traced without
    periodicity."""
    n = 48
    x = np.ones((n, n, n))
    # a neutral slab 3-6 cells beyond the nearer x face, i.e. across the boundary from the source
    step = -1 if cell[0] < n // 2 else 1
    for k in range(3, 7):
        x[:, :, (cell[0] + step * k) % n] = 0.0 if abs(cell[0] + step * k - (n // 2)) > n // 2 - 1 else 1.0
    v = [24 - c for c in cell]                          # moves the source to the centre
    xr = np.roll(x, shift=(v[2], v[1], v[0]), axis=(0, 1, 2))
    rp = oracle.max_radius(x, cell, rmax=16.0, periodic=1)
    rt = oracle.max_radius(xr, [24, 24, 24], rmax=16.0, periodic=0)
    assert rp == rt and rp > 0
    rn = oracle.max_radius(x, cell, rmax=16.0, periodic=0)
    assert rn != rp                                     # the non-periodic shells differ here


def test_merge_periodic_minimum_image_and_unwrapped_centroid():
    """Two sources across the x faces of a periodic, fully ionized grid are 3
    cells apart under the minimum image and merge; without periodicity they are
    45 apart and stay separate. The merged source is placed at the member next
    to the centroid of the unwrapped pair (near the face), not at the naive
    centroid in the middle of the box."""
    n = 48
    x = np.ones((n, n, n))
    cells = np.array([[1, 20, 20], [46, 20, 20]], np.int32)
    nd = np.array([3e52, 2e52])
    mc, mn, rad, lab = oracle.merge_sources(x, cells, nd, rmax=4.0, periodic=1)
    assert len(mn) == 1 and mn[0] == 5e52
    # unwrapped: 1 and -2, centroid (3*1 + 2*(-2))/5 = -0.2 -> 0; nearest member by minimum image: x = 1
    assert mc[0].tolist() == [1, 20, 20]
    mc2, mn2, _, _ = oracle.merge_sources(x, cells, nd, rmax=4.0, periodic=0)
    assert len(mn2) == 2
    # the naive centroid (3*1 + 2*46)/5 = 19 would snap to x = 1 as well, so weight the far member
    nd3 = np.array([1e52, 4e52])
    mc3, _, _, _ = oracle.merge_sources(x, cells, nd3, rmax=4.0, periodic=1)
    # unwrapped: (1*1 + 4*(-2))/5 = -1.4 -> -1 -> 47; nearest member by minimum image: x = 46
    assert mc3[0].tolist() == [46, 20, 20]


@pytest.mark.parametrize("seed", [4, 5])
def test_merge_components_match_dfs_periodic(seed):
    rng = np.random.default_rng(seed)
    n = 24
    # ionized balls (minimum-image distance, so they wrap) with sources scattered around their centres
    zz, yy, xx = np.meshgrid(*(np.arange(n),) * 3, indexing="ij")
    x = np.zeros((n, n, n))
    centres = rng.integers(0, n, size=(6, 3))
    for cx, cy, cz in centres:
        d = [(a - c) % n for a, c in ((xx, cx), (yy, cy), (zz, cz))]
        d = [np.where(2 * v > n, v - n, v) for v in d]
        x[(d[0] ** 2 + d[1] ** 2 + d[2] ** 2) <= rng.uniform(4, 7) ** 2] = 1.0
    pick = centres[rng.integers(0, 6, size=50)] + rng.integers(-3, 4, size=(50, 3))
    cells = (pick % n).astype(np.int32)
    c, nd = oracle.sources_dedup(cells, rng.uniform(1e50, 1e52, size=50))
    mc, mn, rad, lab = oracle.merge_sources(x, c, nd, rmax=8.0, periodic=1)
    edges = []
    for a, b in itertools.combinations(range(len(nd)), 2):
        if rad[a] > 0 and rad[b] > 0:
            d = (c[a].astype(np.int64) - c[b]) % n
            d = np.where(2 * d > n, d - n, d)
            if float(np.sum(d * d)) <= (rad[a] + rad[b]) ** 2 + 1e-6:
                edges.append((a, b))
    comps = _components(len(nd), edges)
    groups = {}
    for i, l in enumerate(lab):
        groups.setdefault(int(l), set()).add(i)
    assert sorted(map(sorted, groups.values())) == sorted(map(sorted, comps))
    assert any(len(g) > 1 for g in comps)
    assert abs(mn.sum() / nd.sum() - 1) < 1e-14
    member_cells = {tuple(v) for v in c.tolist()}
    assert all(tuple(v) in member_cells for v in mc.tolist())


def test_merge_pair_predicate_is_squared():
    """Alg. 3's pair test compares squared distance with the squared overlap length,
    d^2 <= (f_ov (r_a + r_b))^2 + eps (the text's form): two bubbles of radius 7.5 whose
    centres are 10 cells apart give both sources r = 6 (shells 2, 4, 6 fully ionized, the
    shell at 8 not), so they merge (100 <= 144) where d^2 <= f_ov (r_a + r_b) + eps would
    not (100 > 12); with f_ov = 0.8 they stay apart (100 > 92.16), so f_ov sits inside the
    square. The merged source is the member nearest the flux-weighted centroid
    floor((19 + 2 29) / 3 + 1/2) = 26, i.e. the one at 29."""
    n = 48
    zz, yy, xx = np.meshgrid(*(np.arange(n),) * 3, indexing="ij")
    x = np.zeros((n, n, n))
    for cx in (19, 29):
        x[(xx - cx) ** 2 + (yy - 24) ** 2 + (zz - 24) ** 2 <= 7.5 ** 2] = 1.0
    c, nd = oracle.sources_dedup(np.array([[19, 24, 24], [29, 24, 24]], np.int32), np.array([1e51, 2e51]))
    mc, mn, rad, lab = oracle.merge_sources(x, c, nd, f_ov=1.0)
    assert list(rad) == [6.0, 6.0]
    assert mc.tolist() == [[29, 24, 24]] and list(mn) == [3e51]
    mc, mn, rad, lab = oracle.merge_sources(x, c, nd, f_ov=0.8)
    assert len(mn) == 2 and list(mn) == [1e51, 2e51]


def test_merge_two_sources_in_one_bubble():
    n = 48
    zz, yy, xx = np.meshgrid(*(np.arange(n),) * 3, indexing="ij")
    d = np.sqrt((xx - 24) ** 2 + (yy - 24) ** 2 + (zz - 24) ** 2)
    x = (d <= 10.0).astype(float)
    cells = np.array([[22, 24, 24], [26, 24, 24], [2, 2, 2]], np.int32)
    c, nd = oracle.sources_dedup(cells, np.array([1e51, 3e51, 1e51]))
    mc, mn, rad, lab = oracle.merge_sources(x, c, nd, rmax=16.0)
    assert len(mn) == 2
    merged = mn.max()
    assert merged == 4e51
    # flux-weighted centroid (25, 24, 24) snaps to the nearest member (26, 24, 24)
    assert [26, 24, 24] in mc.tolist() and [2, 2, 2] in mc.tolist()


# ------------------------------------------------------------------ automerge switch, heating

def test_automerge_switch_equals_forced_or_no_merge():
    """Sec. 2.8: automerge (merge_mode 2) runs Alg. 3 in a step exactly when the mean ionized
    fraction exceeds the threshold. Below it the step equals the step without merging, above it
    the step with merging forced (catalog, bookkeeping and Gamma)."""
    n = 24
    zz, yy, xx = np.meshgrid(*(np.arange(n),) * 3, indexing="ij")
    x = (np.sqrt((xx - 12) ** 2 + (yy - 12) ** 2 + (zz - 12) ** 2) <= 7.0).astype(float)
    n_h = np.full((n, n, n), 2e-4)
    cells = np.array([[10, 12, 12], [14, 12, 12], [12, 10, 13], [2, 2, 2]], np.int32)
    ndot = np.array([1e51, 2e51, 3e51, 1e51])
    box = n * 7.117e23
    xbar = float(x.mean())
    kw = dict(n_th_cm3=2e-6, merge_rmax_cells=10.0)
    off = oracle.run(n_h, x, cells, ndot, box, merge_mode=0, **kw)
    forced = oracle.run(n_h, x, cells, ndot, box, merge_mode=1, **kw)
    assert forced["stats"]["merged"] == 1 and len(forced["emit_ndot"]) < len(off["emit_ndot"])
    for thr, ref in ((2.0 * xbar, off), (0.5 * xbar, forced)):
        a = oracle.run(n_h, x, cells, ndot, box, merge_mode=2, automerge_xbar=thr, **kw)
        assert a["stats"]["merged"] == ref["stats"]["merged"]
        assert np.array_equal(a["emit_cells"], ref["emit_cells"]) and np.array_equal(a["emit_ndot"], ref["emit_ndot"])
        for k in ("rays", "splits", "segments", "secondary"):
            assert a["stats"][k] == ref["stats"][k]
        assert np.array_equal(a["gamma"], ref["gamma"])


@pytest.mark.parametrize("mode", [0, 2, 3])
def test_heating_equals_absorbed_photon_energy(mode):
    """The heating grid against the ray ledger, an independent sum: with a photon-conserving
    overlap treatment every absorbed photon is deposited, so the total heating over the box,
    sum(heat) dx^3, equals e_heat times the photons absorbed along the rays (photons/s)."""
    w = I.random_small(16, 5, seed=41 + mode, x_mode="patchy", box_cm=16 * 7e22)
    e = 2.5e-12
    r = oracle.run_workload(w, overlap_mode=mode, n_th_cm3=0.3 * float(w.n_h.mean()), e_heat_erg=e)
    vol = (w.box_cm / w.n) ** 3
    total = float(r["heat"].sum()) * vol
    assert r["stats"]["absorbed_ph"] > 0
    assert abs(total / (e * r["stats"]["absorbed_ph"]) - 1) < 1e-12
