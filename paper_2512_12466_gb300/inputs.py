"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds random-number plumbing only: Gaussian random fields,
lognormal densities, source placement and power-law luminosities. It contains
none of the ray-tracing arithmetic, so both the CUDA path and the CPU oracle
may be fed from it.

Workload shapes follow the paper's usage: lognormal gas in a cosmological box
(Sec. 4.1: h = 0.67742, 40 Mpc/h boxes), point sources at halo positions with
an ionizing photon rate per source (Sec. 2.7.1, Eq. 9), and the Stromgren
test of Table 1 (uniform gas, one source).
"""
from __future__ import annotations

import dataclasses
import numpy as np

MPC_CM = 3.0857e24          # 1 Mpc in cm
KPC_CM = 3.0857e21          # 1 kpc in cm
HUBBLE_H = 0.67742          # Sec. 4.1 cosmological parameter h
MYR_S = 3.15576e13          # 1 Myr in s (Julian years)
EV_ERG = 1.602176634e-12    # 1 eV in erg
SIGMA_HI = 6.3e-18          # gray HI cross-section at threshold, cm^2
ALPHA_B_1E4 = 2.59e-13      # case-B recombination at 1e4 K (Table 1), cm^3/s


def seed_for(config: int, stream: int, solve: int = 0) -> int:
    """Seed convention: config k uses 1000k + stream; solve j of a batch adds 100j.

    stream: 1 density field, 2 ionization field, 3 source placement,
    4 luminosities, 5 arrivals.
    """
    return 1000 * config + stream + 100 * solve


def gaussian_random_field(n: int, seed: int) -> np.ndarray:
    """Unit-variance Gaussian random field on an n^3 grid with P(k) ~ k^-2.

    White noise -> rFFT -> multiply by |k|^-1 (k in 2*pi*fftfreq units, the
    k = 0 mode zeroed) -> inverse rFFT -> standardise. Array index order is
    [iz, iy, ix] (x fastest), matching the flat layout (iz*n + iy)*n + ix.
    """
    rng = np.random.default_rng(seed)
    white = rng.standard_normal((n, n, n))
    f = np.fft.rfftn(white)
    kz = 2.0 * np.pi * np.fft.fftfreq(n)
    ky = 2.0 * np.pi * np.fft.fftfreq(n)
    kx = 2.0 * np.pi * np.fft.rfftfreq(n)
    kk = np.sqrt(kz[:, None, None] ** 2 + ky[None, :, None] ** 2 + kx[None, None, :] ** 2)
    amp = np.zeros_like(kk)
    nz = kk > 0
    amp[nz] = 1.0 / kk[nz]
    g = np.fft.irfftn(f * amp, s=(n, n, n), axes=(0, 1, 2))
    g -= g.mean()
    sd = g.std()
    if sd > 0:
        g /= sd
    return g


def lognormal(n: int, mean: float, sigma_ln: float, seed: int) -> np.ndarray:
    """Mean-preserving lognormal field: mean * exp(s g) / <exp(s g)>."""
    g = gaussian_random_field(n, seed)
    v = np.exp(sigma_ln * g)
    return mean * v / v.mean()


def place_sources(n_h: np.ndarray, count: int, seed: int, top_frac: float = 0.01) -> np.ndarray:
    """Source cells drawn uniformly with replacement among the densest cells.

    Returns int32 array (count, 3) of (ix, iy, iz). Duplicates are possible and
    intended (the path deduplicates sources that share a cell).
    """
    n = n_h.shape[0]
    flat = n_h.reshape(-1)
    k = max(1, int(round(top_frac * flat.size)))
    top = np.argpartition(flat, flat.size - k)[flat.size - k:]
    top.sort()
    rng = np.random.default_rng(seed)
    pick = top[rng.integers(0, k, size=count)]
    ix = pick % n
    iy = (pick // n) % n
    iz = pick // (n * n)
    return np.stack([ix, iy, iz], axis=1).astype(np.int32)


def power_law_ndot(count: int, seed: int, lo: float = 1e50, hi: float = 1e53) -> np.ndarray:
    """Photon rates with dN/dNdot ~ Ndot^-2 on [lo, hi] by inverse-CDF sampling."""
    rng = np.random.default_rng(seed)
    u = rng.random(count)
    return 1.0 / (1.0 / lo - u * (1.0 / lo - 1.0 / hi))


@dataclasses.dataclass
class Workload:
    """One solve: grid, physics parameters and sources (host numpy arrays)."""
    name: str
    n: int
    box_cm: float
    n_h: np.ndarray                 # (n, n, n) float64, cm^-3
    x_ion: np.ndarray               # (n, n, n) float64, ionized fraction
    cells: np.ndarray               # (S, 3) int32 source cells (ix, iy, iz)
    ndot: np.ndarray                # (S,) float64 photons/s
    params: dict = dataclasses.field(default_factory=dict)

    @property
    def dx_cm(self) -> float:
        return self.box_cm / self.n


def stromgren_test_a(n: int = 64) -> Workload:
    """Table 1 Test A: n_H = 1e-3, Ndot = 5e48, L = 6.6 kpc, T = 1e4 K, neutral.

    The source sits in cell (n/2, n/2, n/2); its rays start at that cell's
    centre.
    """
    n_h = np.full((n, n, n), 1e-3)
    x = np.zeros((n, n, n))
    c = n // 2
    return Workload(
        name=f"stromgren_A_{n}", n=n, box_cm=6.6 * KPC_CM, n_h=n_h, x_ion=x,
        cells=np.array([[c, c, c]], dtype=np.int32), ndot=np.array([5e48]),
        params=dict(n_min_ray=4.0, tau_max=30.0, dt_s=0.1 * MYR_S, chem_iterate=1,
                    alpha_B=ALPHA_B_1E4, clumping=1.0, C_H=0.0),
    )


# Table 1 Stromgren test problems: (n_H cm^-3, Ndot s^-1, clumping C, L_box Mpc), all at T = 1e4 K.
TABLE1 = {"A": (1e-3, 5e48, 1.0, 0.0066), "B": (1.87e-4, 1e54, 5.0, 1.62), "C": (1.87e-4, 1e57, 1.0, 10.0)}


def stromgren_test(name: str, n: int = 64) -> Workload:
    """Table 1 Test A, B or C on an n^3 grid: uniform neutral hydrogen, one
    source in cell (n/2, n/2, n/2) (centre of the box, to half a cell)."""
    n_hv, ndot, clump, lbox = TABLE1[name]
    c = n // 2
    return Workload(
        name=f"stromgren_{name}_{n}", n=n, box_cm=lbox * MPC_CM, n_h=np.full((n, n, n), n_hv),
        x_ion=np.zeros((n, n, n)), cells=np.array([[c, c, c]], dtype=np.int32), ndot=np.array([ndot]),
        params=dict(n_min_ray=4.0, tau_max=30.0, chem_iterate=1, alpha_B=ALPHA_B_1E4, clumping=clump, C_H=0.0),
    )


def cosmo_box(n: int, box_mpc_h: float, sigma_ln: float, n_sources: int, config: int,
              x_mode: str = "neutral", solve: int = 0, mean_nh: float = 2e-4,
              x_sigma_ln: float = 1.5, thin_xhi: float = 1e-4) -> Workload:
    """Lognormal gas with power-law sources in the densest 1% of cells.

    x_mode: "neutral" (x = 0), "thin" (uniform residual neutral fraction
    thin_xhi), or "patchy" (x = clip(v, 0, 1), v a mean-1 lognormal with
    x_sigma_ln on an independent seed, i.e. x_HI = 1 - clip(v, 0, 1)).
    """
    n_h = lognormal(n, mean_nh, sigma_ln, seed_for(config, 1, solve))
    if x_mode == "neutral":
        x = np.zeros_like(n_h)
    elif x_mode == "thin":
        x = np.full_like(n_h, 1.0 - thin_xhi)
    elif x_mode == "patchy":
        v = lognormal(n, 1.0, x_sigma_ln, seed_for(config, 2, solve))
        x = np.clip(v, 0.0, 1.0)
    else:
        raise ValueError(x_mode)
    cells = place_sources(n_h, n_sources, seed_for(config, 3, solve))
    ndot = power_law_ndot(n_sources, seed_for(config, 4, solve))
    box_cm = box_mpc_h / HUBBLE_H * MPC_CM
    return Workload(name=f"cosmo_{n}_{n_sources}_{x_mode}", n=n, box_cm=box_cm, n_h=n_h,
                    x_ion=x, cells=cells, ndot=ndot,
                    params=dict(n_min_ray=4.0, tau_max=30.0))


def config2(x_mode: str = "thin", n_sources: int = 1024) -> Workload:
    """128^3, 20 Mpc/h, sigma_ln = 1.0, mean n_H = 2e-4, 1024 power-law sources."""
    return cosmo_box(128, 20.0, 1.0, n_sources, config=2, x_mode=x_mode)


def config4(n_sources: int = 32768) -> Workload:
    """256^3, 40 Mpc/h, sigma_ln = 1.5, patchy x_HI, 32768 sources (merging on)."""
    return cosmo_box(256, 40.0, 1.5, n_sources, config=4, x_mode="patchy")


def thin256(n_sources: int = 64) -> Workload:
    """256^3, 40 Mpc/h, sigma_ln = 1.5 (the config-4 density field) in the optically thin
    variant (uniform residual x_HI = 1e-4), with the first n_sources of config 4's power-law
    sources: the box whose kappa and Gamma (67 + 134 MB in FP32 physics) exceed the L2 cache."""
    w = cosmo_box(256, 40.0, 1.5, 32768, config=4, x_mode="thin")
    w.cells, w.ndot = w.cells[:n_sources].copy(), w.ndot[:n_sources].copy()
    w.name = f"cosmo_256_{n_sources}_thin"
    return w


def batch_solves(count: int = 64, config: int = 3, x_mode: str = "thin",
                 sizes=(32, 64, 96, 128), max_sources: int = 4096):
    """Batched workload: grid sizes uniform over `sizes`, source counts
    floor(exp(U * ln(max_sources + 1))) clipped to [1, max_sources], boxes with the
    128^3 / 20 Mpc/h cell size."""
    rng = np.random.default_rng(seed_for(config, 5))
    out = []
    for j in range(count):
        n = int(sizes[rng.integers(0, len(sizes))])
        s = int(np.clip(np.floor(np.exp(rng.random() * np.log(max_sources + 1))), 1, max_sources))
        out.append(cosmo_box(n, 20.0 * n / 128.0, 1.0, s, config=config, x_mode=x_mode, solve=j))
    return out


def poisson_arrivals(rate_hz: float, count: int, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson stream."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_hz, size=count))


def random_small(n: int, n_sources: int, seed: int, x_mode: str = "thin",
                 sigma_ln: float = 1.0, mean_nh: float = 2e-4, box_cm: float | None = None,
                 thin_xhi: float = 1e-3) -> Workload:
    """Small seeded case for parity tests: lognormal gas, sources anywhere."""
    rng = np.random.default_rng(seed)
    n_h = lognormal(n, mean_nh, sigma_ln, seed + 1)
    if x_mode == "neutral":
        x = np.zeros_like(n_h)
    elif x_mode == "thin":
        x = np.full_like(n_h, 1.0 - thin_xhi)
    elif x_mode == "patchy":
        v = lognormal(n, 1.0, 1.5, seed + 2)
        x = np.clip(v, 0.0, 1.0)
    elif x_mode == "mixed":
        x = rng.random(n_h.shape)
        x[rng.random(n_h.shape) < 0.2] = 1.0
    else:
        raise ValueError(x_mode)
    cells = rng.integers(0, n, size=(n_sources, 3)).astype(np.int32)
    ndot = power_law_ndot(n_sources, seed + 3)
    if box_cm is None:
        box_cm = n * 7.117e23 / 1e3   # cells ~ 1/1000 of the cosmological cell: moderate opacity
    return Workload(name=f"small_{n}_{n_sources}_{x_mode}_{seed}", n=n, box_cm=box_cm,
                    n_h=n_h, x_ion=x, cells=cells, ndot=ndot,
                    params=dict(n_min_ray=4.0, tau_max=30.0))
