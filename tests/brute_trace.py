"""Brute-force reference for tiny grids, used to pin the C oracle.

Independent of the oracle's code: its own HEALPix pixel centres, and a
different traversal algorithm. Instead of stepping cell to cell, it lists every
face-crossing time of a ray as an exact rational (Python ``fractions``),
sorts them with the start and split radii, and assigns each interval to the
cell containing its midpoint. Physics is plain float64 Python.

The readings it shares with the oracle are the definitions themselves
(quantised HEALPix directions, split radius R_l = Rq 2^l / 2^24, the
gray photon-conserving rate, the Eq. 5-8 correction measured from the
segment midpoint), not any code.
"""
from __future__ import annotations

import math
from fractions import Fraction as Fr

import numpy as np

S = 21
F = 24


def healpix_nest_vec(level: int, pix: int):
    """HEALPix nested pixel centre (Gorski et al. 2005), written from the
    scheme's definition: the 12 base faces, the Z-order index within a face,
    rings of constant z, equal spacing in phi within a ring."""
    nside = 2 ** level
    face, ipf = divmod(pix, nside * nside)
    fx = fy = 0
    for b in range(level):
        fx += ((ipf >> (2 * b)) & 1) << b
        fy += ((ipf >> (2 * b + 1)) & 1) << b
    face_row = face // 4                      # 0: north faces, 1: equatorial, 2: south
    ring = (face_row + 2) * nside - fx - fy - 1
    face_col = [1, 3, 5, 7, 0, 2, 4, 6, 1, 3, 5, 7][face]
    if ring < nside:
        nr = ring
        q = (nr * nr) / (3 * nside * nside)
        z = 1.0 - q
        sth = math.sqrt(q * (2.0 - q))
        shift = 0
    elif ring > 3 * nside:
        nr = 4 * nside - ring
        q = (nr * nr) / (3 * nside * nside)
        z = q - 1.0
        sth = math.sqrt(q * (2.0 - q))
        shift = 0
    else:
        nr = nside
        z = ((2 * nside - ring) * 2.0) / (3 * nside)
        sth = math.sqrt((1.0 - z) * (1.0 + z))
        shift = (ring - nside) & 1
    jp = (face_col * nr + fx - fy + 1 + shift) // 2
    if jp > 4 * nside:
        jp -= 4 * nside
    if jp < 1:
        jp += 4 * nside
    phi = ((jp - 0.5 * (shift + 1)) * (math.pi / 2)) / nr
    return (sth * math.cos(phi), sth * math.sin(phi), z)


def quantise(v):
    q = []
    for c in v:
        m = int(math.floor(abs(c) * 2 ** S + 0.5))
        q.append(-m if c < 0 else m)
    return q


def split_rq(n_min: float) -> int:
    return int(math.floor(math.sqrt(3.0 / (math.pi * n_min)) * 2 ** F + 0.5))


def periodic_rs(n: int) -> int:
    """Travel-distance cutoff sqrt(3) L_box of periodic boundaries, in 2^-24 cells."""
    return int(math.floor(math.sqrt(3.0) * n * 2 ** F + 0.5))


def ray_segments(n: int, cell0, sd, level: int, rq: int, periodic: bool = False):
    """Exact segments of one ray between R_{l-1} and R_l (periodic: and at most
    the travel distance sqrt(3) n, which ends it without a split when it comes
    first or at the same point).

    Returns (segments, outcome) with segments = list of (cell_xyz, t_a, t_b)
    (Fractions; cells unwrapped, i.e. floor of the position) and outcome in
    {"split", "escape", "stop"}.
    """
    t0 = Fr(rq * 2 ** (level - 1), 2 ** F) if level > 0 else Fr(0)
    t1 = Fr(rq * 2 ** level, 2 ** F)
    outcome = "split"
    if periodic and rq * 2 ** level >= periodic_rs(n):
        t1 = Fr(periodic_rs(n), 2 ** F)
        outcome = "stop"
    times = {t0, t1}
    for a in range(3):
        d = abs(sd[a])
        if d == 0:
            continue
        k = 0
        while True:
            t = Fr((2 * k + 1) * 2 ** (S - 1), d)
            if t >= t1:
                break
            if t > t0:
                times.add(t)
            k += 1
    ts = sorted(times)
    segs = []
    for ta, tb in zip(ts[:-1], ts[1:]):
        tm = (ta + tb) / 2
        cell = []
        for a in range(3):
            pos = Fr(2 * cell0[a] + 1, 2) + tm * Fr(sd[a], 2 ** S)
            cell.append(math.floor(pos))
        if not periodic and any(c < 0 or c >= n for c in cell):
            return segs, "escape"
        segs.append((tuple(cell), ta, tb))
    return segs, outcome


def face_distance(cell, sd, tm, cell0):
    """Distance from the point at parameter tm to the six faces of `cell`,
    order x-, x+, y-, y+, z-, z+ (exact)."""
    out = []
    for a in range(3):
        pos = Fr(2 * cell0[a] + 1, 2) + tm * Fr(sd[a], 2 ** S)
        lo = pos - cell[a]
        out.append(lo)
        out.append(1 - lo)
    return out


def trace(n_h, x, cells, ndot, box_cm, sigma=6.3e-18, n_min=4.0, tau_max=30.0, level_max=None,
          overlap_mode=0, n_th=0.0, periodic=False):
    """Gamma field and visit list by brute force (FP64 physics); periodic:
    cells wrap around the box and rays stop at travel distance sqrt(3) n."""
    n = n_h.shape[0]
    dx = box_cm / n
    nhi = (1.0 - x) * n_h
    kap = (sigma * dx) * nhi
    elig = (n_h >= n_th) & (nhi > 0)
    rq = split_rq(n_min)
    if level_max is None:
        lvl = 0
        while rq * 2.0 ** (lvl - F) < math.sqrt(3.0) * n:
            lvl += 1
        level_max = lvl + 1
    gamma = np.zeros_like(n_h)
    visits = []
    counts = dict(rays={}, splits={}, segments={}, secondary={})
    sigma_over_dx2 = sigma / (dx * dx)
    for j, (c0, nd) in enumerate(zip(cells, ndot)):
        c0 = [int(v) for v in c0]
        g_src = (nd / 12.0) * sigma_over_dx2
        stack = [(0, p, 1.0, 0.0) for p in range(12)]
        while stack:
            lvl, pix, P, tau = stack.pop()
            counts["rays"][lvl] = counts["rays"].get(lvl, 0) + 1
            sd = quantise(healpix_nest_vec(lvl, pix))
            nrm = math.sqrt(sum(v * v for v in sd)) / 2 ** S
            segs, outcome = ray_segments(n, c0, sd, lvl, rq, periodic)
            rid = (j << 36) | (lvl << 31) | pix
            dropped = False
            for seq, (ucell, ta, tb) in enumerate(segs):
                cell = tuple(c % n for c in ucell)       # the same cell unless periodic
                ix, iy, iz = cell
                ds = float(tb - ta) * nrm
                k = kap[iz, iy, ix]
                dtau = k * ds
                if k > 0:
                    a = P * (-math.expm1(-dtau))
                    gseg = (a * g_src) / k
                else:
                    a = 0.0
                    gseg = (P * g_src) * ds
                f = 1.0
                nb = None
                if overlap_mode != 0:
                    tm = (ta + tb) / 2
                    dist = face_distance(ucell, sd, tm, c0)
                    q = min(range(6), key=lambda i: (dist[i], i))
                    de = float(dist[q])
                    lpix = float(tm) * nrm * math.sqrt(math.pi / 3.0) / 2 ** lvl
                    if 2 * de < lpix:
                        if overlap_mode == 1:                    # Eq. 5 alone
                            f = 0.5 + de / lpix
                        elif overlap_mode == 4:                  # squared f_c, nothing to the neighbour
                            f = (0.5 + de / lpix) ** 2
                        else:
                            if overlap_mode == 5:                # naive threshold: Eq. 5 share regardless
                                f = 0.5 + de / lpix
                            nbc = list(cell)
                            nbc[q // 2] += 1 if q % 2 else -1
                            if periodic:
                                nbc = [v % n for v in nbc]
                            if all(0 <= v < n for v in nbc):
                                kn = kap[nbc[2], nbc[1], nbc[0]]
                                ok = elig[nbc[2], nbc[1], nbc[0]] if overlap_mode in (3, 5) else kn > 0
                                if ok:
                                    f = 0.5 + de / lpix
                                    nb = (nbc, ((1.0 - f) * gseg) * (k / kn))
                gamma[iz, iy, ix] += f * gseg
                if nb is not None:
                    gamma[nb[0][2], nb[0][1], nb[0][0]] += nb[1]
                    counts["secondary"][lvl] = counts["secondary"].get(lvl, 0) + 1
                counts["segments"][lvl] = counts["segments"].get(lvl, 0) + 1
                visits.append((rid, seq, (iz * n + iy) * n + ix, ds))
                tau += dtau
                P -= a
                if tau >= tau_max:
                    dropped = True
                    break
            if dropped or outcome != "split":
                continue
            if lvl + 1 > level_max:
                continue
            counts["splits"][lvl] = counts["splits"].get(lvl, 0) + 1
            for q in range(4):
                stack.append((lvl + 1, 4 * pix + q, P * 0.25, tau))
    return gamma, visits, counts
