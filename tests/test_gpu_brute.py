"""GPU march against the exact-rational brute-force tracer, directly.

The oracle's traversal is an integer event machine like the kernel's; this
test takes the oracle out of the loop for the geometry. The brute force
(``brute_trace.trace``) lists every face-crossing time of a ray as an exact
fraction, sorts them and assigns each interval to the cell holding its
midpoint, and evaluates Eq. 1 and the six overlap treatments (Eqs. 5-8, the
squared f_c, the naive threshold) in plain float64 Python. On 5^3-8^3 grids,
with and without periodic boundaries (Sec. 2.5.1), the FP64 march through the
geometry tables and through the walk must reproduce its visit list (as the
order-free visit hash), its per-level ray, split, segment and secondary
counts bit for bit, and its Gamma within 1e-12 relative L2.
"""
import numpy as np
import pytest

import brute_trace as bt
from paper_2512_12466_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

M64 = (1 << 64) - 1


def splitmix64_out(z: int) -> int:
    """The splitmix64 output function (Steele, Lea & Flood 2014)."""
    z &= M64
    z ^= z >> 30
    z = (z * 0xBF58476D1CE4E5B9) & M64
    z ^= z >> 27
    z = (z * 0x94D049BB133111EB) & M64
    z ^= z >> 31
    return z


def visit_hash(visits) -> int:
    """Sum over visits of mix(mix(ray id) ^ seq 2^40 ^ cell), mod 2^64 (independent of order)."""
    h = 0
    for rid, seq, cell, _ds in visits:
        h = (h + splitmix64_out(splitmix64_out(rid) ^ (seq << 40) ^ cell)) & M64
    return h


@pytest.fixture(scope="module")
def nyx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2512_12466_gb300 as m
    m.lib()
    return m


def relerr(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


# (n, sources, seed, x field, overlap mode, n_th as a fraction of the mean n_H, periodic)
CASES = [
    (8, 3, 401, "mixed", 0, 0.01, 0),
    (7, 3, 402, "thin", 1, 0.01, 0),
    (8, 3, 403, "mixed", 2, 0.8, 0),
    (6, 3, 404, "patchy", 3, 0.5, 0),
    (8, 3, 405, "thin", 4, 0.01, 0),
    (7, 3, 406, "mixed", 5, 0.5, 0),
    (5, 2, 411, "thin", 0, 0.3, 1),
    (4, 2, 412, "mixed", 1, 0.3, 1),
    (5, 2, 413, "mixed", 2, 0.3, 1),
    (4, 2, 414, "patchy", 3, 0.3, 1),
    (5, 2, 415, "thin", 4, 0.3, 1),
    (4, 2, 416, "mixed", 5, 0.5, 1),
]


@pytest.mark.parametrize("case", CASES, ids=[f"n{c[0]}-mode{c[4]}-{'per' if c[6] else 'open'}" for c in CASES])
def test_march_matches_brute_force(nyx, case):
    n, k, seed, xm, mode, nth, periodic = case
    w = I.random_small(n, k, seed=seed, x_mode=xm, box_cm=n * 3e21)
    # the catalog the path traces is sorted and deduplicated: give both sides that catalog
    uc, inv = np.unique(w.cells, axis=0, return_inverse=True)
    ndot = np.bincount(inv.reshape(-1), weights=w.ndot)
    cells = uc.astype(np.int32)
    n_th = nth * float(w.n_h.mean())
    g_bt, vis, cnt = bt.trace(w.n_h, w.x_ion, cells, ndot, w.box_cm, overlap_mode=mode, n_th=n_th,
                              periodic=bool(periodic))
    h_bt = visit_hash(vis)
    dev = torch.device("cuda")
    for walk in (False, True):
        flags = nyx.RT_FLAG_VISIT_HASH | (nyx.RT_FLAG_NO_GEOMETRY_TABLE if walk else 0)
        s = nyx.Solver(n, w.box_cm, precision=nyx.RT_FP64, overlap_mode=mode, n_th_cm3=n_th, periodic=periodic,
                       flags=flags)
        s.set_fields(torch.from_numpy(w.n_h.ravel()).to(dev), torch.from_numpy(w.x_ion.ravel()).to(dev))
        s.add_sources(torch.from_numpy(cells.ravel()).to(dev), torch.from_numpy(ndot).to(dev))
        g = torch.empty(n ** 3, dtype=torch.float64, device=dev)
        _, _, st = s.step(0.0, g, None)
        s.close()
        path = "walk" if walk else "table"
        assert st["visit_hash"] == h_bt, path
        assert sum(st["segments"]) == len(vis), path
        for key in ("rays", "splits", "segments", "secondary"):
            got = {lvl: c for lvl, c in enumerate(st[key]) if c}
            assert got == {lvl: c for lvl, c in cnt[key].items() if c}, (path, key)
        assert relerr(g.cpu().numpy(), g_bt.reshape(-1)) < 1e-12, path
