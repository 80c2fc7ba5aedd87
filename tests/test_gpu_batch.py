"""Batched form (one persistent cooperative launch over many solves) against
the per-solve path and the CPU oracle.

Each solve in a batch must give exactly the bookkeeping (per-level counts,
visit hash) of rt_step on the same handle, and the same fields up to the
order of FP64 atomic deposits; graph replay, tuned launch shapes and tiny
slices (deep device-side recursion) must not change any result.
"""
import numpy as np
import pytest

import oracle
from paper_2512_12466_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BOOK = ("rays", "splits", "escaped", "dropped_tau", "dropped_level", "segments", "secondary", "visit_hash")


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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).ravel()).cuda()


def mixed_workloads(count=6, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for j in range(count):
        n = int(rng.choice([8, 16, 24, 33, 40]))
        k = int(rng.integers(1, 20))
        xm = ["thin", "patchy", "mixed"][j % 3]
        dxc = [7e20, 2e22, 7e22][j % 3]
        out.append(I.random_small(n, k, seed=1000 + 17 * j + seed, x_mode=xm, box_cm=n * dxc))
    return out


def make_solver(nyx, w, precision, **kw):
    s = nyx.Solver(w.n, w.box_cm, precision=precision, n_th_cm3=0.3 * float(w.n_h.mean()),
                   flags=nyx.RT_FLAG_VISIT_HASH, **kw)
    s.set_fields(dev(w.n_h), dev(w.x_ion))
    s.add_sources(dev(w.cells.astype(np.int32)), dev(w.ndot))
    return s


def plain(nyx, s, n):
    g = torch.empty(n ** 3, dtype=torch.float64, device="cuda")
    h = torch.empty_like(g)
    _, _, st = s.step(0.0, g, h)
    return g.cpu().numpy(), h.cpu().numpy(), st


def run_batch(nyx, b, ws):
    gs = [torch.empty(w.n ** 3, dtype=torch.float64, device="cuda") for w in ws]
    hs = [torch.empty_like(g) for g in gs]
    stats = b.run(gs, hs)
    return [g.cpu().numpy() for g in gs], [h.cpu().numpy() for h in hs], stats


@pytest.mark.parametrize("heavy_shift", [0, -1], ids=["default", "all-heavy"])
@pytest.mark.parametrize("precision", [0, 1])
def test_batch_matches_per_solve(nyx, precision, heavy_shift):
    # heavy_shift -1: every solve on the heavy path (chunks of sources, device-sized per-level
    # launches on parallel streams); by default these small solves share persistent launches
    ws = mixed_workloads()
    solvers = [make_solver(nyx, w, precision) for w in ws]
    ref = [plain(nyx, s, w.n) for s, w in zip(solvers, ws)]
    b = nyx.Batch(solvers)
    b.set_params(heavy_shift=heavy_shift)
    gs, hs, stats = run_batch(nyx, b, ws)
    tol = 1e-12 if precision == 0 else 1e-10
    for (gr, hr, sr), g, h, st in zip(ref, gs, hs, stats):
        for k in BOOK:
            assert st[k] == sr[k], k
        assert st["n_src_emit"] == sr["n_src_emit"]
        assert relerr(g, gr) < tol and relerr(h, hr) < tol
        assert abs(st["deposited_ph"] - sr["deposited_ph"]) <= 1e-10 * max(1.0, sr["emitted_ph"])
    if precision == 1:
        # the batched FP32 solves against the oracle: bookkeeping and visit hash bit-exact with its
        # FP32 variant, fields within 1e-5 of the FP64 oracle
        for w, g, h, st in zip(ws, gs, hs, stats):
            n_th = 0.3 * float(w.n_h.mean())
            r32 = oracle.run_workload(w, n_th_cm3=n_th, precision=1)
            r64 = oracle.run_workload(w, n_th_cm3=n_th, precision=0)
            for k in BOOK:
                assert st[k] == r32["stats"][k], k
            assert relerr(g, r64["gamma"].ravel()) < 1e-5
            assert relerr(h, r64["heat"].ravel()) < 1e-5
    b.close()
    for s in solvers:
        s.close()


@pytest.mark.parametrize("heavy_shift", [0, -1], ids=["default", "all-heavy"])
def test_batch_matches_oracle(nyx, heavy_shift):
    ws = mixed_workloads(count=3, seed=5)
    solvers = [make_solver(nyx, w, 0) for w in ws]
    b = nyx.Batch(solvers)
    b.set_params(heavy_shift=heavy_shift)
    gs, _, stats = run_batch(nyx, b, ws)
    for w, g, st in zip(ws, gs, stats):
        r = oracle.run_workload(w, n_th_cm3=0.3 * float(w.n_h.mean()))
        for k in BOOK:
            assert st[k] == (r["stats"][k] if k != "visit_hash" else r["stats"]["visit_hash"]), k
        assert relerr(g.reshape(w.n, w.n, w.n), r["gamma"]) < 1e-12
    b.close()


def test_batch_graph_replay_tune_and_tiny_slices(nyx):
    ws = mixed_workloads(count=5, seed=9)
    solvers = [make_solver(nyx, w, 1) for w in ws]
    b = nyx.Batch(solvers)
    g0, h0, s0 = run_batch(nyx, b, ws)
    b.capture()
    for _ in range(2):                               # graph replays
        g1, h1, s1 = run_batch(nyx, b, ws)
        for a, c in zip(s0, s1):
            for k in BOOK:
                assert a[k] == c[k]
        assert all(relerr(x, y) < 1e-10 for x, y in zip(g1, g0))
    best, ms = b.tune(repeats=1)
    assert best.block in (128, 256) and best.tile % 32 == 0 and ms > 0
    g2, _, s2 = run_batch(nyx, b, ws)               # tuned shape, graph re-captured
    for a, c in zip(s0, s2):
        for k in BOOK:
            assert a[k] == c[k]
    b.set_params(slice=1024, tile=32)                # many slices: deep device-side recursion
    g3, _, s3 = run_batch(nyx, b, ws)
    for a, c in zip(s0, s3):
        for k in BOOK:
            assert a[k] == c[k]
    assert all(relerr(x, y) < 1e-10 for x, y in zip(g3, g0))
    for gb in (1, 0):                                # one launch per solve; all solves in one launch
        b.set_params(slice=1 << 22, tile=256, group_bytes=gb)
        g4, _, s4 = run_batch(nyx, b, ws)
        for a, c in zip(s0, s4):
            for k in BOOK:
                assert a[k] == c[k]
        assert all(relerr(x, y) < 1e-10 for x, y in zip(g4, g0))
    b.close()
    for s in solvers:
        s.close()


def test_batch_sees_field_updates(nyx):
    ws = mixed_workloads(count=2, seed=11)
    solvers = [make_solver(nyx, w, 0) for w in ws]
    b = nyx.Batch(solvers)
    b.capture()
    run_batch(nyx, b, ws)
    x2 = np.clip(ws[0].x_ion * 0.5, 0, 1)
    solvers[0].set_fields(dev(ws[0].n_h), dev(x2))
    gs, _, stats = run_batch(nyx, b, ws)
    w2 = I.Workload("u", ws[0].n, ws[0].box_cm, ws[0].n_h, x2, ws[0].cells, ws[0].ndot, ws[0].params)
    r = oracle.run_workload(w2, n_th_cm3=0.3 * float(ws[0].n_h.mean()))
    assert stats[0]["visit_hash"] == r["stats"]["visit_hash"]
    assert relerr(gs[0].reshape(w2.n, w2.n, w2.n), r["gamma"]) < 1e-12
    b.close()


def test_batch_rejects_mixed_precision_and_chemistry(nyx):
    ws = mixed_workloads(count=2, seed=13)
    a = make_solver(nyx, ws[0], 0)
    c = make_solver(nyx, ws[1], 1)
    with pytest.raises(nyx.NyxError) as e:
        nyx.Batch([a, c])
    assert e.value.code == nyx.RT_EINVAL
    d = make_solver(nyx, ws[1], 0, chem_iterate=1)
    with pytest.raises(nyx.NyxError):
        nyx.Batch([a, d])
    for s in (a, c, d):
        s.close()


@pytest.mark.parametrize("heavy_shift", [0, -1], ids=["default", "all-heavy"])
@pytest.mark.parametrize("precision", [0, 1])
def test_batch_periodic_matches_per_solve(nyx, precision, heavy_shift):
    """Periodic solves (Sec. 2.5.1) in one batch, with the geometry tables of their shared grid
    size, against rt_step on each: in the persistent kernel and on the heavy path."""
    ws = [I.random_small(24, 5 + j, seed=700 + j, x_mode=["thin", "mixed", "patchy"][j % 3], box_cm=24 * 3e21)
          for j in range(4)]
    solvers = [make_solver(nyx, w, precision, periodic=1) for w in ws]
    ref = [plain(nyx, s, w.n) for s, w in zip(solvers, ws)]
    b = nyx.Batch(solvers)
    b.set_params(heavy_shift=heavy_shift)
    gs, hs, stats = run_batch(nyx, b, ws)
    tol = 1e-12 if precision == 0 else 1e-10
    for (gr, hr, sr), g, st in zip(ref, gs, stats):
        for k in BOOK:
            assert st[k] == sr[k], k
        assert relerr(g, gr) < tol
    b.close()
    for s in solvers:
        s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_heavy_path_many_chunks(nyx, precision):
    """Solves with more sources than one heavy-path chunk holds (24^3 grids, about 1400 distinct
    source cells against chunks of 512): every chunk's levels sized on the device, chunks spread
    over the lanes, each solve equal to rt_step on it (bookkeeping bit for bit), graph replay
    included."""
    ws = [I.random_small(24, 1500, seed=810 + j, x_mode=["thin", "mixed"][j], box_cm=24 * 7e20) for j in range(2)]
    solvers = [make_solver(nyx, w, precision) for w in ws]
    ref = [plain(nyx, s, w.n) for s, w in zip(solvers, ws)]
    assert all(r[2]["n_src_emit"] > 1024 for r in ref)
    b = nyx.Batch(solvers)
    b.set_params(heavy_shift=-1)
    tol = 1e-12 if precision == 0 else 1e-10
    for replay in (False, True):
        if replay:
            b.capture()
        gs, hs, stats = run_batch(nyx, b, ws)
        for (gr, hr, sr), g, h, st in zip(ref, gs, hs, stats):
            for k in BOOK:
                assert st[k] == sr[k], k
            assert relerr(g, gr) < tol and relerr(h, hr) < tol
            assert st["table_levels"] & 1                     # level 0 read its table
    b.close()
    for s in solvers:
        s.close()


@pytest.mark.parametrize("heavy_shift", [0, -1], ids=["light", "heavy"])
@pytest.mark.parametrize("precision", [0, 1])
def test_batch_blackbody_rate(nyx, precision, heavy_shift):
    """Eq. 1 integrated over a blackbody spectrum in the batched form, through the persistent
    kernel (light, the default before any run) and through the per-level launches (heavy): each
    solve equal to rt_step (bookkeeping bit for bit, fields to the atomics' order) and, for one
    solve, to the oracle's direct quadrature (FP64 1e-9; FP32 2e-6 of the FP64 oracle)."""
    ws = mixed_workloads(count=4, seed=23)
    kw = dict(spectrum=1, t_bb_K=1e5)
    solvers = [make_solver(nyx, w, precision, **kw) for w in ws]
    ref = [plain(nyx, s, w.n) for s, w in zip(solvers, ws)]
    b = nyx.Batch(solvers)
    b.set_params(heavy_shift=heavy_shift)
    gs, hs, stats = run_batch(nyx, b, ws)
    tol = 1e-12 if precision == 0 else 1e-10
    for (gr, hr, sr), g, st in zip(ref, gs, stats):
        for k in BOOK:
            assert st[k] == sr[k], k
        assert relerr(g, gr) < tol
    w = ws[0]
    n_th = 0.3 * float(w.n_h.mean())
    r = oracle.run_workload(w, n_th_cm3=n_th, precision=precision, **kw)
    for k in BOOK:
        assert stats[0][k] == r["stats"][k], k
    r64 = r if precision == 0 else oracle.run_workload(w, n_th_cm3=n_th, precision=0, **kw)
    assert relerr(gs[0].reshape(w.n, w.n, w.n), r64["gamma"]) < (1e-9 if precision == 0 else 2e-6)
    b.close()
    for s in solvers:
        s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_mixes_rates(nyx, precision):
    """Gray solves and blackbody solves at two temperatures in one batch: the persistent launches
    hold one rate each, and every solve equals its own rt_step."""
    ws = mixed_workloads(count=6, seed=29)
    rates = [dict(), dict(spectrum=1, t_bb_K=1e5), dict(spectrum=1, t_bb_K=3e4)] * 2
    solvers = [make_solver(nyx, w, precision, **kw) for w, kw in zip(ws, rates)]
    ref = [plain(nyx, s, w.n) for s, w in zip(solvers, ws)]
    b = nyx.Batch(solvers)
    gs, hs, stats = run_batch(nyx, b, ws)
    tol = 1e-12 if precision == 0 else 1e-10
    for (gr, hr, sr), g, st in zip(ref, gs, stats):
        for k in BOOK:
            assert st[k] == sr[k], k
        assert relerr(g, gr) < tol
    b.close()
    for s in solvers:
        s.close()
