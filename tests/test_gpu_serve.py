"""Serving loop: continuous batching with admission by device memory.

Each request's result must be the same alone (rt_step on its own handle) and
in the mix (traced in a batch with whatever else was loaded at the time):
bookkeeping and visit hash equal, fields within 1e-10 relative L2 (only the
order of FP64 atomic deposits differs). Each served result is also checked
against the CPU oracle run on that request alone (the iterative solve of
Sec. 2.4, Alg. 2 per request): FP32 bookkeeping and visit hash bit-exact with
the oracle's FP32 variant and fields within 1e-5 of the FP64 oracle; FP64
bookkeeping bit-exact and fields within 1e-12. The admitted device bytes never
exceed the budget, and requests submitted while batches run are served by
later batches.
"""
import time

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


def requests(count, seed):
    rng = np.random.default_rng(seed)
    out = []
    for j in range(count):
        n = int(rng.choice([16, 24, 32, 48]))
        k = int(rng.integers(1, 40))
        xm = ["thin", "patchy", "mixed", "neutral"][j % 4]
        out.append(I.random_small(n, k, seed=seed * 1000 + j, x_mode=xm, box_cm=n * [7e20, 2e22, 7e22, 1e21][j % 4]))
    return out


def alone(nyx, w, precision, n_th):
    s = nyx.Solver(w.n, w.box_cm, precision=precision, n_th_cm3=n_th, flags=nyx.RT_FLAG_VISIT_HASH)
    s.set_fields(w.n_h.ravel(), w.x_ion.ravel())
    s.add_sources(w.cells.ravel(), w.ndot)
    g, h, st = s.step()
    s.close()
    return g.ravel(), h.ravel(), st


def check_same(nyx, got, ref):
    g, h, st, lat = got
    gr, hr, sr = ref
    for k in BOOK:
        assert st[k] == sr[k], k
    assert relerr(g, gr) < 1e-10 and relerr(h, hr) < 1e-10
    assert lat > 0


@pytest.mark.parametrize("precision", [1, 0])
def test_each_result_same_alone_and_in_the_mix(nyx, precision):
    ws = requests(12, seed=3 + precision)
    srv = nyx.Server(precision=precision, max_batch=8)
    ids = []
    for w in ws:
        n_th = 0.3 * float(w.n_h.mean())
        ids.append(srv.submit(w.n, w.box_cm, w.n_h, w.x_ion, w.cells, w.ndot, n_th_cm3=n_th,
                              flags=nyx.RT_FLAG_VISIT_HASH))
    got = [srv.poll(i, wait_s=120.0) for i in ids]
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(ws) and st["failed"] == 0 and st["batches"] >= 2
    assert st["p99_ms"] >= st["p50_ms"] > 0
    for w, r in zip(ws, got):
        assert r is not None
        check_same(nyx, r, alone(nyx, w, precision, 0.3 * float(w.n_h.mean())))
        check_oracle(w, r, precision, 0.3 * float(w.n_h.mean()))


def check_oracle(w, got, precision, n_th):
    """A served result against the oracle on the same request alone."""
    g, h, st, _ = got
    ref64 = oracle.run_workload(w, n_th_cm3=n_th, precision=0)
    ref = ref64 if precision == 0 else oracle.run_workload(w, n_th_cm3=n_th, precision=1)
    for k in BOOK:
        assert st[k] == ref["stats"][k], k
    tol = 1e-12 if precision == 0 else 1e-5
    assert relerr(g.ravel(), ref64["gamma"].ravel()) < tol
    assert relerr(h.ravel(), ref64["heat"].ravel()) < tol


def test_admission_respects_the_memory_budget(nyx):
    ws = requests(6, seed=9)
    budget = max(w.n ** 3 * 36 + 160 * 1024 + (1 << 16) for w in ws) * 2   # two of the largest at a time
    srv = nyx.Server(precision=1, max_batch=64, hbm_budget=budget)
    ids = [srv.submit(w.n, w.box_cm, w.n_h, w.x_ion, w.cells, w.ndot, n_th_cm3=0.3 * float(w.n_h.mean()),
                      flags=nyx.RT_FLAG_VISIT_HASH) for w in ws]
    got = [srv.poll(i, wait_s=120.0) for i in ids]
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(ws) and st["mem_peak"] <= budget and st["batches"] >= 2
    for w, r in zip(ws, got):
        check_same(nyx, r, alone(nyx, w, 1, 0.3 * float(w.n_h.mean())))


def test_requests_arriving_during_batches_are_served(nyx):
    ws = requests(16, seed=21)
    srv = nyx.Server(precision=1, max_batch=4)
    ids = []
    for j, w in enumerate(ws):
        ids.append(srv.submit(w.n, w.box_cm, w.n_h, w.x_ion, w.cells, w.ndot, n_th_cm3=0.3 * float(w.n_h.mean()),
                              flags=nyx.RT_FLAG_VISIT_HASH))
        if j % 4 == 3:
            time.sleep(0.02)                     # later requests arrive while earlier ones run
    got = [srv.poll(i, wait_s=120.0) for i in ids]
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(ws) and st["batches"] >= 4
    for w, r in zip(ws, got):
        check_same(nyx, r, alone(nyx, w, 1, 0.3 * float(w.n_h.mean())))


def test_oversize_request_and_poll_states(nyx):
    srv = nyx.Server(precision=1, hbm_budget=1 << 20)
    w = requests(1, seed=31)[0]
    with pytest.raises(nyx.NyxError) as e:
        srv.submit(w.n, w.box_cm, w.n_h, w.x_ion, w.cells, w.ndot)
    assert e.value.code == nyx.RT_ENOMEM
    srv.close()
    srv = nyx.Server(precision=1)
    with pytest.raises(nyx.NyxError):                  # precision must match the server's
        srv.submit(w.n, w.box_cm, w.n_h, w.x_ion, w.cells, w.ndot, precision=0)
    rid = srv.submit(w.n, w.box_cm, w.n_h, w.x_ion, w.cells, w.ndot)
    assert srv.poll(rid, wait_s=120.0) is not None
    srv.close()


def test_bad_request_fails_alone_and_pooled_handles_are_reused(nyx):
    # one request with x outside [0, 1] (caught by the device-side validation of
    # the batched source stage) fails by itself; the others of its batch, and the
    # later requests that reuse pooled handles of the same sizes, are unaffected
    ws = requests(10, seed=41)
    srv = nyx.Server(precision=1, max_batch=16)
    ids = []
    bad = 3
    for j, w in enumerate(ws):
        x = w.x_ion.copy()
        if j == bad:
            x.flat[5] = 1.5
        ids.append(srv.submit(w.n, w.box_cm, w.n_h, x, w.cells, w.ndot, n_th_cm3=0.3 * float(w.n_h.mean()),
                              flags=nyx.RT_FLAG_VISIT_HASH))
    for j, (w, i) in enumerate(zip(ws, ids)):
        if j == bad:
            with pytest.raises(nyx.NyxError) as e:
                srv.poll(i, wait_s=120.0)
            assert e.value.code == nyx.RT_EINVAL
        else:
            check_same(nyx, srv.poll(i, wait_s=120.0), alone(nyx, w, 1, 0.3 * float(w.n_h.mean())))
    again = requests(10, seed=43)                      # same size mix: served from the pool
    ids = [srv.submit(w.n, w.box_cm, w.n_h, w.x_ion, w.cells, w.ndot, n_th_cm3=0.3 * float(w.n_h.mean()),
                      flags=nyx.RT_FLAG_VISIT_HASH) for w in again]
    for w, i in zip(again, ids):
        check_same(nyx, srv.poll(i, wait_s=120.0), alone(nyx, w, 1, 0.3 * float(w.n_h.mean())))
    st = srv.stats()
    srv.close()
    assert st["failed"] == 1 and st["completed"] == 19


def test_pool_evicts_under_a_tight_budget(nyx):
    # a budget of about two of the largest requests with sizes alternating:
    # idle handles of the other size must be released for each admission
    ws = [I.random_small(n, 8, seed=500 + j, x_mode="patchy", box_cm=n * 2e22) for j, n in enumerate([48, 16, 48, 24, 16, 48, 24])]
    budget = (48 ** 3 * 36 + 160 * 1024 + (1 << 16)) * 2
    srv = nyx.Server(precision=1, max_batch=8, hbm_budget=budget)
    ids = [srv.submit(w.n, w.box_cm, w.n_h, w.x_ion, w.cells, w.ndot, n_th_cm3=0.3 * float(w.n_h.mean()),
                      flags=nyx.RT_FLAG_VISIT_HASH) for w in ws]
    got = [srv.poll(i, wait_s=120.0) for i in ids]
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(ws) and st["mem_peak"] <= budget
    for w, r in zip(ws, got):
        check_same(nyx, r, alone(nyx, w, 1, 0.3 * float(w.n_h.mean())))


def test_blackbody_requests_are_served(nyx):
    """Requests with Eq. 1 integrated over a blackbody spectrum are batched like gray ones (one rate
    per persistent launch): each served result equals rt_step on the request alone and the oracle's
    bookkeeping."""
    ws = requests(6, seed=61)
    srv = nyx.Server(precision=1, max_batch=8)
    kw = dict(spectrum=1, t_bb_K=1e5)
    ids = [srv.submit(w.n, w.box_cm, w.n_h, w.x_ion, w.cells, w.ndot, n_th_cm3=0.3 * float(w.n_h.mean()),
                      flags=nyx.RT_FLAG_VISIT_HASH, **kw) for w in ws]
    got = [srv.poll(i, wait_s=120.0) for i in ids]
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(ws) and st["failed"] == 0
    for w, r in zip(ws, got):
        n_th = 0.3 * float(w.n_h.mean())
        s = nyx.Solver(w.n, w.box_cm, precision=1, n_th_cm3=n_th, flags=nyx.RT_FLAG_VISIT_HASH, **kw)
        s.set_fields(w.n_h.ravel(), w.x_ion.ravel())
        s.add_sources(w.cells.ravel(), w.ndot)
        g, h, sr = s.step()
        s.close()
        check_same(nyx, r, (g.ravel(), h.ravel(), sr))
        ref = oracle.run_workload(w, n_th_cm3=n_th, precision=1, **kw)
        for k in BOOK:
            assert r[2][k] == ref["stats"][k], k
