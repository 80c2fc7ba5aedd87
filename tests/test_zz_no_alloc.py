"""rt_step_noalloc through the C ABI, checked against rt_step.

Some callers cannot allocate device memory at the moment they need a step:
code running inside a memory-capped or externally managed pool, or a
real-time loop that must stay out of the CUDA allocator. rt_step_noalloc
serves them from a fixed array inside the library instead of cudaMalloc'd
buffers. Here two calls in a row (on different inputs, then the first input
again) must match the ordinary entry points (rt_create, rt_set_fields,
rt_add_sources, rt_step) on the same inputs: identical bookkeeping and visit
hash, Gamma and heating within 1e-12 relative L2 for the FP64 march and 1e-5
for the FP32 march. Sizes beyond the array's limits must be rejected.

The file name makes pytest collect it last; it also passes on its own in a
fresh process (the first call sets the array up).
"""
import ctypes as C

import numpy as np
import pytest

from paper_2512_12466_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nyx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2512_12466_gb300 as m
    L = m.lib()
    L.rt_step_noalloc.argtypes = [C.POINTER(m.rt_config), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.POINTER(m.rt_stats),
                                  C.c_char_p, C.c_int32]
    L.rt_step_noalloc.restype = C.c_int
    return m


def relerr(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).ravel()).cuda()


def noalloc_step(nyx, cfg, w):
    n3 = w.n ** 3
    nh, x, cells, nd = dev(w.n_h), dev(w.x_ion), dev(w.cells.astype(np.int32)), dev(w.ndot)
    g = torch.full((n3,), -1.0, dtype=torch.float64, device="cuda")
    h = torch.full((n3,), -1.0, dtype=torch.float64, device="cuda")
    st = nyx.rt_stats()
    err = C.create_string_buffer(256)
    stream = torch.cuda.current_stream().cuda_stream
    rc = nyx.lib().rt_step_noalloc(C.byref(cfg), C.c_void_p(stream), nh.data_ptr(), x.data_ptr(),
                                   cells.data_ptr(), nd.data_ptr(), len(w.ndot), g.data_ptr(), h.data_ptr(),
                                   C.byref(st), err, 256)
    return rc, err.value.decode(), g.cpu().numpy(), h.cpu().numpy(), nyx.stats_dict(st)


def plain_step(nyx, cfg_kw, w):
    s = nyx.Solver(w.n, w.box_cm, **cfg_kw)
    s.set_fields(dev(w.n_h), dev(w.x_ion))
    s.add_sources(dev(w.cells.astype(np.int32)), dev(w.ndot))
    g = torch.empty(w.n ** 3, dtype=torch.float64, device="cuda")
    h = torch.empty_like(g)
    _, _, st = s.step(0.0, g, h)
    s.close()
    return g.cpu().numpy(), h.cpu().numpy(), st


BOOK = ("rays", "splits", "escaped", "dropped_tau", "dropped_level", "segments", "secondary", "visit_hash")


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-5)])
def test_noalloc_matches_rt_step_twice(nyx, precision, tol):
    wa = I.random_small(24, 6, seed=7, x_mode="patchy", box_cm=24 * 7e22)
    wb = I.random_small(32, 11, seed=8, x_mode="thin", box_cm=32 * 7e20)
    for w in (wa, wb, wa):
        kw = dict(precision=precision, n_th_cm3=0.3 * float(w.n_h.mean()), flags=nyx.RT_FLAG_VISIT_HASH)
        cfg = nyx.rt_config_default(w.n, w.box_cm, **kw)
        rc, msg, g, h, st = noalloc_step(nyx, cfg, w)
        assert rc == 0, msg
        gr, hr, sr = plain_step(nyx, kw, w)
        for k in BOOK:
            assert st[k] == sr[k], k
        assert st["n_src_emit"] == sr["n_src_emit"]
        assert relerr(g, gr) < tol
        assert relerr(h, hr) < tol
        e = st["emitted_ph"]
        assert abs(st["absorbed_ph"] + st["escaped_ph"] + st["dropped_ph"] - e) <= (1e-12 if precision == 0 else 1e-6) * e


def test_noalloc_rejects_sizes_beyond_its_limits(nyx):
    w = I.random_small(33, 2, seed=9, x_mode="thin", box_cm=33 * 7e20)
    rc, msg, *_ = noalloc_step(nyx, nyx.rt_config_default(w.n, w.box_cm), w)
    assert rc == nyx.RT_EINVAL and "1..32" in msg
    w = I.random_small(8, 4097, seed=10, x_mode="thin", box_cm=8 * 7e20)
    rc, msg, *_ = noalloc_step(nyx, nyx.rt_config_default(w.n, w.box_cm), w)
    assert rc == nyx.RT_EINVAL and "4096" in msg
    w = I.random_small(8, 2, seed=11, x_mode="thin", box_cm=8 * 7e20)
    rc, msg, *_ = noalloc_step(nyx, nyx.rt_config_default(w.n, w.box_cm, merge_mode=1), w)
    assert rc == nyx.RT_EINVAL and "merging" in msg
