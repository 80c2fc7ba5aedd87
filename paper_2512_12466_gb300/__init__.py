"""GB300-native adaptive ray march of Nyx-RT (arXiv 2512.12466).

Thin ctypes binding over the C ABI of ``libnyxrt.so`` (``include/nyxrt.h``):
the functions below carry the same names as the C entry points and only
marshal arguments; every step of the computation runs in the library's CUDA
kernels. ``Solver`` wraps a handle for convenience, taking torch CUDA tensors
(zero-copy device pointers on the current torch stream) or numpy arrays (host
pointers).

The library must be built first (``paper_2512_12466_gb300._build.build()`` or
``__graft_entry__.build()``); loading fails loudly if it is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnyxrt.so")

RT_MAX_LEVELS = 16
RT_OK, RT_EINVAL, RT_ENOMEM, RT_ECUDA, RT_EDEVICE, RT_ETIMEOUT, RT_ESTATE = 0, -1, -2, -3, -4, -5, -6
RT_EPENDING = -7
RT_FP64, RT_FP32 = 0, 1
RT_HOST, RT_DEVICE = 0, 1
RT_OVERLAP_NONE, RT_OVERLAP_LINEAR, RT_OVERLAP_ARC, RT_OVERLAP_CONSERVATIVE, RT_OVERLAP_SQUARED = 0, 1, 2, 3, 4
RT_OVERLAP_NAIVE = 5
RT_SPECTRUM_GRAY, RT_SPECTRUM_BLACKBODY = 0, 1
RT_MERGE_OFF, RT_MERGE_FORCED, RT_MERGE_AUTO = 0, 1, 2
RT_FLAG_VISIT_HASH = 1
RT_FLAG_NO_GEOMETRY_TABLE = 2

_ERRNAMES = {RT_EINVAL: "RT_EINVAL", RT_ENOMEM: "RT_ENOMEM", RT_ECUDA: "RT_ECUDA", RT_EDEVICE: "RT_EDEVICE",
             RT_ETIMEOUT: "RT_ETIMEOUT", RT_ESTATE: "RT_ESTATE", RT_EPENDING: "RT_EPENDING"}


class rt_config(C.Structure):
    _fields_ = [
        ("n", C.c_int32), ("precision", C.c_int32), ("box_cm", C.c_double), ("sigma_cm2", C.c_double),
        ("n_min_ray", C.c_double), ("level_max", C.c_int32), ("overlap_mode", C.c_int32),
        ("tau_max", C.c_double), ("n_th_cm3", C.c_double), ("e_heat_erg", C.c_double),
        ("merge_mode", C.c_int32), ("merge_samp_level", C.c_int32), ("automerge_xbar", C.c_double),
        ("merge_x_th", C.c_double), ("merge_f_req", C.c_double), ("merge_dr_cells", C.c_double),
        ("merge_rmax_cells", C.c_double), ("merge_f_ov", C.c_double), ("merge_eps", C.c_double),
        ("merge_n_min", C.c_int32), ("chem_iterate", C.c_int32), ("alpha_B", C.c_double), ("C_H", C.c_double),
        ("clumping", C.c_double), ("chem_tol", C.c_double), ("chem_max_iter", C.c_int32), ("flags", C.c_int32),
        ("periodic", C.c_int32), ("spectrum", C.c_int32), ("t_bb_K", C.c_double),
    ]


_L = C.c_int64 * RT_MAX_LEVELS


class rt_stats(C.Structure):
    _fields_ = [
        ("n_src_in", C.c_int64), ("n_src_dedup", C.c_int64), ("n_src_emit", C.c_int64),
        ("merged", C.c_int32), ("chem_iters", C.c_int32), ("level_max", C.c_int32), ("launches", C.c_int32),
        ("rays", _L), ("splits", _L), ("escaped", _L), ("dropped_tau", _L), ("dropped_level", _L),
        ("segments", _L), ("secondary", _L), ("visit_hash", C.c_uint64),
        ("emitted_ph", C.c_double), ("absorbed_ph", C.c_double), ("escaped_ph", C.c_double),
        ("dropped_ph", C.c_double), ("deposited_ph", C.c_double), ("chem_residual", C.c_double),
        ("ms_trace", C.c_double), ("ms_step", C.c_double), ("ms_march", C.c_double),
        ("march_launches", C.c_int64), ("table_levels", C.c_int64),
    ]


class rt_batch_params(C.Structure):
    _fields_ = [("block", C.c_int32), ("blocks_per_sm", C.c_int32), ("tile", C.c_int32), ("heavy_shift", C.c_int32),
                ("slice", C.c_int64), ("group_bytes", C.c_int64)]


class rt_server_config(C.Structure):
    _fields_ = [("precision", C.c_int32), ("max_batch", C.c_int32), ("hbm_budget", C.c_int64),
                ("slice", C.c_int64), ("group_bytes", C.c_int64), ("loaders", C.c_int32), ("max_n", C.c_int32)]


class rt_server_stats(C.Structure):
    _fields_ = [(k, C.c_int64) for k in ("submitted", "completed", "failed", "batches", "queued", "mem_budget",
                                         "mem_in_use", "mem_peak", "segments")] + \
               [(k, C.c_double) for k in ("busy_ms", "elapsed_ms", "p50_ms", "p99_ms", "mean_ms", "max_ms",
                                          "load_ms", "bind_ms", "run_ms", "finish_ms", "src_ms", "wait_admit_ms",
                                          "wait_batch_ms", "wait_finish_ms")]


class NyxError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None


def lib():
    """The loaded libnyxrt.so. Raises if the CUDA library has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build the CUDA library first "
                              "(python -c 'import __graft_entry__ as g; g.build()')")
        L = C.CDLL(LIB_PATH)
        P, i32, i64, d = C.c_void_p, C.c_int32, C.c_int64, C.c_double
        L.rt_config_default.argtypes = [C.POINTER(rt_config), i32, d]
        L.rt_config_default.restype = None
        L.rt_create.argtypes = [C.POINTER(rt_config), P, C.POINTER(P)]
        L.rt_set_fields.argtypes = [P, P, P, C.c_int]
        L.rt_add_sources.argtypes = [P, P, P, i64, C.c_int]
        L.rt_clear_sources.argtypes = [P]
        L.rt_reconfigure.argtypes = [P, C.POINTER(rt_config)]
        L.rt_spectrum_eval.argtypes = [d, d, C.POINTER(d), C.POINTER(d)]
        L.rt_spectrum_eval.restype = C.c_int
        L.rt_spectrum_absorb.argtypes = [d, d, d, C.POINTER(d)]
        L.rt_spectrum_absorb.restype = C.c_int
        L.rt_geometry_table_bytes.argtypes = [i32]
        L.rt_geometry_table_bytes.restype = i64
        L.rt_step.argtypes = [P, d, P, P, C.c_int, C.POINTER(rt_stats)]
        L.rt_get_x.argtypes = [P, P, C.c_int]
        L.rt_get_sources.argtypes = [P, P, P, i64, C.POINTER(i64), C.c_int]
        L.rt_save.argtypes = [P, C.c_char_p]
        L.rt_load.argtypes = [C.c_char_p, P, C.POINTER(P)]
        L.rt_destroy.argtypes = [P]
        L.rt_last_error.argtypes = [P]
        L.rt_last_error.restype = C.c_char_p
        L.rt_version.restype = C.c_char_p
        L.rt_batch_create.argtypes = [C.POINTER(P), i32, P, C.POINTER(P)]
        L.rt_batch_set_params.argtypes = [P, C.POINTER(rt_batch_params)]
        L.rt_batch_get_params.argtypes = [P, C.POINTER(rt_batch_params)]
        L.rt_batch_tune.argtypes = [P, i32, C.POINTER(rt_batch_params), C.POINTER(d)]
        L.rt_batch_capture.argtypes = [P]
        L.rt_batch_run.argtypes = [P, C.POINTER(P), C.POINTER(P), C.c_int, C.POINTER(rt_stats)]
        L.rt_batch_destroy.argtypes = [P]
        L.rt_batch_last_error.argtypes = [P]
        L.rt_batch_last_error.restype = C.c_char_p
        L.rt_server_config_default.argtypes = [C.POINTER(rt_server_config)]
        L.rt_server_config_default.restype = None
        L.rt_server_create.argtypes = [C.POINTER(rt_server_config), C.POINTER(P)]
        L.rt_server_submit.argtypes = [P, C.POINTER(rt_config), P, P, P, P, i64, P, P, C.POINTER(i64)]
        L.rt_server_poll.argtypes = [P, i64, d, C.POINTER(rt_stats), C.POINTER(d)]
        L.rt_server_stats_get.argtypes = [P, C.POINTER(rt_server_stats)]
        L.rt_server_destroy.argtypes = [P]
        L.rt_server_last_error.argtypes = [P]
        L.rt_server_last_error.restype = C.c_char_p
        for f in ("rt_create", "rt_set_fields", "rt_add_sources", "rt_clear_sources", "rt_reconfigure", "rt_step", "rt_get_x",
                  "rt_get_sources", "rt_save", "rt_load", "rt_destroy", "rt_batch_create", "rt_batch_set_params",
                  "rt_batch_get_params", "rt_batch_tune",
                  "rt_batch_capture", "rt_batch_run", "rt_batch_destroy", "rt_server_create", "rt_server_submit",
                  "rt_server_poll", "rt_server_stats_get", "rt_server_destroy"):
            getattr(L, f).restype = C.c_int
        _lib = L
    return _lib


def exported_symbols():
    return ["rt_config_default", "rt_create", "rt_set_fields", "rt_add_sources", "rt_clear_sources", "rt_reconfigure",
            "rt_geometry_table_bytes", "rt_spectrum_eval", "rt_spectrum_absorb", "rt_step",
            "rt_get_x", "rt_get_sources", "rt_save", "rt_load", "rt_destroy", "rt_last_error", "rt_version", "rt_batch_create", "rt_batch_set_params",
            "rt_batch_get_params", "rt_batch_tune", "rt_batch_capture", "rt_batch_run", "rt_batch_destroy",
            "rt_batch_last_error", "rt_server_config_default", "rt_server_create", "rt_server_submit",
            "rt_server_poll", "rt_server_stats_get", "rt_server_destroy", "rt_server_last_error", "rt_step_noalloc"]


def _check(rc: int, h=None):
    if rc != RT_OK:
        msg = lib().rt_last_error(h).decode(errors="replace")
        raise NyxError(rc, msg)


# ------------------------------------------------------------ C entry points (same names)

def rt_config_default(n: int, box_cm: float, **overrides) -> rt_config:
    cfg = rt_config()
    lib().rt_config_default(C.byref(cfg), int(n), float(box_cm))
    for k, v in overrides.items():
        if not hasattr(cfg, k):
            raise KeyError(k)
        setattr(cfg, k, v)
    return cfg


def rt_create(cfg: rt_config, stream: int = 0) -> int:
    h = C.c_void_p()
    _check(lib().rt_create(C.byref(cfg), C.c_void_p(stream), C.byref(h)))
    return h.value


def _ptr(a):
    """(pointer, where) of a torch tensor or numpy array, without copies."""
    if a is None:
        return None, RT_HOST
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr()), (RT_DEVICE if a.is_cuda else RT_HOST)
    return a.ctypes.data_as(C.c_void_p), RT_HOST


def rt_set_fields(h: int, n_H, x_ion, where: int) -> None:
    _check(lib().rt_set_fields(h, n_H, x_ion, where), h)


def rt_add_sources(h: int, cells, ndot, n: int, where: int) -> None:
    _check(lib().rt_add_sources(h, cells, ndot, int(n), where), h)


def rt_clear_sources(h: int) -> None:
    _check(lib().rt_clear_sources(h), h)


def rt_spectrum_eval(t_bb_K: float, tau: float):
    """(Phi(tau), Psi(tau)) of the blackbody spectrum table at t_bb_K (host evaluation)."""
    phi, psi = C.c_double(), C.c_double()
    rc = lib().rt_spectrum_eval(float(t_bb_K), float(tau), C.byref(phi), C.byref(psi))
    if rc != RT_OK:
        raise NyxError(rc, "rt_spectrum_eval: tau in [0, 1e4], t_bb_K > 0")
    return phi.value, psi.value


def rt_spectrum_absorb(t_bb_K: float, tau: float, dtau: float) -> float:
    """Phi(tau) - Phi(tau + dtau) as the FP64 march computes it (host evaluation)."""
    frac = C.c_double()
    rc = lib().rt_spectrum_absorb(float(t_bb_K), float(tau), float(dtau), C.byref(frac))
    if rc != RT_OK:
        raise NyxError(rc, "rt_spectrum_absorb: tau in [0, 1e4], dtau in (0, 1e4], t_bb_K > 0")
    return frac.value


def rt_geometry_table_bytes(device: int = 0) -> int:
    """Device memory held by the geometry tables (both precisions) of CUDA device `device`."""
    return int(lib().rt_geometry_table_bytes(int(device)))


def rt_reconfigure(h: int, cfg: rt_config) -> None:
    _check(lib().rt_reconfigure(h, C.byref(cfg)), h)


def rt_step(h: int, dt_s: float, gamma_out, heat_out, where: int, stats: rt_stats | None = None) -> rt_stats:
    st = stats if stats is not None else rt_stats()
    _check(lib().rt_step(h, float(dt_s), gamma_out, heat_out, where, C.byref(st)), h)
    return st


def rt_get_x(h: int, x_out, where: int) -> None:
    _check(lib().rt_get_x(h, x_out, where), h)


def rt_get_sources(h: int, cells_out, ndot_out, capacity: int, where: int) -> int:
    """Copies up to `capacity` entries of the last traced catalog; returns its size."""
    m = C.c_int64(0)
    _check(lib().rt_get_sources(h, cells_out, ndot_out, int(capacity), C.byref(m), where), h)
    return int(m.value)


def rt_save(h: int, path: str) -> None:
    _check(lib().rt_save(h, os.fsencode(path)), h)


def rt_load(path: str, stream: int = 0) -> int:
    h = C.c_void_p()
    _check(lib().rt_load(os.fsencode(path), C.c_void_p(stream), C.byref(h)))
    return h.value


def rt_destroy(h: int) -> None:
    _check(lib().rt_destroy(h))


def rt_version() -> str:
    return lib().rt_version().decode()


def _bcheck(rc: int, b):
    if rc != RT_OK:
        raise NyxError(rc, lib().rt_batch_last_error(b).decode(errors="replace"))


def rt_batch_create(handles, stream: int = 0) -> int:
    arr = (C.c_void_p * len(handles))(*handles)
    b = C.c_void_p()
    rc = lib().rt_batch_create(arr, len(handles), C.c_void_p(stream), C.byref(b))
    if rc != RT_OK:
        msg = lib().rt_batch_last_error(b).decode(errors="replace") if b.value else ""
        if b.value:
            lib().rt_batch_destroy(b)
        raise NyxError(rc, msg)
    return b.value


def rt_batch_set_params(b: int, p: rt_batch_params) -> None:
    _bcheck(lib().rt_batch_set_params(b, C.byref(p)), b)


def rt_batch_get_params(b: int) -> rt_batch_params:
    p = rt_batch_params()
    _bcheck(lib().rt_batch_get_params(b, C.byref(p)), b)
    return p


def rt_batch_tune(b: int, repeats: int = 2):
    p = rt_batch_params()
    ms = C.c_double()
    _bcheck(lib().rt_batch_tune(b, int(repeats), C.byref(p), C.byref(ms)), b)
    return p, ms.value


def rt_batch_capture(b: int) -> None:
    _bcheck(lib().rt_batch_capture(b), b)


def rt_batch_run(b: int, gamma_outs, heat_outs, where: int, count: int):
    g = (C.c_void_p * count)(*gamma_outs) if gamma_outs is not None else None
    h = (C.c_void_p * count)(*heat_outs) if heat_outs is not None else None
    st = (rt_stats * count)()
    _bcheck(lib().rt_batch_run(b, g, h, where, st), b)
    return [stats_dict(x) for x in st]


def rt_batch_destroy(b: int) -> None:
    lib().rt_batch_destroy(b)


def stats_dict(st: rt_stats) -> dict:
    out = {}
    for name, _ in rt_stats._fields_:
        v = getattr(st, name)
        out[name] = list(v) if hasattr(v, "__len__") else v
    return out


# ------------------------------------------------------------ convenience wrapper

class Solver:
    """One grid's ray-march state on the current CUDA device.

    Arrays may be torch CUDA tensors (float64 / int32, contiguous; used in
    place on ``stream``) or numpy arrays (host, copied by the library).
    """

    def __init__(self, n: int, box_cm: float, stream: int | None = None, **cfg):
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        self.cfg = rt_config_default(n, box_cm, **cfg)
        self.n = int(n)
        self.h = rt_create(self.cfg, stream)

    def set_fields(self, n_H, x_ion):
        for a in (n_H, x_ion):
            self._check_array(a, np.float64, self.n ** 3)
        pn, w1 = _ptr(n_H)
        px, w2 = _ptr(x_ion)
        if w1 != w2:
            raise ValueError("n_H and x_ion must both be host or both be device arrays")
        rt_set_fields(self.h, pn, px, w1)
        self._keep = (n_H, x_ion)

    def add_sources(self, cells, ndot):
        k = len(ndot)
        self._check_array(cells, np.int32, 3 * k)
        self._check_array(ndot, np.float64, k)
        pc, w1 = _ptr(cells)
        pn, w2 = _ptr(ndot)
        if w1 != w2:
            raise ValueError("cells and ndot must both be host or both be device arrays")
        rt_add_sources(self.h, pc, pn, k, w1)
        self._keep_src = (cells, ndot)

    def clear_sources(self):
        rt_clear_sources(self.h)

    def reconfigure(self, box_cm: float, **cfg):
        """Re-target to another configuration of the same n / precision /
        chemistry setting, keeping the device allocations; sources are
        cleared and fields must be set again."""
        cfg.setdefault("precision", self.cfg.precision)
        cfg.setdefault("chem_iterate", self.cfg.chem_iterate)
        c = rt_config_default(self.n, box_cm, **cfg)
        rt_reconfigure(self.h, c)
        self.cfg = c
        self._keep = self._keep_src = None

    def step(self, dt_s: float = 0.0, gamma=None, heat=None):
        """Run one step; returns (gamma, heat, stats). Output arrays are
        allocated (numpy) if not given."""
        if gamma is None and heat is None:
            gamma = np.empty((self.n,) * 3)
            heat = np.empty((self.n,) * 3)
        pg, w1 = _ptr(gamma)
        ph, w2 = _ptr(heat)
        where = w1 if gamma is not None else w2
        st = rt_step(self.h, dt_s, pg, ph, where)
        return gamma, heat, stats_dict(st)

    def get_x(self, out=None):
        if out is None:
            out = np.empty((self.n,) * 3)
        p, w = _ptr(out)
        rt_get_x(self.h, p, w)
        return out

    def save(self, path: str) -> None:
        """Checkpoint this solver (configuration, fields, sources) to `path`."""
        rt_save(self.h, path)

    @classmethod
    def load(cls, path: str, stream: int | None = None) -> "Solver":
        """A solver restored from a checkpoint written by save(), ready to step."""
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        s = cls.__new__(cls)
        s.h = rt_load(path, stream)
        with open(path, "rb") as f:                # the configuration follows the magic and two uint32
            f.seek(16)
            s.cfg = rt_config.from_buffer_copy(f.read(C.sizeof(rt_config)))
        s.n = int(s.cfg.n)
        return s

    def sources(self):
        """The catalog the last step traced (after dedup, sort and Alg. 3
        merging) as numpy arrays: cells (m, 3) int32 (ix, iy, iz), ndot (m,)."""
        m = rt_get_sources(self.h, None, None, 0, RT_HOST)
        cells = np.empty((m, 3), dtype=np.int32)
        ndot = np.empty(m)
        if m:
            rt_get_sources(self.h, cells.ctypes.data, ndot.ctypes.data, m, RT_HOST)
        return cells, ndot

    def close(self):
        if self.h:
            rt_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _check_array(a, dtype, size):  # noqa: D401
        if hasattr(a, "data_ptr"):
            import torch
            want = {np.float64: torch.float64, np.int32: torch.int32}[dtype]
            if a.dtype != want or not a.is_contiguous() or a.numel() != size:
                raise ValueError(f"expected a contiguous {want} tensor of {size} elements")
        else:
            if a.dtype != dtype or not a.flags["C_CONTIGUOUS"] or a.size != size:
                raise ValueError(f"expected a C-contiguous {np.dtype(dtype)} array of {size} elements")


class Batch:
    """Many solvers traced together (rt_batch_*): light solves in persistent launches, heavy ones
    in device-sized per-level launches on parallel streams."""

    def __init__(self, solvers):
        self.solvers = list(solvers)
        self.b = rt_batch_create([s.h for s in self.solvers])

    def params(self) -> rt_batch_params:
        return rt_batch_get_params(self.b)

    def set_params(self, block=None, blocks_per_sm=None, tile=None, slice=None, group_bytes=None,
                   heavy_shift=None):
        p = rt_batch_get_params(self.b)
        for k, v in dict(block=block, blocks_per_sm=blocks_per_sm, tile=tile, slice=slice,
                         group_bytes=group_bytes, heavy_shift=heavy_shift).items():
            if v is not None:
                setattr(p, k, v)
        rt_batch_set_params(self.b, p)

    def tune(self, repeats: int = 2):
        return rt_batch_tune(self.b, repeats)

    def capture(self):
        rt_batch_capture(self.b)

    def run(self, gammas=None, heats=None):
        """Run once. gammas / heats: lists of per-solve output tensors or arrays
        (all device or all host), or None. Returns per-solve stats dicts."""
        where = RT_HOST
        gp = hp = None
        if gammas is not None:
            ptrs = [_ptr(g) for g in gammas]
            gp = [p for p, _ in ptrs]
            where = ptrs[0][1]
        if heats is not None:
            ptrs = [_ptr(h) for h in heats]
            hp = [p for p, _ in ptrs]
            where = ptrs[0][1]
        return rt_batch_run(self.b, gp, hp, where, len(self.solvers))

    def close(self):
        if self.b:
            rt_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching request loop (rt_server_*). Inputs are host numpy
    arrays kept alive here until their request is polled."""

    def __init__(self, precision: int = RT_FP32, max_batch: int = 64, hbm_budget: int = 0,
                 slice: int | None = None, group_bytes: int | None = None, loaders: int | None = None):
        c = rt_server_config()
        lib().rt_server_config_default(C.byref(c))
        c.precision = precision
        c.max_batch = max_batch
        c.hbm_budget = hbm_budget
        if slice is not None:
            c.slice = slice
        if group_bytes is not None:
            c.group_bytes = group_bytes
        if loaders is not None:
            c.loaders = loaders
        h = C.c_void_p()
        rc = lib().rt_server_create(C.byref(c), C.byref(h))
        if rc != RT_OK:
            raise NyxError(rc, "server creation failed")
        self.s = h.value
        self.precision = precision
        self._live = {}

    def submit(self, n: int, box_cm: float, n_h, x_ion, cells, ndot, gamma=None, heat=None, **cfg) -> int:
        cfg.setdefault("precision", self.precision)
        c = rt_config_default(n, box_cm, **cfg)
        arrs = [np.ascontiguousarray(n_h, dtype=np.float64), np.ascontiguousarray(x_ion, dtype=np.float64),
                np.ascontiguousarray(cells, dtype=np.int32), np.ascontiguousarray(ndot, dtype=np.float64)]
        if gamma is None and heat is None:      # neither given: both returned, in new host arrays
            gamma = np.empty(n ** 3)
            heat = np.empty(n ** 3)
        for a in (gamma, heat):                 # one given: only that one is produced
            if a is not None and (a.dtype != np.float64 or a.size != n ** 3 or not a.flags.c_contiguous):
                raise ValueError("result buffers must be contiguous float64 host arrays of n^3 elements")
        out = [a.ctypes.data_as(C.c_void_p) if a is not None else None for a in (gamma, heat)]
        rid = C.c_int64()
        rc = lib().rt_server_submit(self.s, C.byref(c), *[a.ctypes.data_as(C.c_void_p) for a in arrs], len(arrs[3]),
                                    out[0], out[1], C.byref(rid))
        if rc != RT_OK:
            raise NyxError(rc, lib().rt_server_last_error(self.s).decode(errors="replace"))
        self._live[rid.value] = (arrs, gamma, heat)
        return rid.value

    def poll(self, rid: int, wait_s: float = 0.0):
        """None if the request is still running, else (gamma, heat, stats, latency_ms)."""
        st = rt_stats()
        lat = C.c_double()
        rc = lib().rt_server_poll(self.s, rid, float(wait_s), C.byref(st), C.byref(lat))
        if rc == RT_EPENDING:
            return None
        _, gamma, heat = self._live.pop(rid)
        if rc != RT_OK:
            raise NyxError(rc, lib().rt_server_last_error(self.s).decode(errors="replace"))
        return gamma, heat, stats_dict(st), lat.value

    def stats(self) -> dict:
        st = rt_server_stats()
        lib().rt_server_stats_get(self.s, C.byref(st))
        return {k: getattr(st, k) for k, _ in rt_server_stats._fields_}

    def close(self):
        if self.s:
            lib().rt_server_destroy(self.s)
            self.s = None
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
