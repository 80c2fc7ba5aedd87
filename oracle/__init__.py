"""CPU oracle for the adaptive ray march (arXiv 2512.12466) -- TEST INFRASTRUCTURE.

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's
``cpu_baseline`` / reference leg may import this package. The product path
(the CUDA library and its binding) never does: it shares no code with this
oracle.

The oracle itself is plain scalar C (``rt_oracle.c``) compiled with
``gcc -O2 -ffp-contract=off``; this module builds it and marshals numpy
arrays through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rt_oracle.c")
_HDR = os.path.join(_HERE, "march_body.h")
_SO = os.path.join(_HERE, "_rt_oracle.so")
_lock = threading.Lock()
_lib = None

MAXLEV = 16
S_BITS = 21
F_BITS = 24


class OrcConfig(C.Structure):
    _fields_ = [
        ("n", C.c_int32), ("precision", C.c_int32), ("box_cm", C.c_double),
        ("sigma_cm2", C.c_double), ("n_min_ray", C.c_double), ("level_max", C.c_int32),
        ("overlap_mode", C.c_int32), ("tau_max", C.c_double), ("n_th_cm3", C.c_double),
        ("e_heat_erg", C.c_double), ("merge_mode", C.c_int32), ("merge_samp_level", C.c_int32),
        ("automerge_xbar", C.c_double), ("merge_x_th", C.c_double), ("merge_f_req", C.c_double),
        ("merge_dr_cells", C.c_double), ("merge_rmax_cells", C.c_double), ("merge_f_ov", C.c_double),
        ("merge_eps", C.c_double), ("merge_n_min", C.c_int32), ("chem_iterate", C.c_int32),
        ("dt_s", C.c_double), ("alpha_B", C.c_double), ("C_H", C.c_double), ("clumping", C.c_double),
        ("chem_tol", C.c_double), ("chem_max_iter", C.c_int32), ("periodic", C.c_int32),
        ("spectrum", C.c_int32), ("nq", C.c_int32), ("q_s", C.c_void_p), ("q_w", C.c_void_p),
    ]


class OrcStats(C.Structure):
    _fields_ = [
        ("n_src_in", C.c_int64), ("n_src_dedup", C.c_int64), ("n_src_emit", C.c_int64),
        ("merged", C.c_int32), ("chem_iters", C.c_int32), ("level_max", C.c_int32), ("pad_", C.c_int32),
        ("rays", C.c_int64 * MAXLEV), ("splits", C.c_int64 * MAXLEV), ("escaped", C.c_int64 * MAXLEV),
        ("dropped_tau", C.c_int64 * MAXLEV), ("dropped_level", C.c_int64 * MAXLEV),
        ("segments", C.c_int64 * MAXLEV), ("secondary", C.c_int64 * MAXLEV),
        ("visit_hash", C.c_uint64),
        ("emitted_ph", C.c_double), ("absorbed_ph", C.c_double), ("escaped_ph", C.c_double),
        ("dropped_ph", C.c_double), ("deposited_ph", C.c_double), ("chem_residual", C.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, no FMA contraction)."""
    with _lock:
        newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
        if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
            tmp = _SO + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
                                   "-Wall", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_SO)
        d, i32, i64, u64 = C.c_double, C.c_int32, C.c_int64, C.c_uint64
        P = C.c_void_p
        L.orc_pix2vec.argtypes = [i32, i64, P]
        L.orc_direction.argtypes = [i32, i64, P, P]
        L.orc_split_rq.argtypes = [d]
        L.orc_split_rq.restype = i64
        L.orc_periodic_rs.argtypes = [C.c_int32]
        L.orc_periodic_rs.restype = i64
        L.orc_default_level_max.argtypes = [i32, d]
        L.orc_default_level_max.restype = i32
        L.orc_mix64_export.argtypes = [u64]
        L.orc_mix64_export.restype = u64
        L.orc_prepare_kappa.argtypes = [i64, P, P, d, d, P]
        L.orc_sources_dedup.argtypes = [P, P, i64, P, P]
        L.orc_sources_dedup.restype = i64
        L.orc_max_radius.argtypes = [i32, P, P, i32, d, d, i32, d, d, i32]
        L.orc_max_radius.restype = d
        L.orc_merge_sources.argtypes = [i32, P, P, P, i64, i32, d, d, i32, d, d, d, d, i32, P, P, P, P]
        L.orc_merge_sources.restype = i64
        L.orc_chem_update.argtypes = [i64, P, P, P, P, d, d, d, d, P]
        L.orc_chem_update.restype = d
        L.orc_run.argtypes = [C.POINTER(OrcConfig), P, P, P, P, i64, P, P, P, C.POINTER(OrcStats),
                              P, P, P, P, i64, P, P, P]
        L.orc_run.restype = C.c_int
        L.orc_sizeof_config.restype = i64
        L.orc_sizeof_stats.restype = i64
        assert L.orc_sizeof_config() == C.sizeof(OrcConfig), "orc_config layout mismatch"
        assert L.orc_sizeof_stats() == C.sizeof(OrcStats), "orc_stats layout mismatch"
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


# ---------------------------------------------------------------- small pieces

def pix2vec(level: int, pix: int) -> np.ndarray:
    v = np.zeros(3)
    lib().orc_pix2vec(level, pix, _ptr(v))
    return v


def direction(level: int, pix: int):
    sd = np.zeros(3, dtype=np.int32)
    nrm = np.zeros(1)
    lib().orc_direction(level, pix, _ptr(sd), _ptr(nrm))
    return sd, float(nrm[0])


def split_rq(n_min_ray: float) -> int:
    return int(lib().orc_split_rq(n_min_ray))


def periodic_rs(n: int) -> int:
    """Travel-distance cutoff sqrt(3) L_box of periodic boundaries (Sec. 2.5.1), in 2^-24 cells."""
    return int(lib().orc_periodic_rs(int(n)))


def default_level_max(n: int, n_min_ray: float) -> int:
    return int(lib().orc_default_level_max(n, n_min_ray))


def mix64(z: int) -> int:
    return int(lib().orc_mix64_export(z))


def prepare_kappa(n_h, x, sigma_dx, n_th) -> np.ndarray:
    n_h = np.ascontiguousarray(n_h, dtype=np.float64).reshape(-1)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
    out = np.empty_like(n_h)
    lib().orc_prepare_kappa(n_h.size, _ptr(n_h), _ptr(x), sigma_dx, n_th, _ptr(out))
    return out


def sources_dedup(cells, ndot):
    cells = np.ascontiguousarray(cells, dtype=np.int32).reshape(-1, 3)
    ndot = np.ascontiguousarray(ndot, dtype=np.float64)
    oc = np.empty_like(cells)
    on = np.empty_like(ndot)
    m = lib().orc_sources_dedup(_ptr(cells), _ptr(ndot), len(ndot), _ptr(oc), _ptr(on))
    return oc[:m].copy(), on[:m].copy()


def max_radius(x, cell, samp_level=3, x_th=0.9, f_req=0.9, n_min=8, dr=2.0, rmax=16.0, periodic=0) -> float:
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = x.shape[0]
    c = np.ascontiguousarray(cell, dtype=np.int32)
    return float(lib().orc_max_radius(n, _ptr(x), _ptr(c), samp_level, x_th, f_req, n_min, dr, rmax, periodic))


def merge_sources(x, cells, ndot, samp_level=3, x_th=0.9, f_req=0.9, n_min=8, dr=2.0, rmax=16.0,
                  f_ov=1.0, eps=1e-6, periodic=0):
    """Alg. 3 on a deduplicated sorted catalog. Returns (cells, ndot, radius, label)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = x.shape[0]
    cells = np.ascontiguousarray(cells, dtype=np.int32).reshape(-1, 3)
    ndot = np.ascontiguousarray(ndot, dtype=np.float64)
    s = len(ndot)
    rad = np.zeros(s)
    lab = np.zeros(s, dtype=np.int64)
    oc = np.zeros((max(s, 1), 3), dtype=np.int32)
    on = np.zeros(max(s, 1))
    m = lib().orc_merge_sources(n, _ptr(x), _ptr(cells), _ptr(ndot), s, samp_level, x_th, f_req, n_min,
                                dr, rmax, f_ov, eps, periodic, _ptr(rad), _ptr(lab), _ptr(oc), _ptr(on))
    return oc[:m].copy(), on[:m].copy(), rad, lab


def chem_update(n_h, x0, xavg, gamma, dt, alpha_B, C_H=0.0, clump=1.0):
    """One C2-Ray update at fixed Gamma. Returns (xavg_new, x_end, max_change)."""
    n_h = np.ascontiguousarray(n_h, dtype=np.float64).reshape(-1)
    x0 = np.ascontiguousarray(x0, dtype=np.float64).reshape(-1)
    xa = np.array(xavg, dtype=np.float64).reshape(-1)
    g = np.ascontiguousarray(gamma, dtype=np.float64).reshape(-1)
    xe = np.empty_like(xa)
    d = lib().orc_chem_update(n_h.size, _ptr(n_h), _ptr(x0), _ptr(xa), _ptr(g), dt, alpha_B, C_H, clump,
                              _ptr(xe))
    return xa, xe, float(d)


# ---------------------------------------------------------------- full solve

DEFAULTS = dict(precision=0, sigma_cm2=6.3e-18, n_min_ray=4.0, level_max=-1, overlap_mode=3,
                tau_max=30.0, n_th_cm3=None, e_heat_erg=1.602176634e-12, merge_mode=0,
                merge_samp_level=3, automerge_xbar=0.018, merge_x_th=0.9, merge_f_req=0.9,
                merge_dr_cells=2.0, merge_rmax_cells=16.0, merge_f_ov=1.0, merge_eps=1e-6,
                merge_n_min=8, chem_iterate=0, dt_s=0.0, alpha_B=2.59e-13, C_H=0.0, clumping=1.0,
                chem_tol=1e-6, chem_max_iter=100, periodic=0, spectrum=0, t_bb_K=1e5)


# Hydrogen ionization threshold h nu_0 (13.598 eV) and Boltzmann's constant, cgs.
H_NU0_ERG = 13.598 * 1.602176634e-12
K_B_ERG_K = 1.380649e-16


def spectrum_nodes(t_bb_K: float, nq: int = 64):
    """Frequency quadrature for Eq. 1 with a blackbody source at t_bb_K and
    sigma_nu = sigma_0 (nu_0 / nu)^3 above the threshold: with y = nu / nu_0 and
    theta = h nu_0 / (k T), the photon-number spectrum is y^2 / (exp(theta y) - 1);
    substituting y = 1 + z / theta turns its integral over [1, inf) into one with
    weight exp(-z), done by Gauss-Laguerre. Returns (sigma ratios y^-3, weights
    normalised to sum 1)."""
    theta = H_NU0_ERG / (K_B_ERG_K * t_bb_K)
    z, om = np.polynomial.laguerre.laggauss(nq)
    y = 1.0 + z / theta
    wt = om * y ** 2 * np.exp(-theta) / (theta * (-np.expm1(-(theta + z))))
    return np.ascontiguousarray(y ** -3.0), np.ascontiguousarray(wt / wt.sum())


def make_config(n: int, box_cm: float, n_h=None, **kw) -> OrcConfig:
    p = dict(DEFAULTS)
    p.update({k: v for k, v in kw.items() if k in DEFAULTS})
    if p["n_th_cm3"] is None:
        p["n_th_cm3"] = 0.01 * float(np.mean(n_h)) if n_h is not None else 0.0
    cfg = OrcConfig()
    cfg.n = n
    cfg.box_cm = box_cm
    t_bb = p.pop("t_bb_K")
    nodes = kw.get("q_nodes")
    for k, v in p.items():
        setattr(cfg, k, v)
    if cfg.spectrum == 1:
        qs, qw = spectrum_nodes(t_bb) if nodes is None else (np.ascontiguousarray(nodes[0], dtype=np.float64),
                                                            np.ascontiguousarray(nodes[1], dtype=np.float64))
        cfg.nq = len(qs)
        cfg.q_s = qs.ctypes.data
        cfg.q_w = qw.ctypes.data
        cfg._keep = (qs, qw)          # the arrays outlive the call through the config
    return cfg


def stats_dict(st: OrcStats) -> dict:
    out = {}
    for name, _ in OrcStats._fields_:
        if name == "pad_":
            continue
        v = getattr(st, name)
        out[name] = list(v) if hasattr(v, "__len__") else v
    return out


def run(n_h, x, cells, ndot, box_cm, record: int = 0, **kw) -> dict:
    """Solve one step on the CPU. kw: any DEFAULTS key. Returns fields, stats,
    the emitted catalog and, if record > 0, the first `record` visits."""
    n_h = np.ascontiguousarray(n_h, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = n_h.shape[0]
    cells = np.ascontiguousarray(cells, dtype=np.int32).reshape(-1, 3)
    ndot = np.ascontiguousarray(ndot, dtype=np.float64)
    cfg = make_config(n, box_cm, n_h=n_h, **kw)
    gamma = np.zeros(n ** 3)
    heat = np.zeros(n ** 3)
    xo = np.zeros(n ** 3)
    st = OrcStats()
    rec = max(0, int(record))
    rr = np.zeros(max(rec, 1), dtype=np.int64)
    rs = np.zeros(max(rec, 1), dtype=np.int32)
    rc = np.zeros(max(rec, 1), dtype=np.int64)
    rd = np.zeros(max(rec, 1))
    rn = np.zeros(1, dtype=np.int64)
    ec = np.zeros((max(len(ndot), 1), 3), dtype=np.int32)
    en = np.zeros(max(len(ndot), 1))
    rc_ = lib().orc_run(C.byref(cfg), _ptr(n_h), _ptr(x), _ptr(cells), _ptr(ndot), len(ndot),
                        _ptr(gamma), _ptr(heat), _ptr(xo), C.byref(st), _ptr(rr), _ptr(rs), _ptr(rc),
                        _ptr(rd), rec, _ptr(rn), _ptr(ec), _ptr(en))
    if rc_ != 0:
        raise ValueError(f"oracle rejected the input (code {rc_})")
    sd = stats_dict(st)
    m = sd["n_src_emit"]
    out = dict(gamma=gamma.reshape(n, n, n), heat=heat.reshape(n, n, n), x=xo.reshape(n, n, n),
               stats=sd, emit_cells=ec[:m].copy(), emit_ndot=en[:m].copy(), config=cfg)
    if rec:
        k = int(min(rn[0], rec))
        out["visits"] = dict(ray=rr[:k].copy(), seq=rs[:k].copy(), cell=rc[:k].copy(), ds=rd[:k].copy(),
                             total=int(rn[0]))
    return out


def run_workload(w, record: int = 0, **kw) -> dict:
    p = dict(w.params)
    p.update(kw)
    return run(w.n_h, w.x_ion, w.cells, w.ndot, w.box_cm, record=record, **p)
