#!/usr/bin/env python
"""Benchmark: ray-cell segments per second of the adaptive ray march.

A step is one full radiative-transfer step through the C ABI (rt_step):
source dedup/sort, optical-depth field, the level-by-level fused march +
split over every ray of every source, heating and ledger. Workload: the
128^3 lognormal box (20 Mpc/h, sigma_ln = 1, mean n_H = 2e-4) with 1024
power-law sources in the densest 1% of cells, in its optically thin variant
(uniform residual x_HI = 1e-4, so rays cross the box). The headline march is
FP32 with Kahan-compensated budgets (FP64 deposits); the FP64 march is
measured beside it.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl nyx|reference]
Under torchrun (N > 1) each rank runs its own replica of the workload
(independent solves, no collective on the data path); the value is the
segments of all ranks over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2512_12466_gb300 import inputs as I  # noqa: E402

METRIC = "ray-cell segments/s"
WORKLOAD = "128^3 lognormal box, 1024 power-law sources, thin (x_HI=1e-4)"
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM = 6800.0
NOMINAL_HBM = 7900.0          # GB300 HBM3e nominal, for the second fraction beside the measured one
L2_FLUSH_BYTES = 512 << 20


# DRAM traffic of the march from one ncu capture per precision (dram__bytes_read.sum +
# dram__bytes_write.sum over every march launch of one step of the same box with its first 64
# sources, taken with `python -m paper_2512_12466_gb300.profile_case --sources 64 --steps 1 --levels
# [--precision fp64]`), scaled to the full workload by primary segments. Valid only for the kernel
# sources it was taken on.
TRAFFIC_CAPTURE = {"kernel": "march_table_kernel",
                   "bytes_per_segment": {"fp32": 8.80868621095342, "fp64": 19.254816976037528},
                   "sources": {"paper_2512_12466_gb300/csrc/march.cu": "e97eefbf436b7d8a",
                               "paper_2512_12466_gb300/csrc/rt_internal.h": "7b899d1021ce1758",
                               "paper_2512_12466_gb300/csrc/dfloat.h": "459135c9d92ee117"}}


def traffic_per_launch(segments_per_step: float, launches_per_step: float, precision: str = "fp32"):
    """Scaled DRAM bytes of the average march launch, or None once the kernel changed since the capture."""
    import hashlib
    for rel, h in TRAFFIC_CAPTURE["sources"].items():
        try:
            if hashlib.sha256(open(os.path.join(ROOT, rel), "rb").read()).hexdigest()[:16] != h:
                return None
        except OSError:
            return None
    return TRAFFIC_CAPTURE["bytes_per_segment"][precision] * segments_per_step / max(1.0, launches_per_step)


def atomic_peak():
    """FP64 atomic adds per second into an L2-resident array the size of the 128^3 Gamma grid (random
    cells and neighbouring cells per warp), measured now with the committed probe library: the
    deposit roofline of the march."""
    import ctypes as C
    from paper_2512_12466_gb300 import _build
    lib = C.CDLL(_build.build_probe())
    lib.nyxrt_probe_red_f64.argtypes = [C.c_int64, C.c_int64, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]
    lib.nyxrt_probe_red_f64.restype = C.c_int
    out = {}
    for name, pat in (("random", 0), ("neighbours", 1)):
        best = 0.0
        for _ in range(3):
            ps, ms = C.c_double(), C.c_double()
            if lib.nyxrt_probe_red_f64(128 ** 3, 256, pat, C.byref(ps), C.byref(ms)) == 0:
                best = max(best, ps.value)
        out[name] = best
    return out


def load_peaks():
    try:
        p = json.load(open(PEAKS))
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM, "fallback"


def workload():
    w = I.config2("thin")
    return w, 0.01 * float(w.n_h.mean())


def algorithmic_bytes(st: dict, precision: int) -> float:
    """Algorithmic bytes of the march kernels of one trace: per primary segment
    and per secondary deposit one kappa read (8 B FP64 / 4 B FP32) and one FP64
    read-modify-write of Gamma (16 B); per ray its 16-B direction entry and a
    quarter of its parent record; per split one parent record written."""
    rec = 24  # src 4 + pix 4 + P + tau (8+8) or P, tau, cP, ctau (4 x 4)
    seg_b = (8 if precision == 0 else 4) + 16
    segs = sum(st["segments"])
    sec = sum(st["secondary"])
    rays = sum(st["rays"])
    splits = sum(st["splits"])
    return seg_b * (segs + sec) + 16 * rays + rec / 4.0 * rays + rec * splits


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = [r.split(", ") for r in open(self.path).read().strip().splitlines() if r.strip()]
        os.unlink(self.path)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower().startswith("active"):
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(value: float, world: int) -> float:
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, world: int) -> float:
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# The oracle over many host cores: Gamma is additive over sources at fixed x, so the sources of a
# sample are traced one per task by a pool of processes (spawned, each with its own copy of the
# workload), the oracle itself unchanged; the rate is all their segments over the wall time.
_POOL_WORKLOAD = None


def _pool_init():
    global _POOL_WORKLOAD
    _POOL_WORKLOAD = workload()


def _pool_source(i: int) -> int:
    import oracle
    w, n_th = _POOL_WORKLOAD
    i = i % len(w.ndot)
    r = oracle.run(w.n_h, w.x_ion, w.cells[i:i + 1], w.ndot[i:i + 1], w.box_cm, n_th_cm3=n_th, precision=0,
                   n_min_ray=4.0, tau_max=30.0)
    return sum(r["stats"]["segments"])


def oracle_pool(cores: int):
    import multiprocessing as mp
    pool = mp.get_context("spawn").Pool(cores, initializer=_pool_init)
    pool.map(_pool_source, range(cores), chunksize=1)          # every worker up, oracle loaded
    return pool


def pooled_rate(pool, first: int, count: int):
    t0 = time.perf_counter()
    segs = sum(pool.map(_pool_source, range(first, first + count), chunksize=1))
    return segs, time.perf_counter() - t0


def cpu_baseline(budget_s: float = 12.0):
    """The CPU oracle as it stands on a bounded sample of the same workload, first single-threaded
    (sources taken in order until ~budget_s / 2 of work), then on every host core (a pool of
    os.cpu_count() processes, one source per task, ~budget_s of wall time)."""
    import oracle
    w, n_th = workload()
    segs, t_total, used = 0, 0.0, 0
    while t_total < budget_s / 2 and used < len(w.ndot):
        t0 = time.perf_counter()
        r = oracle.run(w.n_h, w.x_ion, w.cells[used:used + 1], w.ndot[used:used + 1], w.box_cm, n_th_cm3=n_th,
                       precision=0, n_min_ray=4.0, tau_max=30.0)
        t_total += time.perf_counter() - t0
        segs += sum(r["stats"]["segments"])
        used += 1
    single = {"value": segs / t_total, "cores": 1,
              "sample": f"{used} of 1024 sources, {segs} segments in {t_total:.1f} s"}
    cores = os.cpu_count() or 1
    per_source = t_total / max(used, 1)
    count = max(2 * cores, int(budget_s * cores / max(per_source, 1e-3)))
    with oracle_pool(cores) as pool:
        psegs, wall = pooled_rate(pool, used, count)
    return {"value": psegs / wall, "unit": "segments/s", "cores": cores, "kind": "oracle",
            "sample": f"{count} of the 1024 sources of the same 128^3 thin workload (from source {used}, "
                      f"wrapping), one per task over {cores} processes, FP64 oracle, {psegs} segments in "
                      f"{wall:.1f} s of wall time",
            "single_thread": single}


def run_reference(args, world, rank):
    """Reference arm: the CPU oracle on the same workload, each step a bounded sample (the next
    2 sources per host core), traced by a pool of os.cpu_count() processes on the host cores."""
    if rank != 0:
        return 0
    cores = os.cpu_count() or 1
    k = 2 * cores
    times, segs = [], 0
    with oracle_pool(cores) as pool:
        for i in range(args.warmup + args.steps):
            s_i, dt = pooled_rate(pool, i * k, k)
            if i >= args.warmup:
                times.append(dt)
                segs += s_i
    total = sum(times)
    value = segs / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "segments/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": 128, "sources": 1024, "step_sample": f"{k} sources per step"},
            "cpu_baseline": {"value": value, "unit": "segments/s", "cores": cores, "kind": "oracle",
                             "sample": f"{k} sources of the 1024 per step, one per task over {cores} processes, "
                                       f"FP64 oracle"},
            "e2e": {"value": value, "unit": "segments/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def time_steps(solver, steps, flush, g, h, torch):
    """Per-step CUDA-event timing on the solver's stream, L2 flushed before each step."""
    stream = torch.cuda.current_stream()
    ms, stats = [], []
    for _ in range(steps):
        flush.add_(1)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, _, st = solver.step(0.0, g, h)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
        stats.append(st)
    return ms, stats


def bench_overlap_modes(nyx, torch, w, n_th):
    """Beam-overlap treatments (Sec. 2.6) on the same box, FP32, one step each: photons deposited
    over photons absorbed (1 for the photon-conserving modes), secondary deposits, march time."""
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).ravel()).cuda()
    names = {0: "none", 1: "Eq. 5 only", 2: "Eqs. 5-6 (Arc, unthresholded)", 3: "Eqs. 7-8 (conservative threshold)",
             4: "squared f_c (Wise)", 5: "naive threshold"}
    nh, xx, cc, nd = dev(w.n_h), dev(w.x_ion), dev(w.cells), dev(w.ndot)
    g = torch.empty(w.n ** 3, dtype=torch.float64, device="cuda")
    out = {}
    for mode, name in names.items():
        s = nyx.Solver(w.n, w.box_cm, precision=nyx.RT_FP32, n_th_cm3=n_th, n_min_ray=4.0, tau_max=30.0,
                       overlap_mode=mode)
        s.set_fields(nh, xx)
        s.add_sources(cc, nd)
        _, _, st = s.step(0.0, g, None)
        s.close()
        out[name] = {"overlap_mode": mode, "deposited_over_absorbed": st["deposited_ph"] / st["absorbed_ph"],
                     "secondary_per_step": sum(st["secondary"]), "march_ms": st["ms_march"],
                     "segments_per_s": sum(st["segments"]) / (st["ms_march"] / 1e3)}
    return out


def bench_config4(nyx, torch):
    """256^3 patchy box (40 Mpc/h, sigma_ln 1.5), 32768 sources, Alg. 3 merging forced (default f_req 0.9,
    and 0.5, where groups form), conservative correction, FP32 and FP64: one step each (a second,
    timed, after a first that builds the geometry tables); catalog sizes, segments, merge and march cost."""
    w = I.config4()
    n_th = 0.01 * float(w.n_h.mean())
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).ravel()).cuda()
    nh, xx, cc, nd = dev(w.n_h), dev(w.x_ion), dev(w.cells), dev(w.ndot)
    g = torch.empty(w.n ** 3, dtype=torch.float64, device="cuda")
    out = {}
    for label, prec, f_req in (("fp32_f_req_0.9", nyx.RT_FP32, 0.9), ("fp32_f_req_0.5", nyx.RT_FP32, 0.5),
                               ("fp64_f_req_0.5", nyx.RT_FP64, 0.5)):
        s = nyx.Solver(w.n, w.box_cm, precision=prec, n_th_cm3=n_th, n_min_ray=4.0, tau_max=30.0, merge_mode=1,
                       merge_f_req=f_req)
        s.set_fields(nh, xx)
        s.add_sources(cc, nd)
        s.step(0.0, g, None)
        _, _, st = s.step(0.0, g, None)
        s.close()
        seg = sum(st["segments"])
        out[label] = {"sources_in": st["n_src_in"], "sources_dedup": st["n_src_dedup"],
                      "sources_traced": st["n_src_emit"], "segments": seg, "secondary": sum(st["secondary"]),
                      "step_ms": st["ms_step"], "march_ms": st["ms_march"],
                      "segments_per_s": seg / (st["ms_march"] / 1e3),
                      "deposited_over_absorbed": st["deposited_ph"] / st["absorbed_ph"]}
    return out


def bench_beyond_l2(nyx, torch, n_sources: int = 64):
    """The 256^3 thin box (40 Mpc/h, sigma_ln = 1.5, x_HI = 1e-4) with its first 64 sources: kappa
    and Gamma (67 + 134 MB with FP32 physics, 134 + 134 MB with FP64) exceed the 129 MB L2, so
    the march's own bytes come from HBM. Both precisions, one untimed step that builds the
    geometry tables, then timed steps with L2 flushed; the roofline of the march kernels in
    algorithmic bytes, the table bytes this box added and which levels read tables or walked."""
    w = I.thin256(n_sources)
    n_th = 0.01 * float(w.n_h.mean())
    dev = torch.device("cuda", torch.cuda.current_device())
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a).ravel()).to(dev)
    d_nh, d_x, d_c, d_nd = d(w.n_h), d(w.x_ion), d(w.cells), d(w.ndot)
    n3 = w.n ** 3
    g = torch.empty(n3, dtype=torch.float64, device=dev)
    h = torch.empty_like(g)
    flush = torch.zeros(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    hbm, _ = load_peaks()
    out = {"workload": f"256^3 lognormal box (40 Mpc/h, sigma_ln 1.5), thin (x_HI=1e-4), first {n_sources} of "
                       "config 4's power-law sources",
           "l2_bytes": 129 << 20}
    for prec, label in ((nyx.RT_FP32, "fp32"), (nyx.RT_FP64, "fp64")):
        before = nyx.rt_geometry_table_bytes(torch.cuda.current_device())
        s = nyx.Solver(w.n, w.box_cm, precision=prec, n_th_cm3=n_th, n_min_ray=4.0, tau_max=30.0)
        s.set_fields(d_nh, d_x)
        s.add_sources(d_c, d_nd)
        s.step(0.0, g, h)
        torch.cuda.synchronize()
        built = nyx.rt_geometry_table_bytes(torch.cuda.current_device()) - before
        ms, stats = time_steps(s, 2, flush, g, h, torch)
        s.close()
        st = stats[-1]
        march_ms = sum(x["ms_march"] for x in stats) / len(stats)
        segs = sum(st["segments"])
        alg = algorithmic_bytes(st, prec)
        levels = [lv for lv in range(len(st["rays"])) if st["rays"][lv]]
        out[label] = {
            "value": segs / (statistics.mean(ms) / 1e3), "unit": "segments/s",
            "march_segments_per_s": segs / (march_ms / 1e3), "ms_per_step": statistics.mean(ms),
            "march_ms_per_step": march_ms, "segments_per_step": segs, "secondary_per_step": sum(st["secondary"]),
            "kappa_gamma_bytes": n3 * ((4 if prec == nyx.RT_FP32 else 8) + 8),
            "roofline": {"bound": "hbm", "achieved": alg / (march_ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                         "frac": alg / (march_ms / 1e3) / 1e9 / hbm,
                         "algorithmic_bytes_per_step": alg},
            "table_levels": [lv for lv in levels if (st["table_levels"] >> lv) & 1],
            "walked_levels": [lv for lv in levels if not (st["table_levels"] >> lv) & 1],
            "segments_by_level": [st["segments"][lv] for lv in levels],
            "geometry_table_bytes_added": built,
        }
    out["geometry_table_bytes_total"] = nyx.rt_geometry_table_bytes(torch.cuda.current_device())
    return out


def bench_spectrum(nyx, torch, w, n_th):
    """Eq. 1 over a blackbody spectrum (1e5 K) on the same box, FP32 and FP64 (geometry tables), a
    timed step after one that builds the tables, beside the gray rate: throughput and the photons
    absorbed."""
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).ravel()).cuda()
    nh, xx, cc, nd = dev(w.n_h), dev(w.x_ion), dev(w.cells), dev(w.ndot)
    g = torch.empty(w.n ** 3, dtype=torch.float64, device="cuda")
    out = {}
    for label, prec, spec in (("fp32_gray", nyx.RT_FP32, 0), ("fp32_blackbody", nyx.RT_FP32, 1),
                              ("fp64_gray", nyx.RT_FP64, 0), ("fp64_blackbody", nyx.RT_FP64, 1)):
        s = nyx.Solver(w.n, w.box_cm, precision=prec, n_th_cm3=n_th, n_min_ray=4.0, tau_max=30.0, spectrum=spec,
                       t_bb_K=1e5)
        s.set_fields(nh, xx)
        s.add_sources(cc[: 3 * 128], nd[:128])          # 128 of the 1024 sources: the FP64 march is slow
        s.step(0.0, g, None)
        _, _, st = s.step(0.0, g, None)
        s.close()
        out[label] = {"segments_per_s": sum(st["segments"]) / (st["ms_march"] / 1e3), "march_ms": st["ms_march"],
                      "absorbed_over_emitted": st["absorbed_ph"] / st["emitted_ph"],
                      "dropped_over_emitted": st["dropped_ph"] / st["emitted_ph"]}
    return out


def bench_batched(nyx, torch, x_mode: str, steps: int, tune: bool, slice_: int | None = None,
                  tile: int | None = None, precision: int | None = None, spectrum: int = 0):
    """64 independent solves (grid sizes from {32,64,96,128}^3, log-uniform source counts on
    [1, 4096], per-solve seeds), FP32 unless `precision` says otherwise, gray unless `spectrum` is 1
    (a 1e5 K blackbody): the graph-captured batch (light
    solves in persistent launches, heavy ones in device-sized per-level launches on parallel
    streams) vs one rt_step per solve. Returns timings, segments and the largest field difference."""
    if precision is None:
        precision = nyx.RT_FP32
    ws = I.batch_solves(64, config=3, x_mode=x_mode)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).ravel()).cuda()
    solvers, outs = [], []
    for w in ws:
        s = nyx.Solver(w.n, w.box_cm, precision=precision, n_th_cm3=0.01 * float(w.n_h.mean()),
                       n_min_ray=4.0, tau_max=30.0, spectrum=spectrum, t_bb_K=1e5)
        s.set_fields(dev(w.n_h), dev(w.x_ion))
        s.add_sources(dev(w.cells), dev(w.ndot))
        solvers.append(s)
        outs.append(torch.empty(w.n ** 3, dtype=torch.float64, device="cuda"))
    plain_out = [torch.empty_like(o) for o in outs]

    def plain_step():
        segs = 0
        for s, o in zip(solvers, plain_out):
            _, _, st = s.step(0.0, o, None)
            segs += sum(st["segments"])
        return segs

    plain_step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        segs = plain_step()
    torch.cuda.synchronize()
    plain_s = (time.perf_counter() - t0) / steps
    b = nyx.Batch(solvers)
    if slice_:
        b.set_params(slice=slice_)
    if tile:
        b.set_params(tile=tile)
    tuned = None
    if tune:
        p, ms = b.tune(repeats=1)
        tuned = {"block": p.block, "blocks_per_sm": p.blocks_per_sm, "tile": p.tile, "slice": p.slice,
                 "group_bytes": p.group_bytes, "ms": ms}
    p_final = b.params()
    b.run(outs, None)              # one direct run: the grouping the graph captures uses its per-solve work
    b.capture()
    b.run(outs, None)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        st = b.run(outs, None)
    torch.cuda.synchronize()
    batch_s = (time.perf_counter() - t0) / steps
    bsegs = sum(sum(x["segments"]) for x in st)
    diff = max(float(torch.linalg.norm(a - c) / max(float(torch.linalg.norm(c)), 1e-300))
               for a, c in zip(outs, plain_out))
    b.close()
    for s in solvers:
        s.close()
    return {"x_variant": x_mode, "precision": "f64" if precision == nyx.RT_FP64 else "f32",
            "rate": "blackbody 1e5 K" if spectrum else "gray", "solves": 64,
            "segments_per_step": bsegs, "plain_segments_per_step": segs,
            "plain_ms_per_step": plain_s * 1e3, "batched_ms_per_step": batch_s * 1e3,
            "plain_value": segs / plain_s, "batched_value": bsegs / batch_s, "factor": plain_s / batch_s,
            "max_rel_l2_batched_vs_plain": diff, "steps": steps, "graph": True, "tuned": tuned,
            "params": {k: getattr(p_final, k) for k in ("block", "blocks_per_sm", "tile", "slice", "group_bytes",
                                                        "heavy_shift")},
            "heavy_solves": sum(1 for x in st if sum(x["segments"]) >= (1 << 26))}


def serving_requests(n_req: int, torch):
    """Config 5 request stream: Poisson arrivals at 200/s (seeded), grids from {64,128,256}^3
    (constant cell size of the 128^3 / 20 Mpc/h box), source counts log-uniform on
    [16, 32768], density per the 128^3 recipe (lognormal sigma_ln 1, mean 2e-4) and x per the
    256^3 recipe (x = clip(v, 0, 1), v a mean-1 lognormal, sigma_ln 1.5). Fields come from a
    pool of 2 seeded realizations per size in pinned memory; sources are drawn per request."""
    rng = np.random.default_rng(I.seed_for(5, 5))
    arrivals = I.poisson_arrivals(200.0, n_req, I.seed_for(5, 5))
    pool = {}
    for n in (64, 128, 256):
        for r in range(2):
            n_h = I.lognormal(n, 2e-4, 1.0, I.seed_for(5, 1, solve=10 * n + r))
            x = np.clip(I.lognormal(n, 1.0, 1.5, I.seed_for(5, 2, solve=10 * n + r)), 0.0, 1.0)
            flat = n_h.reshape(-1)
            k = int(round(0.01 * flat.size))
            top = np.sort(np.argpartition(flat, flat.size - k)[flat.size - k:])
            pin = lambda a: torch.from_numpy(np.ascontiguousarray(a).ravel()).pin_memory().numpy()
            pool[(n, r)] = (pin(n_h), pin(x), top, float(n_h.mean()))
    reqs = []
    for j in range(n_req):
        n = int((64, 128, 256)[rng.integers(0, 3)])
        r = int(rng.integers(0, 2))
        k = int(np.clip(np.floor(np.exp(rng.uniform(np.log(16), np.log(32769)))), 16, 32768))
        n_h, x, top, mean = pool[(n, r)]
        pick = top[rng.integers(0, len(top), size=k)]
        cells = np.stack([pick % n, (pick // n) % n, pick // (n * n)], axis=1).astype(np.int32)
        ndot = I.power_law_ndot(k, I.seed_for(5, 4, solve=j))
        reqs.append(dict(t=float(arrivals[j]), n=n, box=20.0 * n / 128.0 / I.HUBBLE_H * I.MPC_CM, n_h=n_h, x=x,
                         cells=np.ascontiguousarray(cells.ravel()), ndot=ndot, n_th=0.01 * mean))
    return reqs


def bench_serving(nyx, torch, n_req: int):
    """FP32 continuous-batching server vs a plain FIFO server running rt_step (FP64) per request,
    on the same arrival stream; latency = done - arrival."""
    reqs = serving_requests(n_req, torch)
    ring = {n: [torch.empty(n ** 3, dtype=torch.float64).pin_memory().numpy() for _ in range(96)]
            for n in (64, 128, 256)}
    # warm-up, identical for both paths: one request of each grid size through each
    warm = {}
    for q in reqs:
        warm.setdefault(q["n"], q)
    srv = nyx.Server(precision=nyx.RT_FP32, max_batch=64)
    for q in warm.values():
        g = np.empty(q["n"] ** 3)
        srv.poll(srv.submit(q["n"], q["box"], q["n_h"], q["x"], q["cells"], q["ndot"], gamma=g, heat=None,
                            n_th_cm3=q["n_th"], n_min_ray=4.0, tau_max=30.0), wait_s=600.0)
        s = nyx.Solver(q["n"], q["box"], precision=nyx.RT_FP64, n_th_cm3=q["n_th"], n_min_ray=4.0, tau_max=30.0)
        s.set_fields(q["n_h"], q["x"])
        s.add_sources(q["cells"], q["ndot"])
        s.step(0.0, g, None)
        s.close()
    srv.close()
    # ---- served (FP32, batched); the same server (its handle pool warm) then takes the capacity burst
    srv = nyx.Server(precision=nyx.RT_FP32, max_batch=64)
    ids = []
    t0 = time.perf_counter()
    for j, q in enumerate(reqs):
        delay = q["t"] - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        ids.append(srv.submit(q["n"], q["box"], q["n_h"], q["x"], q["cells"], q["ndot"],
                              gamma=ring[q["n"]][j % 96], heat=None, n_th_cm3=q["n_th"], n_min_ray=4.0,
                              tau_max=30.0))
        # keep the output ring safe: never more than 96 requests of a size in flight
        if j >= 64:
            srv.poll(ids[j - 64], wait_s=600.0) if ids[j - 64] is not None else None
            ids[j - 64] = None
    for i in ids:
        if i is not None:
            srv.poll(i, wait_s=600.0)
    t_end = time.perf_counter() - t0
    st = srv.stats()
    served = {"achieved_rps": st["completed"] / t_end, "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
              "mean_ms": st["mean_ms"], "max_ms": st["max_ms"], "segments_per_s": st["segments"] / t_end,
              "segments": st["segments"], "batches": st["batches"], "mem_peak_bytes": st["mem_peak"],
              "gpu_busy_ms": st["busy_ms"], "wall_s": t_end, "completed": st["completed"], "failed": st["failed"],
              "host_phase_ms": {k: st[k] for k in ("load_ms", "src_ms", "bind_ms", "run_ms", "finish_ms", "wait_admit_ms",
                                                   "wait_batch_ms", "wait_finish_ms")}}
    # ---- capacity: every request submitted at once, each path as fast as it goes. The served form's
    # first burst meets a handle pool sized by the Poisson stream and creates most handles; the timed
    # burst is the second, the server's steady state (the plain arms reuse one warm handle per size).
    def burst():
        t0 = time.perf_counter()
        ids = [srv.submit(q["n"], q["box"], q["n_h"], q["x"], q["cells"], q["ndot"], gamma=ring[q["n"]][j % 96],
                          heat=None, n_th_cm3=q["n_th"], n_min_ray=4.0, tau_max=30.0) for j, q in enumerate(reqs[:96])]
        for i in ids:
            srv.poll(i, wait_s=600.0)
        return 96 / (time.perf_counter() - t0)

    cap_first = burst()
    st = srv.stats()
    b0 = st["batches"]
    cap_served = burst()
    st2 = srv.stats()
    cap_batches = st2["batches"] - b0
    cap_phase = {k: st2[k] - st[k] for k in ("load_ms", "src_ms", "bind_ms", "run_ms", "finish_ms", "wait_admit_ms",
                                             "wait_batch_ms", "wait_finish_ms", "busy_ms")}
    srv.close()

    # ---- plain per-request launches, first-come first-served, in FP64 (the per-request baseline) and
    # in FP32 (the same precision as the served form, to separate batching's gain from precision's);
    # one handle per grid size, re-targeted to each request (rt_reconfigure), so no path allocates
    # per request
    def plain_arm(precision, keep_check):
        solvers = {}

        def plain_step(q, out):
            s = solvers.get(q["n"])
            if s is None:
                s = solvers[q["n"]] = nyx.Solver(q["n"], q["box"], precision=precision, n_th_cm3=q["n_th"],
                                                 n_min_ray=4.0, tau_max=30.0)
            else:
                s.reconfigure(q["box"], n_th_cm3=q["n_th"], n_min_ray=4.0, tau_max=30.0)
            s.set_fields(q["n_h"], q["x"])
            s.add_sources(q["cells"], q["ndot"])
            return s.step(0.0, out, None)[2]

        lat, segs, check = [], 0, []
        t0 = time.perf_counter()
        for j, q in enumerate(reqs):
            now = time.perf_counter() - t0
            if q["t"] > now:
                time.sleep(q["t"] - now)
            out = ring[q["n"]][j % 96]
            stp = plain_step(q, out)
            lat.append(1e3 * (time.perf_counter() - t0 - q["t"]))
            segs += sum(stp["segments"])
            if keep_check and j < 4:
                check.append((j, out.copy()))
        t_end_p = time.perf_counter() - t0
        lat_s = sorted(lat)
        q_ = lambda p: lat_s[min(len(lat_s) - 1, int(round(p * (len(lat_s) - 1))))]
        res = {"achieved_rps": len(reqs) / t_end_p, "p50_ms": q_(0.5), "p99_ms": q_(0.99),
               "mean_ms": float(np.mean(lat)), "max_ms": lat_s[-1], "segments_per_s": segs / t_end_p,
               "segments": segs, "wall_s": t_end_p}
        t0 = time.perf_counter()
        for j, q in enumerate(reqs[:96]):
            plain_step(q, ring[q["n"]][j % 96])
        cap = 96 / (time.perf_counter() - t0)
        for s in solvers.values():
            s.close()
        return res, cap, check

    plain, cap_plain, check = plain_arm(nyx.RT_FP64, True)
    plain32, cap_plain32, _ = plain_arm(nyx.RT_FP32, False)
    # accuracy: the first requests served again in FP32 through the server vs their FP64 plain results
    srv = nyx.Server(precision=nyx.RT_FP32)
    errs = []
    for j, ref in check:
        q = reqs[j]
        g = np.empty(q["n"] ** 3)
        rid = srv.submit(q["n"], q["box"], q["n_h"], q["x"], q["cells"], q["ndot"], gamma=g, heat=None,
                         n_th_cm3=q["n_th"], n_min_ray=4.0, tau_max=30.0)
        srv.poll(rid, wait_s=600.0)
        errs.append(float(np.linalg.norm(g - ref) / max(np.linalg.norm(ref), 1e-300)))
    srv.close()
    offered = n_req / reqs[-1]["t"]
    return {"requests": n_req, "offered_rps": offered,
            "capacity_rps": {"served_fp32_batched": cap_served, "plain_fp64_per_request": cap_plain,
                             "plain_fp32_per_request": cap_plain32,
                             "factor": cap_served / cap_plain, "factor_same_precision": cap_served / cap_plain32,
                             "served_first_burst": cap_first,
                             "requests": 96, "batches": cap_batches, "wall_ms": 96e3 / cap_served,
                             "gpu_busy_fraction": cap_phase["busy_ms"] / (96e3 / cap_served),
                             "served_host_phase_ms": cap_phase},
            "served_fp32_batched": served,
            "geometry_table_bytes": nyx.rt_geometry_table_bytes(torch.cuda.current_device()),
            "plain_fp64_per_request": plain, "plain_fp32_per_request": plain32,
            "throughput_factor": served["achieved_rps"] / plain["achieved_rps"],
            "saturated_served": served["achieved_rps"] < 0.95 * offered,
            "saturated_plain": plain["achieved_rps"] < 0.95 * offered,
            "saturated_plain_fp32": plain32["achieved_rps"] < 0.95 * offered,
            "max_rel_l2_fp32_served_vs_fp64_plain": max(errs)}


def run_nyx(args, world, rank, local):
    import torch
    import paper_2512_12466_gb300 as nyx
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    w, n_th = workload()
    n3 = w.n ** 3
    d_nh = torch.from_numpy(w.n_h.ravel()).to(dev)
    d_x = torch.from_numpy(w.x_ion.ravel()).to(dev)
    d_cells = torch.from_numpy(w.cells.ravel()).to(dev)
    d_ndot = torch.from_numpy(w.ndot).to(dev)
    g = torch.empty(n3, dtype=torch.float64, device=dev)
    h = torch.empty_like(g)
    flush = torch.zeros(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)

    results = {}
    for prec, label in ((nyx.RT_FP32, "fp32"), (nyx.RT_FP64, "fp64")):
        s = nyx.Solver(w.n, w.box_cm, precision=prec, n_th_cm3=n_th, n_min_ray=4.0, tau_max=30.0)
        s.set_fields(d_nh, d_x)
        s.add_sources(d_cells, d_ndot)
        steps = args.steps if prec == nyx.RT_FP32 else max(1, min(args.steps, 3))
        for _ in range(args.warmup if prec == nyx.RT_FP32 else 1):
            s.step(0.0, g, h)
        torch.cuda.synchronize()
        clocks = None
        if prec == nyx.RT_FP32:
            sampler = ClockSampler(torch.cuda.current_device())
            sampler.start()
            time.sleep(0.3)
        barrier(world)
        torch.cuda.synchronize()
        ms, stats = time_steps(s, steps, flush, g, h, torch)
        torch.cuda.synchronize()
        barrier(world)
        if prec == nyx.RT_FP32:
            clocks = sampler.stop()
        total_ms = max_over_ranks(sum(ms), world)
        segs = sum(sum(st["segments"]) for st in stats)
        segs_all = sum_over_ranks(float(segs), world)
        st0 = stats[-1]
        march_ms = sum(st["ms_march"] for st in stats)
        alg = sum(algorithmic_bytes(st, prec) for st in stats)
        results[label] = dict(value=segs_all / (total_ms / 1e3), ms_per_step=total_ms / steps, steps=steps,
                              segments_per_step=sum(st0["segments"]), secondary_per_step=sum(st0["secondary"]),
                              rays_per_step=sum(st0["rays"]), march_ms_per_step=march_ms / steps,
                              march_launches_per_step=st0["march_launches"],
                              launches=sum(st["launches"] for st in stats),
                              achieved_gbs=alg / (march_ms / 1e3) / 1e9, clocks=clocks, stats=st0)
        s.close()

    # end to end: pinned host inputs copied in and Gamma read back every step, through the public API
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    hn, hx, hc, hd = pin(w.n_h.ravel()), pin(w.x_ion.ravel()), pin(w.cells.ravel()), pin(w.ndot)
    hg, hh = torch.empty(n3, dtype=torch.float64).pin_memory(), torch.empty(n3, dtype=torch.float64).pin_memory()
    s = nyx.Solver(w.n, w.box_cm, precision=nyx.RT_FP32, n_th_cm3=n_th, n_min_ray=4.0, tau_max=30.0)
    e2e_steps = max(1, min(args.steps, 5))
    for i in range(1 + e2e_steps):
        if i == 1:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
        s.set_fields(hn, hx)
        s.clear_sources()
        s.add_sources(hc, hd)
        _, _, st = s.step(0.0, hg, hh)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)
    e2e_val = sum_over_ranks(float(sum(st["segments"]) * e2e_steps), world) / e2e_s
    s.close()
    h2d = 2 * 8 * n3 + w.cells.nbytes + w.ndot.nbytes
    d2h = 2 * 8 * n3

    if rank != 0:
        return 0
    hbm, peak_kind = load_peaks()
    red = atomic_peak()
    f32 = results["fp32"]
    f64 = results["fp64"]
    line = {
        "metric": METRIC, "value": f32["value"], "unit": "segments/s", "n_gpus": world, "steps": f32["steps"],
        "warmup": args.warmup, "ms_per_step": f32["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": 128, "box_mpc_h": 20.0, "sigma_ln": 1.0, "mean_nH": 2e-4,
                   "sources": 1024, "n_min_ray": 4, "tau_max": 30, "overlap": "conservative (Eqs. 7-8)",
                   "march": "FP32 physics, Kahan-compensated budgets, FP64 deposits and ledger",
                   "l2": "flushed before every timed step (512 MB write)", "parallelism": f"replicas x{world}"},
        "geometry_table_bytes": nyx.rt_geometry_table_bytes(torch.cuda.current_device()),
        "segments_per_step": f32["segments_per_step"], "secondary_per_step": f32["secondary_per_step"],
        "rays_per_step": f32["rays_per_step"],
        "gpu_launches": f32["launches"],
        "roofline": {"bound": "hbm", "achieved": f32["achieved_gbs"], "peak": hbm, "unit": "GB/s",
                     "frac": f32["achieved_gbs"] / hbm, "frac_nominal": f32["achieved_gbs"] / NOMINAL_HBM,
                     "traffic": traffic_per_launch(f32["segments_per_step"], f32["march_launches_per_step"]),
                     "algorithmic_bytes_per_launch": f32["achieved_gbs"] * 1e6 * f32["march_ms_per_step"]
                     / max(1, f32["march_launches_per_step"]),
                     "kernel": "march_table_kernel (FP32, geometry tables)", "peak_kind": peak_kind,
                     # what the counters show binds this kernel: the algorithmic bytes above divide by
                     # the HBM peak by convention, but kappa and Gamma of this box stay in L2
                     "limiter": "L1/L2 throughput and load latency (ncu, one level-7 launch: L1 77%, L2 76% "
                                "of peak, DRAM 6%); kappa and Gamma (25 MB) L2-resident on this box",
                     "march_ms_per_step": f32["march_ms_per_step"],
                     "march_launches_per_step": f32["march_launches_per_step"],
                     # the march's FP64 deposits (one per primary segment and per secondary deposit)
                     # against FP64 atomic adds into an L2-resident array of the same size, measured in
                     # this run: the rates match, but removing the primary deposits (a timing-only
                     # variant) leaves the march time unchanged, so they are not what binds it
                     "l2_atomics": {"achieved": (f32["segments_per_step"] + f32["secondary_per_step"])
                                    / (f32["march_ms_per_step"] / 1e3),
                                    "peak": red["random"], "peak_neighbouring_cells": red["neighbours"],
                                    "unit": "FP64 atomic adds/s",
                                    "frac": (f32["segments_per_step"] + f32["secondary_per_step"])
                                    / (f32["march_ms_per_step"] / 1e3) / max(red["random"], 1.0)}},
        "fp64": {"value": f64["value"], "ms_per_step": f64["ms_per_step"], "steps": f64["steps"],
                 "roofline": {"achieved": f64["achieved_gbs"], "peak": hbm, "unit": "GB/s",
                              "frac": f64["achieved_gbs"] / hbm, "frac_nominal": f64["achieved_gbs"] / NOMINAL_HBM,
                              "traffic": traffic_per_launch(f64["segments_per_step"], f64["march_launches_per_step"],
                                                            "fp64"),
                              "algorithmic_bytes_per_launch": f64["achieved_gbs"] * 1e6 * f64["march_ms_per_step"]
                              / max(1, f64["march_launches_per_step"]),
                              "kernel": "march_table_kernel<double> (FP64, geometry tables, double-float)",
                              "bound": "instruction issue of the double-float arithmetic (ncu, one level-7 launch: "
                                       "issue 68% active, 322 thread instructions per segment at 25.3 of 32 lanes, "
                                       "FP64 pipe 31%, DRAM 9%, before the neighbour cell became selects)"}},
        "e2e": {"value": e2e_val, "unit": "segments/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "steps": e2e_steps},
        "clocks": f32["clocks"],
    }
    if not args.no_variants:
        line["overlap_modes"] = bench_overlap_modes(nyx, torch, w, n_th)
        line["spectrum"] = bench_spectrum(nyx, torch, w, n_th)
        line["config4"] = bench_config4(nyx, torch)
        line["beyond_l2"] = bench_beyond_l2(nyx, torch)
    if not args.no_batched:
        line["batched"] = {"neutral": bench_batched(nyx, torch, "neutral", steps=5, tune=True),
                           "neutral_fp64": bench_batched(nyx, torch, "neutral", steps=5, tune=True,
                                                         precision=nyx.RT_FP64),
                           "neutral_blackbody": bench_batched(nyx, torch, "neutral", steps=5, tune=False,
                                                              spectrum=1),
                           "thin": bench_batched(nyx, torch, "thin", steps=1, tune=False, slice_=1 << 27,
                                                 tile=32)}
    if args.serve_requests > 0:
        line["serving"] = bench_serving(nyx, torch, args.serve_requests)
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line))
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="nyx", choices=["nyx", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the untimed side measurements (overlap modes, spectrum, 256^3 box)")
    ap.add_argument("--serve-requests", type=int, default=2000)
    args = ap.parse_args(argv)
    world, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, world, rank)
    return run_nyx(args, world, rank, local)


if __name__ == "__main__":
    sys.exit(main())
