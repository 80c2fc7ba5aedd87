"""Small, fixed march workloads for profilers (ncu): the 128^3 thin box with
its first k sources, traced by rt_step on device-resident inputs.

    python -m paper_2512_12466_gb300.profile_case --sources 64 --precision fp32 --steps 1

Each step launches the field preparation, the source stage, one march launch
per level (slices of 2^27 children at most) and the finalize kernel, in that
order, so `ncu -k regex:march_kernel -s L -c 1` selects the level-L launch of
the first step. Prints one line per step (segments, march time, launches).
--merge adds the Alg. 3 kernels (the 256^3 patchy box with its first k of
32768 sources, f_req = 0.5), --chem the C2-Ray iteration (Table 1 Test A over
1 Myr), --batch K the persistent batched kernel over the first K solves of
the 64-solve uneven mix (one direct run), --thin256 the 256^3 thin box (40
Mpc/h, sigma_ln = 1.5, x_HI = 1e-4) with its first k sources, whose kappa and
Gamma do not fit the L2 cache.
"""
import argparse
import sys

import numpy as np


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--sources", type=int, default=64, help="first k sources of the 1024 (default 64)")
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--x", choices=["thin", "neutral"], default="thin", help="ionized-fraction variant")
    ap.add_argument("--overlap", type=int, default=3, help="overlap_mode (0 none .. 3 conservative, 4 squared, 5 naive)")
    ap.add_argument("--levels", action="store_true", help="also print segments and rays per level")
    ap.add_argument("--walk", action="store_true", help="walk every ray instead of reading geometry tables")
    ap.add_argument("--merge", action="store_true", help="256^3 patchy box, Alg. 3 merging forced")
    ap.add_argument("--chem", action="store_true", help="Table 1 Test A (64^3) with the C2-Ray iteration")
    ap.add_argument("--batch", type=int, default=0, help="K solves of the uneven mix through the batched kernel")
    ap.add_argument("--spectrum", action="store_true", help="Eq. 1 over a 1e5 K blackbody instead of the gray rate")
    ap.add_argument("--thin256", action="store_true", help="256^3 thin box (kappa and Gamma beyond L2)")
    a = ap.parse_args(argv)
    import torch
    import paper_2512_12466_gb300 as nyx
    from paper_2512_12466_gb300 import inputs as I
    prec = nyx.RT_FP32 if a.precision == "fp32" else nyx.RT_FP64
    flags = nyx.RT_FLAG_NO_GEOMETRY_TABLE if a.walk else 0
    dev = torch.device("cuda")
    d = lambda v: torch.from_numpy(np.ascontiguousarray(v).ravel()).to(dev)
    if a.batch:
        solves = I.batch_solves(x_mode=a.x)[: a.batch]
        ss = []
        for w in solves:
            s = nyx.Solver(w.n, w.box_cm, precision=nyx.RT_FP32, n_th_cm3=0.01 * float(w.n_h.mean()),
                           n_min_ray=4.0, tau_max=30.0, flags=flags)
            s.set_fields(d(w.n_h), d(w.x_ion))
            s.add_sources(d(w.cells.astype(np.int32)), d(w.ndot))
            ss.append(s)
        b = nyx.Batch(ss)
        outs = [torch.empty(w.n ** 3, dtype=torch.float64, device=dev) for w in solves]
        for r in range(a.steps):
            sts = b.run(outs, None)
            seg = sum(sum(st["segments"]) for st in sts)
            print(f"step {r}: solves {len(ss)} segments {seg} batch_ms {sts[0]['ms_step']:.3f}", flush=True)
        b.close()
        for s in ss:
            s.close()
        return 0
    dt = 0.0
    if a.merge:
        w = I.config4()
        cfg = dict(merge_mode=1, merge_f_req=0.5)
    elif a.thin256:
        w = I.thin256(max(1, a.sources))
        cfg = {}
    elif a.chem:
        w = I.stromgren_test("A", 64)
        cfg = {k: w.params[k] for k in ("chem_iterate", "alpha_B", "clumping", "C_H")}
        dt = 1.0 * I.MYR_S
    else:
        w = I.config2(a.x)
        cfg = {}
    k = max(0, min(a.sources, len(w.ndot)))
    if a.spectrum:
        cfg.update(spectrum=nyx.RT_SPECTRUM_BLACKBODY, t_bb_K=1e5)
    s = nyx.Solver(w.n, w.box_cm, precision=prec, n_th_cm3=0.01 * float(w.n_h.mean()), overlap_mode=a.overlap,
                   n_min_ray=4.0, tau_max=30.0, flags=flags, **cfg)
    s.set_fields(d(w.n_h), d(w.x_ion))
    if k:
        s.add_sources(d(w.cells[:k].astype(np.int32)), d(w.ndot[:k]))
    g = torch.empty(w.n ** 3, dtype=torch.float64, device=dev)
    h = torch.empty_like(g)
    for r in range(a.steps):
        _, _, st = s.step(dt, g, h)
        seg = sum(st["segments"])
        print(f"step {r}: sources {k} segments {seg} secondary {sum(st['secondary'])} "
              f"step_ms {st['ms_step']:.3f} march_ms {st['ms_march']:.3f} march_launches {st['march_launches']} "
              f"Gseg/s {seg / max(st['ms_march'], 1e-9) / 1e6:.2f} traced {st['n_src_emit']} "
              f"chem_iters {st['chem_iters']}", flush=True)
        if a.levels:
            for l, (sg, ry, sc) in enumerate(zip(st["segments"], st["rays"], st["secondary"])):
                if ry:
                    print(f"  level {l}: rays {ry} segments {sg} secondary {sc}", flush=True)
    print(f"geometry tables on device {torch.cuda.current_device()}: "
          f"{nyx.rt_geometry_table_bytes(torch.cuda.current_device()) / 2**20:.1f} MiB", flush=True)
    s.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
