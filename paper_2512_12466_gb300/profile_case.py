"""Small, fixed march workloads for profilers (ncu): the 128^3 thin box with
its first k sources, traced by rt_step on device-resident inputs.

    python -m paper_2512_12466_gb300.profile_case --sources 64 --precision fp32 --steps 1

Each step launches the field preparation, the source stage, one march launch
per level (slices of 2^27 children at most) and the finalize kernel, in that
order, so `ncu -k regex:march_kernel -s L -c 1` selects the level-L launch of
the first step. Prints one line per step (segments, march time, launches).
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
    ap.add_argument("--overlap", type=int, default=3, help="overlap_mode (0 none .. 3 conservative, 4 squared)")
    ap.add_argument("--levels", action="store_true", help="also print segments and rays per level")
    ap.add_argument("--walk", action="store_true", help="FP32: walk every ray instead of reading geometry tables")
    a = ap.parse_args(argv)
    import torch
    import paper_2512_12466_gb300 as nyx
    from paper_2512_12466_gb300 import inputs as I
    w = I.config2(a.x)
    k = max(0, min(a.sources, len(w.ndot)))
    dev = torch.device("cuda")
    d = lambda v: torch.from_numpy(np.ascontiguousarray(v).ravel()).to(dev)
    s = nyx.Solver(w.n, w.box_cm, precision=nyx.RT_FP32 if a.precision == "fp32" else nyx.RT_FP64,
                   n_th_cm3=0.01 * float(w.n_h.mean()), overlap_mode=a.overlap,
                   flags=nyx.RT_FLAG_NO_GEOMETRY_TABLE if a.walk else 0)
    s.set_fields(d(w.n_h), d(w.x_ion))
    if k:
        s.add_sources(d(w.cells[:k].astype(np.int32)), d(w.ndot[:k]))
    g = torch.empty(w.n ** 3, dtype=torch.float64, device=dev)
    h = torch.empty_like(g)
    for r in range(a.steps):
        _, _, st = s.step(0.0, g, h)
        seg = sum(st["segments"])
        print(f"step {r}: sources {k} segments {seg} secondary {sum(st['secondary'])} "
              f"march_ms {st['ms_march']:.3f} march_launches {st['march_launches']} "
              f"Gseg/s {seg / max(st['ms_march'], 1e-9) / 1e6:.2f}", flush=True)
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
