"""Fused multiply-add throughput of the FP32 and FP64 pipes on GPU 0 (the ALU roofline
denominators of the march kernels), from libnyxrt_probe.so, and with --copies the host<->device
copy bandwidth from pinned memory (the serving form's transfer roofline):

    python -m paper_2512_12466_gb300.probe_peaks [--copies]

Prints one JSON line: TFLOP/s (2 flops per FMA) and FMA instructions per second for each
precision, best of three timed launches; FP64 atomic adds per second into an L2-resident and a
2 GB array, at random and at neighbouring cells; with --copies, GB/s of 128 MiB copies host to device,
device to host and both at once, on 1, 2 and 4 streams (torch copies, wall time of 8 rounds).
"""
import ctypes as C
import json
import os
import sys


def main() -> int:
    from paper_2512_12466_gb300 import _build
    path = _build.build_probe()
    lib = C.CDLL(path)
    lib.nyxrt_probe_fma.argtypes = [C.c_int, C.c_int64, C.POINTER(C.c_double), C.POINTER(C.c_double)]
    lib.nyxrt_probe_fma.restype = C.c_int
    out = {}
    for bits, iters in ((32, 1 << 16), (64, 1 << 11)):
        best, ms_best = 0.0, 0.0
        for _ in range(3):
            tf, ms = C.c_double(), C.c_double()
            rc = lib.nyxrt_probe_fma(bits, iters, C.byref(tf), C.byref(ms))
            if rc != 0:
                print(json.dumps({"error": f"probe returned {rc} for FP{bits}"}))
                return 1
            if tf.value > best:
                best, ms_best = tf.value, ms.value
        out[f"fp{bits}"] = {"tflops": best, "fma_per_s": best * 1e12 / 2, "kernel_ms": ms_best, "iters": iters}
    out["fp32_over_fp64"] = out["fp32"]["tflops"] / out["fp64"]["tflops"]
    # FP64 atomic adds (the march's deposits): an L2-resident array the size of a 128^3 Gamma grid
    # and one of 2 GB (beyond L2), random cells, neighbouring cells per warp, and one random cell per
    # group of 4 or 16 lanes
    lib.nyxrt_probe_red_f64.argtypes = [C.c_int64, C.c_int64, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]
    lib.nyxrt_probe_red_f64.restype = C.c_int
    red = {}
    for label, n in (("l2_128cubed", 128 ** 3), ("dram_2GB", 1 << 28)):
        for pname, pat in (("random", 0), ("neighbours", 1), ("shared4", 2), ("shared16", 3)):
            best = 0.0
            for _ in range(3):
                ps, ms = C.c_double(), C.c_double()
                rc = lib.nyxrt_probe_red_f64(n, 256, pat, C.byref(ps), C.byref(ms))
                if rc != 0:
                    print(json.dumps({"error": f"atomic probe returned {rc}"}))
                    return 1
                best = max(best, ps.value)
            red[f"{label}_{pname}_per_s"] = best
    out["red_add_f64"] = red
    if "--copies" in sys.argv[1:]:
        out["copies_gbs"] = copy_bandwidth()
    print(json.dumps(out))
    return 0


def copy_bandwidth(size: int = 128 << 20, rounds: int = 8) -> dict:
    import time

    import torch
    torch.cuda.set_device(0)
    res = {}
    for direction in ("h2d", "d2h", "both"):
        for k in (1, 2, 4):
            host = [torch.empty(size // 8, dtype=torch.float64).pin_memory() for _ in range(2 * k)]
            dev = [torch.empty(size // 8, dtype=torch.float64, device="cuda") for _ in range(2 * k)]
            streams = [torch.cuda.Stream() for _ in range(2 * k)]
            best = 0.0
            for _ in range(2):
                torch.cuda.synchronize()
                t = time.perf_counter()
                for _ in range(rounds):
                    for i in range(k):
                        if direction in ("h2d", "both"):
                            with torch.cuda.stream(streams[i]):
                                dev[i].copy_(host[i], non_blocking=True)
                        if direction in ("d2h", "both"):
                            with torch.cuda.stream(streams[k + i]):
                                host[k + i].copy_(dev[k + i], non_blocking=True)
                torch.cuda.synchronize()
                dt = time.perf_counter() - t
                moved = rounds * k * size * (2 if direction == "both" else 1)
                best = max(best, moved / dt / 1e9)
            res[f"{direction}_{k}_streams"] = round(best, 1)
    return res


if __name__ == "__main__":
    sys.exit(main())
