"""The multi-process path of bench.py on CPU (gloo, world size 2).

The march shards by source with no data-path collective (each rank runs an
independent replica); what the ranks share is the timing protocol: a
barrier on both sides of the timed region, the slowest rank's time and the
sum of every rank's segments. These tests run that protocol's reductions on
two gloo ranks, and the reference arm under torchrun, where rank 0 alone
times the oracle and prints the one JSON line.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, loc = bench.dist_setup()
    assert (w, r, loc) == (world, rank, rank)
    bench.barrier(world)
    mx = bench.max_over_ranks(10.0 + rank, world)          # per-rank step times: the job takes the slowest
    sm = bench.sum_over_ranks(1000.0 * (rank + 1), world)  # per-rank segments: the job processed them all
    bench.barrier(world)
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"max": mx, "sum": sm, "value": sm / mx}, f)
    dist.destroy_process_group()


def test_rank_reductions_gloo(tmp_path):
    """Two gloo ranks: max over ranks of the time, sum of the segments, and
    the whole-job value (all segments over the slowest time) agree on both."""
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    got = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    for g in got:
        assert g["max"] == 11.0 and g["sum"] == 3000.0
        assert g["value"] == pytest.approx(3000.0 / 11.0)


def test_single_process_reductions_are_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5 and bench.sum_over_ranks(2.0, 1) == 2.0
    bench.barrier(1)


def test_reference_arm_under_torchrun():
    """`bench.py --impl reference` launched as the driver launches N > 1: rank 0
    times the oracle and prints one JSON line; rank 1 exits 0 without work."""
    port = _free_port()
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus",
           "2", "--steps", "1", "--warmup", "0"]
    p = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, p.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["steps"] == 1
    assert d["value"] > 0 and d["unit"] == "segments/s" and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
