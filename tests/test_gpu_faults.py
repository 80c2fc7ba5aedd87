"""Failure injection on the host: with NYXRT_FAULT_ALLOC=k the k-th handle allocation (dalloc) of
the process fails as if the device were out of memory. Whichever call meets it (creating the solver,
adding sources, or a step sizing its ray buffers) must return RT_ENOMEM without leaving the solver
unusable: retried once, it succeeds, and the step's result still matches the oracle. Each case runs
in a child process (the allocation count is per process); no device work faults. The ordinals each
stage allocates are read first from a counting run (NYXRT_FAULT_ALLOC_TRACE), so the cases follow
the library's allocation order instead of fixing it."""
import json
import os
import re
import subprocess
import sys

import numpy as np
import pytest

import oracle
from paper_2512_12466_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
import paper_2512_12466_gb300 as nyx
from paper_2512_12466_gb300 import inputs as I
w = I.random_small(12, 3, seed=5, x_mode="mixed", box_cm=12 * 3e21)
failed = []
def attempt(f, label):
    sys.stderr.write("stage " + label + "\n")
    sys.stderr.flush()
    for _ in range(2):
        try:
            return f()
        except nyx.NyxError as e:
            if e.code != nyx.RT_ENOMEM:
                raise
            failed.append(label)
    raise SystemExit("retry failed: " + label)
s = attempt(lambda: nyx.Solver(w.n, w.box_cm, stream=0, n_th_cm3=1e-3), "create")
attempt(lambda: s.set_fields(w.n_h.ravel(), w.x_ion.ravel()), "fields")
attempt(lambda: s.add_sources(w.cells.ravel(), w.ndot), "sources")
g, _, st = attempt(lambda: s.step(), "step")
sys.stderr.write("stage done\n")
s.close()
np.save(sys.argv[2], g)
print(json.dumps({"failed": failed, "segments": sum(st["segments"])}))
"""


def run_child(tmp_path, env_extra):
    out = tmp_path / "gamma.npy"
    env = dict(os.environ, **env_extra)
    p = subprocess.run([sys.executable, "-c", CHILD, ROOT, str(out)], env=env, capture_output=True, text=True,
                       timeout=300)
    assert p.returncode == 0, p.stderr[-2000:]
    return json.loads(p.stdout.strip().splitlines()[-1]), np.load(out), p.stderr


@pytest.fixture(scope="module")
def reference():
    w = I.random_small(12, 3, seed=5, x_mode="mixed", box_cm=12 * 3e21)
    return oracle.run_workload(w, n_th_cm3=1e-3)


@pytest.fixture(scope="module")
def ordinals(tmp_path_factory):
    """Stage -> the dalloc ordinals it makes, from one run without injection."""
    _, _, err = run_child(tmp_path_factory.mktemp("count"), {"NYXRT_FAULT_ALLOC_TRACE": "1"})
    stage, out = None, {}
    for line in err.splitlines():
        m = re.match(r"stage (\w+)$", line)
        if m:
            stage = m.group(1)
            continue
        m = re.match(r"nyxrt-dalloc (\d+)$", line)
        if m:
            out.setdefault(stage, []).append(int(m.group(1)))
    return out


@pytest.mark.parametrize("stage,which", [("create", 0), ("create", -1), ("sources", 0), ("sources", -1),
                                         ("step", 0), ("step", -1), (None, None)])
def test_allocation_failure_is_recoverable(reference, ordinals, tmp_path, stage, which):
    assert set(ordinals) >= {"create", "sources", "step"}, ordinals
    k = ordinals[stage][which] if stage else 1 + max(max(v) for v in ordinals.values())
    res, g, _ = run_child(tmp_path, {"NYXRT_FAULT_ALLOC": str(k)})
    assert res["failed"] == ([stage] if stage else []), (k, res, ordinals)
    g = g.reshape(reference["gamma"].shape)
    assert np.linalg.norm(g - reference["gamma"]) / np.linalg.norm(reference["gamma"]) < 1e-12
    assert res["segments"] == sum(reference["stats"]["segments"])
