"""C-ABI checks that need no GPU: the library builds for sm_103a, loads,
exports every entry point include/nyxrt.h declares, and the ctypes binding's
struct layouts match the C header (checked with a gcc-compiled probe)."""
import ctypes as C
import os
import re
import subprocess

import pytest

import paper_2512_12466_gb300 as nyx
from paper_2512_12466_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nyxrt.h")


@pytest.fixture(scope="module")
def built():
    return _build.build()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rt_\w+)\s*\(", text)))


def test_header_declares_expected_entry_points():
    names = declared_functions()
    for f in ["rt_create", "rt_set_fields", "rt_add_sources", "rt_step", "rt_destroy"]:
        assert f in names


def test_library_exports_every_declared_symbol(built):
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(rt_\w+)", out))
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing
    lib = C.CDLL(built)
    for f in declared_functions():
        getattr(lib, f)
    assert set(nyx.exported_symbols()) == set(declared_functions())


def test_struct_layout_matches_header(tmp_path):
    """Every struct the binding mirrors has the header's size and field offsets (a gcc probe
    compiled from the header as C)."""
    structs = [nyx.rt_config, nyx.rt_stats, nyx.rt_batch_params, nyx.rt_server_config, nyx.rt_server_stats]
    prog = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', "int main(void) {"]
    for st in structs:
        name = st.__name__
        prog.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in st._fields_:
            prog.append(f'printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    prog.append("return 0; }")
    src = tmp_path / "probe.c"
    src.write_text("\n".join(prog))
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-o", str(exe), str(src)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split("\n")
               if line)
    for st in structs:
        name = st.__name__
        assert int(got[name]) == C.sizeof(st), name
        for f, _ in st._fields_:
            assert int(got[f"{name}.{f}"]) == getattr(st, f).offset, (name, f)


def test_config_defaults_host_only(built):
    cfg = nyx.rt_config_default(64, 1e22)
    assert cfg.n == 64 and cfg.box_cm == 1e22
    assert cfg.precision == nyx.RT_FP64 and cfg.overlap_mode == nyx.RT_OVERLAP_CONSERVATIVE
    assert cfg.n_min_ray == 4.0 and cfg.tau_max == 30.0 and cfg.level_max == -1
    assert cfg.merge_dr_cells == 2.0 and cfg.merge_samp_level == 3
    assert "sm_103a" in nyx.rt_version()


def test_product_path_has_no_oracle_dependency():
    """The binding and the CUDA sources never reference the CPU oracle."""
    pkg = os.path.join(ROOT, "paper_2512_12466_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cpp", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in text.lower() or f == "inputs.py", f


def _checkpoint_bytes(n: int, nc: int, ns: int, payload: int) -> bytes:
    """A checkpoint header (magic, version, configuration, cell count), `payload` bytes of data
    and a source count, as rt_save lays them out."""
    cfg = nyx.rt_config_default(n, 1e22)
    head = b"NYXRTCK1" + (1).to_bytes(4, "little") + C.sizeof(nyx.rt_config).to_bytes(4, "little")
    head += bytes(cfg) + nc.to_bytes(8, "little", signed=True)
    return head + bytes(payload) + ns.to_bytes(8, "little", signed=True) + bytes(64)


@pytest.mark.parametrize("n,ns,payload", [
    (8, 1 << 30, 16 * 512),            # a source count of 2^30 in a file that holds 64 bytes of sources
    (1024, 0, 4096),                   # a 1024^3 grid (16 GB of fields) in a file of a few kB
    (8, 3, 16 * 512),                  # 3 sources claimed, 64 bytes present (60 needed): trailing bytes
])
def test_load_checks_counts_against_the_file_size(built, tmp_path, n, ns, payload):
    """rt_load sizes nothing from a count in the header before the file is known to hold that
    much data: a short or padded file is RT_EINVAL, before any host buffer or CUDA call."""
    p = tmp_path / "bad.ckpt"
    p.write_bytes(_checkpoint_bytes(n, n ** 3, ns, payload))
    with pytest.raises(nyx.NyxError) as e:
        nyx.rt_load(str(p))
    assert e.value.code == nyx.RT_EINVAL
    assert "not a complete checkpoint" in str(e.value)
