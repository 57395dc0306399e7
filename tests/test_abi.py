"""The C-ABI library builds, loads and exports every entry point of
include/sp.h (no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sp.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2507_11094_gb300 import build, sp
    build.build()
    return sp.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sp_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("sp_graph_create", "sp_sssp_init", "sp_apply_batch", "sp_get_dist",
                     "sp_graph_destroy", "sp_status_str"):
        assert required in names


def test_library_exports_every_declared_function(lib):
    from paper_2507_11094_gb300 import build
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(sp_[a-z_0-9]+)$", out, flags=re.M))
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing
    for f in declared_functions():
        assert hasattr(lib, f)


def test_binding_covers_every_declared_function():
    from paper_2507_11094_gb300 import sp
    assert sorted(sp.SIGNATURES) == declared_functions()


def test_status_strings_and_version(lib):
    from paper_2507_11094_gb300 import sp
    for code, name in sp.STATUS.items():
        assert sp.status_str(code).startswith(name)
    assert re.match(rb"^\d+\.\d+\.\d+$", lib.sp_version())


def test_argument_checks_need_no_device(lib):
    # rejected before any CUDA call
    h = ctypes.c_void_p()
    assert lib.sp_graph_create(0, 0, None, None, None, 0, 0.25, None, None,
                               ctypes.byref(h)) == -1
    assert lib.sp_graph_destroy(None) == 0
    assert lib.sp_sssp_init(None, 0, None) == -1
    assert lib.sp_apply_batch(None, 0, None, None, 0, None, None, None, 0, None) == -1
    assert lib.sp_apply_batch_get(None, 0, None, None, 0, None, None, None, 0, None, None, 1,
                                  None) == -1
    from paper_2507_11094_gb300 import sp
    srv = ctypes.c_void_p()
    assert lib.sp_server_create(None, ctypes.byref(srv)) == -1
    bad = sp.ServerConfig(1 << 30, 0, 0, 0.25, 0)           # no worker slots
    assert lib.sp_server_create(ctypes.byref(bad), ctypes.byref(srv)) == -1
    bad = sp.ServerConfig(0, 2, 0, 0.25, 0)                 # no budget
    assert lib.sp_server_create(ctypes.byref(bad), ctypes.byref(srv)) == -1
    assert lib.sp_server_destroy(None) == 0
    assert lib.sp_server_drain(None) == -1


def test_stats_struct_layout_matches_header():
    from paper_2507_11094_gb300 import sp
    # 10 int64 + 4 int32 + 8 int64 + 8 float + 1 float, 8-byte aligned
    assert ctypes.sizeof(sp.BatchStats) == 10 * 8 + 4 * 4 + 8 * 8 + 8 * 4 + 4 + 4


def test_product_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2507_11094_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "liboracle" not in txt, f


def test_struct_layouts_match_the_c_compiler(tmp_path):
    """sizeof/offsetof of every struct of the header, as gcc lays them out,
    equal the ctypes mirrors."""
    from paper_2507_11094_gb300 import sp
    mirrors = {"sp_batch_stats": sp.BatchStats, "sp_graph_info": sp.GraphInfo,
               "sp_server_config": sp.ServerConfig, "sp_request_info": sp.RequestInfo,
               "sp_server_stats": sp.ServerStats}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "sp.h"',
             "int main(void) {"]
    for cname, py in mirrors.items():
        lines.append(f'printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True,
                               check=True).stdout.splitlines():
        c, f, v = line.split()
        got[(c, f)] = int(v)
    for cname, py in mirrors.items():
        assert got[(cname, "sizeof")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)


def test_export_targets_are_checked_before_any_launch():
    """export_csr_device writes through raw device pointers, so a wrong dtype,
    a short or strided tensor, a host tensor or overlapping targets must be
    refused in the binding, before the C call."""
    import types

    import torch
    from paper_2507_11094_gb300 import sp
    g = types.SimpleNamespace(n=10, m=20, device=0)
    ok = (torch.zeros(11, dtype=torch.int64), torch.zeros(20, dtype=torch.int32),
          torch.zeros(20, dtype=torch.int32))
    cases = [
        ((torch.zeros(11, dtype=torch.int32),) + ok[1:], "dtype"),
        ((torch.zeros(10, dtype=torch.int64),) + ok[1:], "at least 11"),
        ((ok[0], torch.zeros(19, dtype=torch.int32), ok[2]), "at least 20"),
        ((ok[0], ok[1], torch.zeros(20, dtype=torch.float32)), "dtype"),
        ((ok[0], torch.zeros(40, dtype=torch.int32)[::2], ok[2]), "contiguous"),
        ((ok[0], [0] * 20, ok[2]), "torch tensor"),
        (ok, "CUDA tensor"),
    ]
    for args, msg in cases:
        with pytest.raises(ValueError, match=msg):
            sp._check_export_targets(g, *args)


def test_apply_batch_get_outputs_are_checked_before_the_call():
    """apply_batch_get writes n distances (and parents) through raw pointers:
    host outputs of the wrong dtype, length or layout, or read-only ones, are
    refused in the binding before the C call (no GPU needed)."""
    from paper_2507_11094_gb300 import sp
    g = sp.Graph.__new__(sp.Graph)
    g.n, g.device, g._h = 10, 0, None
    z = np.zeros(3, np.int32)
    ro = np.zeros(10, np.int32)
    ro.flags.writeable = False
    for bad in (np.zeros(9, np.int32), np.zeros(10, np.int64), np.zeros(20, np.int32)[::2],
                ro, [0] * 10):
        with pytest.raises(sp.SpError):
            g.apply_batch_get(z, z, z, z, z, bad)
    with pytest.raises(sp.SpError):   # a bad parent array with a good dist
        g.apply_batch_get(z, z, z, z, z, np.zeros(10, np.int32), np.zeros(9, np.int32))
    with pytest.raises(sp.SpError):   # batch arrays of different lengths
        g.apply_batch_get(z, z[:2], z, z, z, np.zeros(10, np.int32))
