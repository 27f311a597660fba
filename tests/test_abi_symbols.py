"""The C-ABI library loads (no GPU needed) and exports every symbol include/gd.h declares."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "gd.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:gd_status|const char\*)\s+(gd_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_boundary():
    names = _declared()
    for want in ("gd_create", "gd_destroy", "gd_build_neighbors", "gd_collision_rates",
                 "gd_sample_collisions", "gd_push_staggered", "gd_stats"):
        assert want in names


def test_library_exports_every_declared_symbol():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available to build libgd.so")
    from paper_2609_35967_gb300 import binding, build
    build.build()
    lib = ctypes.CDLL(binding.LIB_PATH)
    for name in _declared():
        assert hasattr(lib, name), name
    assert set(_declared()) == set(binding.SIGNATURES)


def test_status_strings_without_gpu():
    from paper_2609_35967_gb300 import binding, build
    if not os.path.exists(binding.LIB_PATH):
        build.build()
    assert binding.gd_status_string(0) == "ok"
    assert binding.gd_status_string(-8) == "calls out of order"


def test_create_rejects_bad_arguments_without_gpu():
    """Argument checks run before any CUDA call."""
    from paper_2609_35967_gb300 import binding, build
    if not os.path.exists(binding.LIB_PATH):
        build.build()
    L = binding.load()
    h = ctypes.c_void_p()
    assert L.gd_create(ctypes.byref(h), None) == binding.GD_ERR_ARG
    cfg = binding.Config()
    cfg.n_instances = 1
    cfg.K = 1                         # K must be at least 2
    assert L.gd_create(ctypes.byref(h), ctypes.byref(cfg)) == binding.GD_ERR_ARG
    assert L.gd_build_neighbors(None, None, None) == binding.GD_ERR_ARG
    assert L.gd_stats(None, None, None) == binding.GD_ERR_ARG


def test_binding_structs_match_the_header(tmp_path):
    """The ctypes mirrors of the header's structs have the C sizes and field offsets
    (a C program built with gcc prints them; no GPU)."""
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    import subprocess
    from paper_2609_35967_gb300 import binding
    structs = {"gd_instance_params": binding.InstanceParams, "gd_config": binding.Config,
               "gd_stats_t": binding.Stats, "gd_instance_stats": binding.InstanceStats,
               "gd_group_stats_t": binding.GroupStats, "gd_dt_rule": binding.DtRule}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "gd.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'  printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("  return 0;\n}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = dict(line.rsplit(" ", 1) for line in out if line)
    for cname, py in structs.items():
        assert int(got[cname]) == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert int(got[f"{cname}.{f}"]) == getattr(py, f).offset, (cname, f)
