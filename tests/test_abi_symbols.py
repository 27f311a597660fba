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
