"""The C-ABI library builds, loads and exports every entry point declared in
include/labs.h (no GPU: no compute call is made)."""
from __future__ import annotations

import ctypes
import os
import re

import pytest

from paper_2011_00068_gb300 import _native, build

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "labs.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return re.findall(r"\b(labs_[a-z_]+)\s*\(", text)


@pytest.fixture(scope="module")
def lib():
    try:
        build.nvcc()
    except RuntimeError:
        pytest.skip("no nvcc in this environment")
    return _native.load()


def test_header_matches_binding_table():
    assert declared_functions() == _native.EXPORTS


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_host_only_calls(lib):
    cfg = _native.LabsConfig()
    lib.labs_default_config(ctypes.byref(cfg))
    assert (cfg.tabu_log2, cfg.probe_cap, cfg.patience, cfg.target_num, cfg.target_den) == (16, 32, 0, 17, 2)
    n = ctypes.c_size_t()
    assert lib.labs_enumerate_scratch_bytes(41, ctypes.byref(n)) == 0 and n.value > 0
    assert lib.labs_enumerate_scratch_bytes(40, ctypes.byref(n)) == _native.LABS_EINVAL
    assert lib.labs_enumerate_scratch_bytes(65, ctypes.byref(n)) == _native.LABS_EINVAL
    assert lib.labs_last_error(None) == b"null context"


def test_built_for_sm103a(lib):
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)
