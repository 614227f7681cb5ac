"""labs_enumerate_noalloc: the enumeration for callers that cannot allocate device
memory when they call (its scratch is a fixed array inside the library).

Called through the C ABI and compared with labs_enumerate (which takes a caller
scratch buffer) on two calls in a row of different sizes, so that the second call
runs on an array that still holds the first call's contents.  The results are
integers, compared exactly, as in the other enumeration tests.  This file is collected
last on purpose."""
from __future__ import annotations

import ctypes

import pytest
import torch

from paper_2011_00068_gb300 import _native

pytestmark = pytest.mark.gpu


def with_caller_scratch(lib, L, stream):
    n = ctypes.c_size_t()
    assert lib.labs_enumerate_scratch_bytes(L, ctypes.byref(n)) == 0
    scratch = torch.empty(n.value, dtype=torch.uint8, device="cuda")
    m, c, f = ctypes.c_int64(), ctypes.c_uint64(), ctypes.c_uint64()
    rc = lib.labs_enumerate(L, ctypes.c_void_p(scratch.data_ptr()), n.value, ctypes.byref(m), ctypes.byref(c),
                            ctypes.byref(f), ctypes.c_void_p(stream.cuda_stream))
    assert rc == 0
    return m.value, c.value, f.value


def without_allocation(lib, L, stream):
    m, c, f = ctypes.c_int64(), ctypes.c_uint64(), ctypes.c_uint64()
    rc = lib.labs_enumerate_noalloc(L, ctypes.byref(m), ctypes.byref(c), ctypes.byref(f),
                                    ctypes.c_void_p(stream.cuda_stream))
    assert rc == 0
    return m.value, c.value, f.value


def test_noalloc_matches_scratch_entry_point_twice():
    lib = _native.load()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    for L in (41, 27):  # the larger size first: the second call sees stale partials
        want = with_caller_scratch(lib, L, stream)
        got = without_allocation(lib, L, stream)
        assert got == want
    assert without_allocation(lib, 41, stream) == (108, 2, with_caller_scratch(lib, 41, stream)[2])


def test_noalloc_rejects_lengths_beyond_its_limit():
    lib = _native.load()
    stream = torch.cuda.current_stream()
    m, c, f = ctypes.c_int64(), ctypes.c_uint64(), ctypes.c_uint64()
    for L in (65, 64, 1):
        assert lib.labs_enumerate_noalloc(L, ctypes.byref(m), ctypes.byref(c), ctypes.byref(f),
                                          ctypes.c_void_p(stream.cuda_stream)) == _native.LABS_EINVAL
