"""CPU-only checks of the C ABI: the library builds for sm_103a, loads, and
exports every function include/semisort.h declares; host-side argument checks
work without a GPU (no compute call is made)."""
import ctypes
import os
import re

import pytest

import paper_2304_10078_gb300 as ss

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    ss.build()
    return ss.lib()


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ ]*?\**\s*\**\b([a-z_][a-z0-9_]*)\s*\(",
                                text, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "semisort_equal" in names and "ss_workspace_size" in names
    for name in names:
        assert hasattr(lib, name), name


def test_workspace_size_and_argument_checks(lib):
    n = 1 << 20
    nbytes = ss.workspace_size(ss.OP_EQUAL, ss.SS_U64, ss.SS_U64, n)
    assert nbytes >= 16 * n  # the temporary array T (Sec. 3.2) alone
    with pytest.raises(ss.SemisortError) as e:
        ss.workspace_size(ss.OP_EQUAL, ss.SS_U64, ss.SS_U64, 1 << 33)
    assert e.value.code == 2
    u64 = ctypes.c_uint64
    # null keys with n > 0 is rejected on the host
    rc = lib.semisort_equal(ss.SS_U64, ss.SS_U64, None, None, None, None, 10, None, 0, None, None)
    assert rc == 1
    # n = 0 is valid and enqueues nothing
    rc = lib.semisort_equal(ss.SS_U64, ss.SS_U64, None, None, None, None, 0, None, 0, None, None)
    assert rc == 0
    # pointers not aligned to their element size are rejected
    rc = lib.semisort_equal(ss.SS_U64, ss.SS_U64, ctypes.c_void_p(12), ctypes.c_void_p(4096),
                            ctypes.c_void_p(1 << 20), ctypes.c_void_p(1 << 21), 4, ctypes.c_void_p(1 << 22),
                            1 << 30, None, None)
    assert rc == 1
    # partial overlap of input and output is rejected
    rc = lib.semisort_equal(ss.SS_U64, ss.SS_U64, ctypes.c_void_p(1 << 20), None, ctypes.c_void_p((1 << 20) + 16),
                            None, 100, ctypes.c_void_p(1 << 30), 1 << 30, None, None)
    assert rc == 1
    # a workspace below the planned size is rejected
    rc = lib.semisort_equal(ss.SS_U64, ss.SS_U64, ctypes.c_void_p(1 << 20), None, ctypes.c_void_p(1 << 24),
                            None, 100_000, ctypes.c_void_p(1 << 30), 1024, None, None)
    assert rc == 3
    assert lib.ss_status_string(3) == b"workspace too small"
