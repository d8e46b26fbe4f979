"""The C-ABI library loads and exports every entry point declared in include/*.h.

No compute call is made here, so these run on a machine without a GPU.
"""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(adpar_\w+)\s*\(", src, re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2202_10297_gb300 import build as B
    path = B.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = _declared()
    assert "adpar_vjp_scan" in names and "adpar_workspace_size" in names
    assert len(names) >= 5


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_without_gpu(lib):
    lib.adpar_status_string.restype = ctypes.c_char_p
    assert lib.adpar_status_string(0) == b"ok"
    assert lib.adpar_status_string(6).startswith(b"device-side")


def test_host_side_validation_without_gpu():
    """Argument errors return before any CUDA call, so they work without a GPU."""
    from paper_2202_10297_gb300 import adpar as A
    L = A.lib()
    d = A.OpDesc(A.OP_LINREC, A.F32, 1)  # wrong width for LINREC
    assert L.adpar_vjp_scan(d, 10, None, None, None, None, None, None, None, None, 0, None, 0, None) == 1
    d = A.OpDesc(A.OP_ADD, A.F32, 1)
    assert L.adpar_vjp_scan(d, -1, None, None, None, None, None, None, None, None, 0, None, 0, None) == 1
    # misaligned pointer
    assert L.adpar_vjp_scan(d, 10, None, None, 0x1004, None, 0x2000, None, None, None, 0, None, 0, None) == 3
    # workspace missing
    assert L.adpar_vjp_scan(d, 10, None, None, 0x1000, None, 0x2000, None, None, None, 0, None, 0, None) == 4
    # n == 0 with a valid workspace is a no-op
    ws = A.adpar_workspace_size(A.RULE_SCAN, A.OP_ADD, A.F32, 0)
    assert ws >= 256
    assert A.adpar_workspace_size(A.RULE_SCAN, A.OP_LINREC, A.F64, 1 << 26) > A.adpar_workspace_size(
        A.RULE_SCAN, A.OP_LINREC, A.F64, 1 << 20)
    # the full scan workspace of FP64 MUL/LINREC holds the factored forward
    # result (8 bytes per element and component); elsewhere both sizes agree
    n = 100001
    for op, w in ((A.OP_MUL, 1), (A.OP_LINREC, 2)):
        full = A.adpar_workspace_size(A.RULE_SCAN, op, A.F64, n)
        mini = A.adpar_workspace_size(A.RULE_SCAN | A.WS_MINIMAL, op, A.F64, n)
        assert full >= mini + 8 * w * n
    for op in (A.OP_ADD, A.OP_MUL, A.OP_MIN, A.OP_MAX, A.OP_LINREC):
        assert A.adpar_workspace_size(A.RULE_SCAN, op, A.F32, n) == A.adpar_workspace_size(
            A.RULE_SCAN | A.WS_MINIMAL, op, A.F32, n)
    for op in (A.OP_ADD, A.OP_MIN, A.OP_MAX):
        assert A.adpar_workspace_size(A.RULE_SCAN, op, A.F64, n) == A.adpar_workspace_size(
            A.RULE_SCAN | A.WS_MINIMAL, op, A.F64, n)
