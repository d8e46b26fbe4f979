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
    # the full scan workspace of FP64 MUL holds the factored forward result
    # (8 bytes per element), that of the linear recurrence the carries of
    # its runs (3 elements per run of 16 FP64 / 32 FP32 elements); elsewhere
    # both sizes agree
    n = 100001
    full = A.adpar_workspace_size(A.RULE_SCAN, A.OP_MUL, A.F64, n)
    mini = A.adpar_workspace_size(A.RULE_SCAN | A.WS_MINIMAL, A.OP_MUL, A.F64, n)
    assert full >= mini + 8 * n
    for dt, run, es in ((A.F64, 16, 8), (A.F32, 32, 4)):
        full = A.adpar_workspace_size(A.RULE_SCAN, A.OP_LINREC, dt, n)
        mini = A.adpar_workspace_size(A.RULE_SCAN | A.WS_MINIMAL, A.OP_LINREC, dt, n)
        assert full >= 3 * es * (n // run) and full < mini + es * n
    for op in (A.OP_ADD, A.OP_MUL, A.OP_MIN, A.OP_MAX):
        assert A.adpar_workspace_size(A.RULE_SCAN, op, A.F32, n) == A.adpar_workspace_size(
            A.RULE_SCAN | A.WS_MINIMAL, op, A.F32, n)
    for op in (A.OP_ADD, A.OP_MIN, A.OP_MAX):
        assert A.adpar_workspace_size(A.RULE_SCAN, op, A.F64, n) == A.adpar_workspace_size(
            A.RULE_SCAN | A.WS_MINIMAL, op, A.F64, n)


def test_new_rules_validate_and_size_without_gpu():
    """The general reduce_by_index rule and the wide-element scan refuse bad
    arguments and a missing workspace before any CUDA call; their workspace
    sizes are host arithmetic (two sort buffers plus one destination record
    per radix pass; the full d x d lin_o's slots)."""
    from paper_2202_10297_gb300 import adpar as A
    L = A.lib()
    V = None
    # general reduce_by_index: LINREC needs width 2; negative sizes; too many elements; no workspace
    d = A.OpDesc(A.OP_LINREC, A.F32, 1)
    assert L.adpar_vjp_hist_general(d, 10, 4, V, V, V, A.I32, V, V, V, V, V, V, 0, V, 0, V) == 1
    d = A.OpDesc(A.OP_ADD, A.F32, 1)
    assert L.adpar_vjp_hist_general(d, 10, -1, V, V, V, A.I32, V, V, V, V, V, V, 0, V, 0, V) == 1
    assert L.adpar_vjp_hist_general(d, 1 << 33, 4, V, V, V, A.I32, V, V, V, V, V, V, 0, V, 0, V) == 2
    assert L.adpar_vjp_hist_general(d, 10, 4, 0x1000, V, 0x2000, A.I32, 0x3000, V, 0x4000, V, V, V, 0, V, 0,
                                    V) == 4
    assert L.adpar_vjp_hist_general(d, 10, 4, 0x1000, V, 0x2000, A.I32, 0x3000, V, 0x4000, V, V, V, 0x2, V, 0,
                                    V) == 2  # unknown flag
    n = 1 << 20
    small = A.adpar_workspace_size(A.RULE_HIST_GENERAL, A.OP_ADD, A.F32, n, 256)
    wide_m = A.adpar_workspace_size(A.RULE_HIST_GENERAL, A.OP_ADD, A.F32, n, 1 << 22)
    pair = A.adpar_workspace_size(A.RULE_HIST_GENERAL, A.OP_LINREC, A.F64, n, 256)
    assert small >= 2 * 8 * n + 4 * n          # keys and values twice, one pass of destinations
    assert wide_m - small >= 2 * 4 * n         # three passes instead of one
    assert pair >= 2 * (4 + 16) * n + 4 * n    # FP64 pairs travel with the keys
    # wide-element scan: MATREC2 is width 6; MAX is not a wide operator; unknown flag; misaligned; no workspace
    assert L.adpar_vjp_scan_wide(A.OpDesc(A.OP_MATREC2, A.F32, 2), 4, V, V, V, V, 0, V, 0, V) == 1
    assert L.adpar_vjp_scan_wide(A.OpDesc(A.OP_MAX, A.F32, 1), 4, V, V, V, V, 0, V, 0, V) == 1
    d = A.OpDesc(A.OP_MATREC2, A.F32, 6)
    assert L.adpar_vjp_scan_wide(d, 4, 0x1000, 0x2000, 0x3000, V, 0x2, V, 0, V) == 2
    assert L.adpar_vjp_scan_wide(d, 4, 0x1004, 0x2000, 0x3000, V, 0, V, 0, V) == 3
    assert L.adpar_vjp_scan_wide(d, 4, 0x1000, 0x2000, 0x3000, V, A.FULL_LIN_O, V, 0, V) == 4
    w6 = A.adpar_workspace_size(A.RULE_SCAN_WIDE, A.OP_MATREC2, A.F32, n, 0, width=6)
    w2 = A.adpar_workspace_size(A.RULE_SCAN_WIDE, A.OP_LINREC, A.F32, n, 0, width=2)
    assert w6 > w2 > 0


def test_older_entry_points_validate_without_gpu(lib):
    """reduce, reduce_by_index, scatter, map-accumulator and k-means refuse bad
    arguments before any CUDA call (C status codes, no GPU needed)."""
    from paper_2202_10297_gb300 import adpar as A
    C = ctypes
    VP, I64 = C.c_void_p, C.c_int64
    lib.adpar_vjp_reduce.argtypes = [A.OpDesc, I64] + [VP] * 7 + [C.c_uint32, VP, C.c_size_t, VP]
    lib.adpar_vjp_reduce.restype = C.c_int
    V = None
    # LINREC has no special reduce rule; width must be 1; log domain is for * only
    assert lib.adpar_vjp_reduce(A.OpDesc(A.OP_LINREC, A.F32, 2), 8, V, V, V, V, V, V, V, 0, V, 0, V) == 1
    assert lib.adpar_vjp_reduce(A.OpDesc(A.OP_ADD, A.F32, 2), 8, V, V, V, V, V, V, V, 0, V, 0, V) == 1
    assert lib.adpar_vjp_reduce(A.OpDesc(A.OP_ADD, A.F32, 1), 8, V, 0x1000, 0x2000, V, V, V, V, A.PROD_LOGDOMAIN,
                                V, 0, V) == 2
    assert lib.adpar_vjp_reduce(A.OpDesc(A.OP_MAX, A.F32, 1), 8, 0x1004, 0x1000, 0x2000, V, V, V, V, 0,
                                V, 0, V) == 3
    lib.adpar_vjp_scatter.argtypes = [C.c_int, I64, I64, VP, C.c_int, VP, VP, VP, VP, C.c_uint32, VP]
    lib.adpar_vjp_scatter.restype = C.c_int
    assert lib.adpar_vjp_scatter(7, 10, 4, V, A.I32, V, V, V, V, 0, V) == 1          # bad dtype
    assert lib.adpar_vjp_scatter(A.F32, 10, 4, V, 9, V, V, V, V, 0, V) == 1          # bad itype
    assert lib.adpar_vjp_scatter(A.F32, -1, 4, V, A.I32, V, V, V, V, 0, V) == 1      # negative size
    lib.adpar_vjp_map_acc.argtypes = [C.c_int, C.c_int, I64, I64, C.c_int, VP, VP, C.c_int, VP, VP, VP, VP,
                                      C.c_uint32, VP, C.c_size_t, VP]
    lib.adpar_vjp_map_acc.restype = C.c_int
    assert lib.adpar_vjp_map_acc(9, A.F32, 10, 4, 1, V, V, A.I32, V, V, V, V, 0, V, 0, V) == 1   # bad g
    assert lib.adpar_vjp_map_acc(A.G_GATHER, A.F32, 10, 4, 3, V, V, A.I32, V, V, V, V, 0, V, 0, V) == 1  # width
    lib.adpar_kmeans_vjp.argtypes = [I64, C.c_int, C.c_int] + [VP] * 6 + [C.c_uint32, VP, C.c_size_t, VP]
    lib.adpar_kmeans_vjp.restype = C.c_int
    assert lib.adpar_kmeans_vjp(100, 32, 48, V, V, V, V, V, V, 0, V, 0, V) == 2   # k not a multiple of 32
    assert lib.adpar_kmeans_vjp(100, 16, 64, V, V, V, V, V, V, 0, V, 0, V) == 2   # d != 32
    assert lib.adpar_kmeans_vjp(100, 32, 64, V, V, V, V, V, V, 0, V, 0, V) == 1   # X, C missing
    lib.adpar_kmeans_hessdiag.argtypes = [C.c_int, VP, VP, C.c_size_t, VP, C.c_uint32, VP]
    lib.adpar_kmeans_hessdiag.restype = C.c_int
    assert lib.adpar_kmeans_hessdiag(64, V, V, 0, V, 0, V) == 1                    # ybar, Hdiag missing
    assert lib.adpar_kmeans_hessdiag(48, 0x1000, V, 0, 0x2000, 0, V) == 2          # k not a multiple of 32
    assert lib.adpar_kmeans_hessdiag(64, 0x1000, V, 0, 0x2000, 0, V) == 4          # workspace missing


def test_noalloc_binding_checks_every_array_without_gpu():
    """The allocation-free scan VJP reads and writes n elements of every array
    it is given, n taken from ybar_a: an array of another length or dtype
    would be overrun on the device, so the binding refuses it on the host."""
    import torch
    from paper_2202_10297_gb300 import adpar as A
    n = 64
    f64 = lambda k=n: torch.zeros(k, dtype=torch.float64)  # noqa: E731
    with pytest.raises(ValueError, match="abar"):
        A.adpar_vjp_scan_noalloc("linrec", f64(), f64(), b=f64(), ybar_b=f64(), abar=f64(n - 1), bbar=f64())
    with pytest.raises(ValueError, match="bbar"):
        A.adpar_vjp_scan_noalloc("linrec", f64(), f64(), b=f64(), ybar_b=f64(), abar=f64(),
                                 bbar=torch.zeros(n, dtype=torch.float32))
    with pytest.raises(ValueError, match="ys_b"):
        A.adpar_vjp_scan_noalloc("linrec", f64(), f64(), b=f64(), ybar_b=f64(), abar=f64(), bbar=f64(),
                                 ys_a=f64(), ys_b=f64(2 * n))
    # right shapes, but host tensors: refused before the library is called
    with pytest.raises(ValueError, match="CUDA"):
        A.adpar_vjp_scan_noalloc("add", None, f64(), abar=f64())
    # the status reader checks its output pointer before any CUDA call
    assert A.lib().adpar_noalloc_status(None, None) == A.ERR_INVALID


def test_forward_mode_entry_points_validate_without_gpu():
    """The forward-mode entry points refuse bad arguments on the host, before
    any CUDA call, and size their workspaces."""
    from paper_2202_10297_gb300 import adpar as A
    L = A.lib()
    d = A.OpDesc(A.OP_MUL, A.F64, 1)
    assert L.adpar_jvp_reduce(d, -1, None, None, None, None, None, None, 0, None) == A.ERR_INVALID
    assert L.adpar_jvp_reduce(A.OpDesc(A.OP_LINREC, A.F64, 2), 4, None, None, None, None, None, None, 0,
                              None) == A.ERR_INVALID
    assert L.adpar_jvp_reduce(d, 4, 0x1000, 0x2000, None, None, None, None, 0, None) == A.ERR_INVALID  # no ydot
    assert L.adpar_jvp_reduce(d, 4, 0x1004, 0x2000, None, 0x3000, None, None, 0, None) == 3  # misaligned
    assert L.adpar_jvp_reduce(d, 4, 0x1000, 0x2000, None, 0x3000, None, None, 0, None) == 4  # no workspace
    dh = A.OpDesc(A.OP_ADD, A.F32, 1)
    assert L.adpar_jvp_hist(dh, 10, 4, 0x1000, 0x2000, 0x3000, 0, None, 0x4000, 0x5000, None, 0,
                            None) == 2  # log-domain tangents are for * only
    assert L.adpar_jvp_hist(dh, 10, 4, 0x1000, 0x2000, 0x3000, 7, None, 0x4000, None, None, 0,
                            None) == A.ERR_INVALID  # bad index type
    assert L.adpar_jvp_map_acc(A.G_GATHER, A.F32, 10, 4, 2, None, 0x1000, 0, None, 0x2000, None, 0x3000,
                               None) == A.ERR_INVALID  # width 2 for a scalar g
    assert L.adpar_jvp_map_acc(A.G_SCALE, A.F32, 10, 4, 1, 0x1000, 0x2000, 0, None, 0x3000, None, 0x4000,
                               None) == A.ERR_INVALID  # scale without ws
    assert L.adpar_kmeans_fwd_rev(100, 16, 64, None, None, None, None, None, None, 0, None, 0,
                                  None) == A.ERR_INVALID  # d must be 32
    for op in (A.OP_ADD, A.OP_MUL, A.OP_MIN, A.OP_MAX):
        assert A.adpar_workspace_size(A.RULE_JVP_REDUCE, op, A.F32, 1000) >= A.adpar_workspace_size(
            A.RULE_REDUCE, op, A.F32, 1000)
        assert A.adpar_workspace_size(A.RULE_JVP_HIST, op, A.F64, 1000, 300) >= A.adpar_workspace_size(
            A.RULE_HIST, op, A.F64, 1000, 300) + 300 * 8
    assert A.adpar_workspace_size(A.RULE_KMEANS_FWD_REV, 0, A.F32, 1 << 20, 256) >= 4 << 20
