"""The allocation-free scan VJP entry point (adpar_vjp_scan_noalloc).

It serves callers that cannot allocate device memory where they need a
gradient (an allocator hook that must not re-enter itself, a loop that
forbids allocation after start-up).  Its scratch is a static device array
inside the library, so these tests check that it gives what the ordinary
entry point with a caller workspace gives, on calls in a row (a call must
not be disturbed by what the one before left in the shared array), that a
call takes no device memory, that a timed-out device wait is visible through
adpar_noalloc_status, and that sizes beyond the array are refused on the host.

This file sorts last so that a run stopping at the first failure has run
every other test before it; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2202_10297_gb300 import synth

pytestmark = pytest.mark.gpu


def rel_l2(x, ref):
    x = np.asarray(x, np.float64)
    ref = np.asarray(ref, np.float64)
    d = np.linalg.norm(ref)
    return float(np.linalg.norm(x - ref) / (d if d > 0 else 1.0))


@pytest.fixture(scope="module")
def A():
    from paper_2202_10297_gb300 import adpar
    adpar.lib()
    return adpar


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def test_noalloc_matches_workspace_entry_two_calls(A):
    # call 1: linear-recurrence scan VJP, FP32, several tiles and a ragged tail
    n1 = 300007
    a, b, ya, yb = synth.linrec(n1, np.float32, seed=31)
    ab_ref, bb_ref, _ = A.adpar_vjp_scan("linrec", dev(a), dev(ya), b=dev(b), ybar_b=dev(yb))
    ab = torch.empty(n1, dtype=torch.float32, device="cuda")
    bb = torch.empty_like(ab)
    A.adpar_vjp_scan_noalloc("linrec", dev(a), dev(ya), b=dev(b), ybar_b=dev(yb), abar=ab, bbar=bb)
    torch.cuda.synchronize()
    assert rel_l2(ab.cpu().numpy(), ab_ref.cpu().numpy()) < 1e-4
    assert rel_l2(bb.cpu().numpy(), bb_ref.cpu().numpy()) < 1e-4

    # call 2, right after: a max scan VJP in FP64 of a different length, on
    # the scratch the first call left behind
    n2 = 123457
    g = synth.rng(32)
    x = (np.round(g.standard_normal(n2) * 8) / 8).astype(np.float64)
    y = g.standard_normal(n2)
    ref, _, _ = A.adpar_vjp_scan("max", dev(x), dev(y))
    out = torch.empty(n2, dtype=torch.float64, device="cuda")
    A.adpar_vjp_scan_noalloc("max", dev(x), dev(y), abar=out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    r = ref.cpu().numpy()
    assert rel_l2(got, r) < 1e-12
    np.testing.assert_array_equal(got != 0, r != 0)

    # call 3: FP64 linear recurrence at a size whose factored forward result
    # fits the static array (the path that keeps per-tile results there),
    # accumulating into adjoints that already hold values
    n3 = 1 << 16
    assert A.adpar_workspace_size(A.RULE_SCAN, A.OP_LINREC, A.F64, n3) <= A.adpar_noalloc_scratch_bytes()
    a3, b3, ya3, yb3 = synth.linrec(n3, np.float64, seed=33)
    g3 = synth.rng(34)
    ab0 = g3.standard_normal(n3)
    bb0 = g3.standard_normal(n3)
    ab_ref = dev(ab0)
    bb_ref = dev(bb0)
    A.adpar_vjp_scan("linrec", dev(a3), dev(ya3), b=dev(b3), ybar_b=dev(yb3), abar=ab_ref, bbar=bb_ref,
                     accumulate=True)
    ab3 = dev(ab0)
    bb3 = dev(bb0)
    A.adpar_vjp_scan_noalloc("linrec", dev(a3), dev(ya3), b=dev(b3), ybar_b=dev(yb3), abar=ab3, bbar=bb3,
                             accumulate=True)
    assert A.adpar_noalloc_status() == A.OK
    assert rel_l2(ab3.cpu().numpy(), ab_ref.cpu().numpy()) < 1e-12
    assert rel_l2(bb3.cpu().numpy(), bb_ref.cpu().numpy()) < 1e-12

    # call 4: + scan VJP in FP32 over many TMA tiles of 16384 elements and a
    # ragged one, overwriting, then accumulating
    n4 = 200 * 16384 + 9
    y4 = synth.normal(n4, np.float32, seed=36)
    ref4, _, _ = A.adpar_vjp_scan("add", None, dev(y4))
    out4 = torch.empty(n4, dtype=torch.float32, device="cuda")
    A.adpar_vjp_scan_noalloc("add", None, dev(y4), abar=out4)
    torch.cuda.synchronize()
    assert A.adpar_noalloc_status() == A.OK
    assert rel_l2(out4.cpu().numpy(), ref4.cpu().numpy()) < 1e-5
    A.adpar_vjp_scan_noalloc("add", None, dev(y4), abar=out4, accumulate=True)
    torch.cuda.synchronize()
    assert A.adpar_noalloc_status() == A.OK
    assert rel_l2(out4.cpu().numpy(), 2 * ref4.cpu().numpy()) < 1e-5


def test_noalloc_call_takes_no_device_memory(A):
    # inputs and outputs first; one warm-up call loads every kernel the call uses
    n = 1 << 16
    a, b, ya, yb = synth.linrec(n, np.float64, seed=35)
    a, b, ya, yb = dev(a), dev(b), dev(ya), dev(yb)
    ab = torch.empty_like(a)
    bb = torch.empty_like(a)
    A.adpar_vjp_scan_noalloc("linrec", a, ya, b=b, ybar_b=yb, abar=ab, bbar=bb)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        A.adpar_vjp_scan_noalloc("linrec", a, ya, b=b, ybar_b=yb, abar=ab, bbar=bb)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_status_reports_a_timed_out_wait(A):
    # a bounded wait on a flag that nothing sets, run in the static array,
    # gives up and leaves ADPAR_ERR_TIMEOUT in its status word ...
    A.adpar_noalloc_selftest_timeout()
    assert A.adpar_noalloc_status() == A.ERR_TIMEOUT
    # ... which the next call clears; the context and the array still serve
    n = 50001
    x = synth.normal(n, np.float32, seed=36)
    y = synth.normal(n, np.float32, seed=37)
    ref, _, _ = A.adpar_vjp_scan("max", dev(x), dev(y))
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    A.adpar_vjp_scan_noalloc("max", dev(x), dev(y), abar=out)
    assert A.adpar_noalloc_status() == A.OK
    assert rel_l2(out.cpu().numpy(), ref.cpu().numpy()) < 1e-4


def test_noalloc_refuses_sizes_beyond_static_scratch(A):
    L = A.lib()
    assert A.adpar_noalloc_scratch_bytes() == 8 << 20
    d = A.OpDesc(A.OP_ADD, A.F32, 1)
    # a 2^34-element scan needs far more than 8 MiB of look-back state; the
    # size check refuses it on the host before any pointer is read
    st = L.adpar_vjp_scan_noalloc(d, 1 << 34, None, None, None, None, None, None, None, None, 0, None)
    assert st == A.ERR_TOO_LARGE
    assert "static" in A.status_string(st)
    # the largest benchmark-size scans fit
    for op, dt, n in ((A.OP_ADD, A.F32, 1 << 28), (A.OP_MAX, A.F32, 1 << 28),
                      (A.OP_LINREC, A.F64, 1 << 26), (A.OP_LINREC, A.F32, 1 << 26)):
        assert A.adpar_workspace_size(A.RULE_SCAN | A.WS_MINIMAL, op, dt, n) <= A.adpar_noalloc_scratch_bytes()
