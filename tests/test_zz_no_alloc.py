"""The allocation-free scan VJP entry point (adpar_vjp_scan_noalloc).

It serves callers that cannot allocate device memory where they need a
gradient (an allocator hook that must not re-enter itself, a loop that
forbids allocation after start-up).  Its scratch is a static device array
inside the library, so these tests check that it gives what the ordinary
entry point with a caller workspace gives, on two calls in a row (the
second call must not be disturbed by what the first left in the shared
array), and that sizes beyond the array are refused on the host.

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
