"""GPU parity of the general reduce_by_index rule (Sec. 5.1.2: radix sort by
bin, forward and reverse segmented scans for l_i and r_i, then
d(l_i (.) a_i (.) r_i)/d a_i with hsbar[inds_i]) against the FP64 oracle's
plain tape sweep, through the C ABI.

Covers every operator (LINREC, which does not commute, keeps index order
inside a bin), FP32 and FP64, int32 and int64 indices, bin counts that take
one, two and three radix passes, uniform and Zipf bins with 1% of the
indices out of range, sizes spanning several sort rounds and scan tiles with
ragged tails, accumulation, empty inputs and bins, and the recomputed bins.

Tolerances (relative L2): FP32 1e-4, FP64 1e-12; min/max adjoints, which
are selections of hsbar, are compared exactly.
"""
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


def tol(dt):
    return 1e-12 if dt == np.float64 else 1e-4


@pytest.fixture(scope="module")
def A():
    from paper_2202_10297_gb300 import adpar
    adpar.lib()
    return adpar


@pytest.fixture(scope="module")
def O():
    from oracle import oracle
    return oracle


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def inputs(op, n, m, dt, it, dist, seed):
    g = synth.rng(seed)
    _, inds, _ = synth.hist(n, m, dist=dist, itype=it, seed=seed)
    b = hb = None
    if op == "linrec":
        a = g.uniform(0.9, 1.0, n).astype(dt)
        b = g.standard_normal(n).astype(dt)
        hb = g.standard_normal(m).astype(dt)
    elif op == "mul":
        a = g.uniform(0.97, 1.03, n).astype(dt)  # bin products stay in range
        if n > 50:
            a[g.choice(n, size=3, replace=False)] = 0
    elif op in ("min", "max"):
        a = (np.round(g.standard_normal(n) * 8) / 8).astype(dt)  # ties
    else:
        a = g.standard_normal(n).astype(dt)
    ha = g.standard_normal(m).astype(dt)
    return a, b, inds, ha, hb


def check(A, O, op, n, m, dt, it=np.int32, dist="uniform", seed=1, accumulate=False):
    a, b, inds, ha, hb = inputs(op, n, m, dt, it, dist, seed)
    w2 = op == "linrec"
    g = synth.rng(seed + 100)
    ab0 = g.standard_normal(n).astype(dt) if accumulate else None
    bb0 = g.standard_normal(n).astype(dt) if accumulate and w2 else None
    ab, bb, hsa, hsb = A.adpar_vjp_hist_general(
        op, dev(a), dev(inds), m, dev(ha), b=dev(b) if w2 else None, hsbar_b=dev(hb) if w2 else None,
        abar=dev(ab0) if accumulate else None, bbar=dev(bb0) if accumulate and w2 else None,
        want_hs=True, accumulate=accumulate)
    torch.cuda.synchronize()
    rab, rbb, rhsa, rhsb = O.hist_general_vjp(op, a, inds, m, ha, b=b, hsbar_b=hb, valsbar=ab0, bbar=bb0)
    ab = ab.cpu().numpy()
    if op in ("min", "max") or (op == "add" and not accumulate):
        np.testing.assert_array_equal(ab, rab.astype(dt))
    else:
        assert rel_l2(ab, rab) <= tol(dt), (op, n, m, rel_l2(ab, rab))
    if w2:
        assert rel_l2(bb.cpu().numpy(), rbb) <= tol(dt)
        assert rel_l2(hsb.cpu().numpy(), rhsb) <= tol(dt)
    hsa = hsa.cpu().numpy()
    if op in ("min", "max"):
        np.testing.assert_array_equal(hsa, rhsa.astype(dt))
    else:
        assert rel_l2(hsa, rhsa) <= tol(dt), (op, n, m, rel_l2(hsa, rhsa))


@pytest.mark.parametrize("dt", [np.float32, np.float64])
@pytest.mark.parametrize("op", ["add", "mul", "min", "max", "linrec"])
@pytest.mark.parametrize("n,m", [(1, 1), (7, 3), (2047, 5), (4096 + 3, 256), (20011, 300), (70001, 4096),
                                 (150001, 70000)])
def test_hist_general_matches_oracle(A, O, op, dt, n, m):
    check(A, O, op, n, m, dt, seed=n % 97 + m)


@pytest.mark.parametrize("op", ["add", "max", "linrec", "mul"])
@pytest.mark.parametrize("m", [256, 1 << 16])
def test_hist_general_zipf_int64(A, O, op, m):
    check(A, O, op, 300007, m, np.float32, it=np.int64, dist="zipf", seed=7)


@pytest.mark.parametrize("op", ["add", "min", "linrec"])
def test_hist_general_accumulates(A, O, op):
    check(A, O, op, 33333, 1000, np.float32, accumulate=True, seed=11)
    check(A, O, op, 5001, 17, np.float64, accumulate=True, seed=12)


def test_hist_general_matches_special_rules(A):
    """Through the C ABI, the general rule and the special rules of
    adpar_vjp_hist give the same max adjoint (exact) and + bins."""
    vals, inds, hsbar = synth.hist(200003, 4096, dist="zipf", seed=5)
    vt, it, ht = dev(vals), dev(inds), dev(hsbar)
    ab, _, hs, _ = A.adpar_vjp_hist_general("max", vt, it, 4096, ht, want_hs=True)
    sp = A.adpar_vjp_hist("max", it, 4096, ht, vals=vt, want_hs=True)
    assert torch.equal(ab, sp["valsbar"]) and torch.equal(hs, sp["hs"])
    ab, _, hs, _ = A.adpar_vjp_hist_general("add", vt, it, 4096, ht, want_hs=True)
    sp = A.adpar_vjp_hist("add", it, 4096, ht, vals=vt, want_hs=True)
    assert torch.equal(ab, sp["valsbar"])
    assert rel_l2(hs.cpu().numpy(), sp["hs"].cpu().numpy()) <= 1e-5


def test_hist_general_edges(A, O):
    # n = 0 with bins: hs is the neutral element everywhere
    e = torch.empty(0, device="cuda")
    ab, bb, hsa, hsb = A.adpar_vjp_hist_general("linrec", e, torch.empty(0, dtype=torch.int32, device="cuda"), 4,
                                                torch.ones(4, device="cuda"), b=e,
                                                hsbar_b=torch.ones(4, device="cuda"), want_hs=True)
    assert ab.numel() == 0 and hsa.tolist() == [1.0] * 4 and hsb.tolist() == [0.0] * 4
    # m = 0 and every index out of range: adjoints are 0 (or kept)
    a = torch.randn(5000, device="cuda")
    ab, _, _, _ = A.adpar_vjp_hist_general("mul", a, torch.full((5000,), 3, dtype=torch.int32, device="cuda"), 0,
                                           torch.empty(0, device="cuda"))
    assert torch.count_nonzero(ab).item() == 0
    keep = torch.randn(5000, device="cuda")
    ab, _, _, _ = A.adpar_vjp_hist_general("add", a, torch.full((5000,), -1, dtype=torch.int32, device="cuda"), 8,
                                           torch.ones(8, device="cuda"), abar=keep.clone(), accumulate=True)
    assert torch.equal(ab, keep)
    # all elements in one bin: the general reduce rule
    check(A, O, "linrec", 9000, 1, np.float64, seed=3)
    # one element per bin (every bin a segment of length one)
    n = 6000
    idx = np.random.default_rng(4).permutation(n).astype(np.int32)
    a = np.random.default_rng(5).uniform(0.9, 1.0, n).astype(np.float32)
    b = np.random.default_rng(6).standard_normal(n).astype(np.float32)
    ha = np.random.default_rng(7).standard_normal(n).astype(np.float32)
    hb = np.random.default_rng(8).standard_normal(n).astype(np.float32)
    ab, bb, hsa, hsb = A.adpar_vjp_hist_general("linrec", dev(a), dev(idx), n, dev(ha), b=dev(b), hsbar_b=dev(hb),
                                                want_hs=True)
    rab, rbb, rha, rhb = O.hist_general_vjp("linrec", a, idx, n, ha, b=b, hsbar_b=hb)
    assert rel_l2(ab.cpu().numpy(), rab) <= 1e-6 and rel_l2(bb.cpu().numpy(), rbb) <= 1e-6
    assert rel_l2(hsa.cpu().numpy(), rha) <= 1e-6 and rel_l2(hsb.cpu().numpy(), rhb) <= 1e-6


def test_hist_general_invalid_arguments(A):
    import ctypes as C
    L = A.lib()
    d = A.OpDesc(A.OP_LINREC, A.F32, 1)  # LINREC needs width 2
    assert L.adpar_vjp_hist_general(d, 10, 4, None, None, None, A.I32, None, None, None, None, None, None, 0,
                                    None, 0, None) == 1
    d = A.OpDesc(A.OP_ADD, A.F32, 1)
    assert L.adpar_vjp_hist_general(d, -1, 4, None, None, None, A.I32, None, None, None, None, None, None, 0,
                                    None, 0, None) == 1
    assert L.adpar_vjp_hist_general(d, 1 << 33, 4, None, None, None, A.I32, None, None, None, None, None, None, 0,
                                    None, 0, None) == 2
    a = torch.randn(100, device="cuda")
    i = torch.zeros(100, dtype=torch.int32, device="cuda")
    h = torch.ones(4, device="cuda")
    # workspace missing
    assert L.adpar_vjp_hist_general(d, 100, 4, C.c_void_p(a.data_ptr()), None, C.c_void_p(i.data_ptr()), A.I32,
                                    C.c_void_p(h.data_ptr()), None, C.c_void_p(a.data_ptr()), None, None, None, 0,
                                    None, 0, None) == 4


def test_hist_general_full_size_linrec(A, O):
    """The benchmark's LINREC case (n = 2^26 FP32 into m = 2^16 bins,
    Zipf, 1% out of range) against the oracle on every output."""
    n, m = 1 << 26, 1 << 16
    check(A, O, "linrec", n, m, np.float32, dist="zipf", seed=synth.SEED_BASE + 6)
