"""GPU parity of the forward-mode (JVP) rules of reduce, reduce_by_index,
scatter and map with a free array, and of the k-means forward-over-reverse
path, against the FP64 oracle's dual-number sweeps, through the C ABI.

Index decisions are exact: the tangent of a min/max (of a reduce or of a
bin) is the tangent at the lowest-index extremum, compared bit-exactly with
forced ties; scatter and gather tangents are data movement, bit-exact.
Values: relative error 1e-4 (FP32) / 1e-12 (FP64); long products in the log
domain (ln|tangent| within 1e-10, sign exact).  Also forward-mode gradcheck
of the autograd wrappers.
"""
import numpy as np
import pytest
import torch

from paper_2202_10297_gb300 import synth

pytestmark = pytest.mark.gpu

SIZES = [1, 7, 1000, 4097, 100003, (1 << 20) + 7]
DTS = [np.float32, np.float64]


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


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


# ---------------------------------------------------------------- reduce
@pytest.mark.parametrize("dt", DTS)
@pytest.mark.parametrize("op", ["add", "min", "max"])
@pytest.mark.parametrize("n", SIZES)
def test_jvp_reduce_vs_oracle(A, oracle, op, dt, n):
    g = synth.rng(n + len(op))
    a = g.standard_normal(n)
    if op != "add":
        a = np.round(a * 8) / 8  # ties: the lowest index keeps the tangent
    a = a.astype(dt)
    ad = g.standard_normal(n).astype(dt)
    out = A.adpar_jvp_reduce(op, dev(a), dev(ad), want_y=True)
    y, yd = oracle.reduce_jvp(op, a, ad)
    got = float(out["ydot"].item())
    if op == "add":
        # FP64 accumulation on the GPU: the output's rounding dominates
        assert abs(got - yd) <= (1e-6 if dt == np.float32 else 1e-13) * np.abs(ad).astype(np.float64).sum()
        assert abs(float(out["y"].item()) - y) <= 1e-5 * np.abs(a).astype(np.float64).sum()
    else:
        assert got == yd and float(out["y"].item()) == y  # bit-exact


@pytest.mark.parametrize("dt", DTS)
@pytest.mark.parametrize("nz", [0, 1, 2])
@pytest.mark.parametrize("n", [1, 5, 600, 65536, 300007])
def test_jvp_prod_reduce_vs_oracle(A, oracle, dt, nz, n):
    a, _ = synth.prod_reduce(n, min(nz, n), dtype=dt, seed=n + 7 * nz)
    ad = synth.normal(n, dt, seed=n + 11)
    out = A.adpar_jvp_reduce("mul", dev(a), dev(ad), want_aux=True)
    ref = oracle.prod_reduce_jvp(a, ad)
    aux = out["aux"]
    assert int(aux["sign"]) == ref["sign"]
    if ref["sign"] != 0:
        assert abs(float(aux["log_abs"]) - ref["log"]) <= 1e-10 * max(1.0, abs(ref["log"]))
    got = float(out["ydot"].item())
    refv = float(np.asarray(ref["ydot"]).astype(dt))  # the oracle's value rounded to the output type
    tiny = np.finfo(dt).smallest_subnormal
    assert abs(got - refv) <= tol(dt) * abs(refv) + 2 * tiny


# ------------------------------------------------------- reduce_by_index
HCASES = [(1000, 7, "uniform"), (100003, 256, "zipf"), (200001, 1 << 16, "uniform"), (300007, 20000, "zipf")]


@pytest.mark.parametrize("n,m,dist", HCASES)
@pytest.mark.parametrize("op", ["add", "min", "max"])
@pytest.mark.parametrize("dt", DTS)
@pytest.mark.parametrize("itype", [np.int32, np.int64])
def test_jvp_hist_vs_oracle(A, oracle, n, m, dist, op, dt, itype):
    vals, inds, _ = synth.hist(n, m, dist, itype=itype, seed=n + m)
    if op != "add":
        vals = np.round(vals * 4) / 4  # forced ties inside bins
    vals = vals.astype(dt)
    vd = synth.normal(n, dt, seed=n + 1)
    out = A.adpar_jvp_hist(op, dev(vals), dev(vd), dev(inds), m, want_hs=True)
    hs, hd = oracle.hist_jvp(op, vals, vd, inds, m)
    got = out["hsdot"].cpu().numpy()
    if op == "add":
        assert rel_l2(got, hd) < (1e-5 if dt == np.float32 else 1e-12)
        assert rel_l2(out["hs"].cpu().numpy(), hs) < (1e-5 if dt == np.float32 else 1e-12)
    else:
        np.testing.assert_array_equal(got.astype(np.float64), hd)  # the tangent at the bin's first extremum
        used = np.isfinite(hs)
        np.testing.assert_array_equal(out["hs"].cpu().numpy().astype(np.float64)[used], hs[used])


@pytest.mark.parametrize("n,m,dist", HCASES)
@pytest.mark.parametrize("dt", DTS)
def test_jvp_hist_prod_vs_oracle(A, oracle, n, m, dist, dt):
    vals, inds, _ = synth.hist(n, m, dist, seed=n + 3 * m)
    g = synth.rng(n)
    vals = g.uniform(0.5, 1.5, n) * np.sign(vals)
    for b, k in ((1, 1), (2, 2), (3, 1)):  # bins with one and two zeros
        members = np.flatnonzero(inds == b)
        vals[members[:k]] = 0
    vals = vals.astype(dt)
    vd = synth.normal(n, dt, seed=n + 5)
    out = A.adpar_jvp_hist("mul", dev(vals), dev(vd), dev(inds), m, want_aux=True)
    ref = oracle.hist_prod_jvp(vals, vd, inds, m)
    aux = out["aux"]
    np.testing.assert_array_equal(aux["sign"], ref["sign"])
    nzb = ref["sign"] != 0
    err = np.abs(aux["log_abs"][nzb] - ref["log"][nzb]) / np.maximum(1.0, np.abs(ref["log"][nzb]))
    assert err.max(initial=0.0) < 1e-10
    got = out["hsdot"].cpu().numpy().astype(np.float64)
    refv = ref["hsdot"].astype(dt).astype(np.float64)
    tiny = np.finfo(dt).smallest_subnormal
    assert np.linalg.norm(got - refv) <= tol(dt) * np.linalg.norm(refv) + 2 * tiny * np.sqrt(m)


# --------------------------------------------------------------- scatter
@pytest.mark.parametrize("dt", DTS)
@pytest.mark.parametrize("sort", [False, True])
def test_jvp_scatter_vs_oracle(A, oracle, dt, sort):
    n, m = 1 << 20, 1 << 18
    is_, _, _ = synth.scatter(n, m, sort=sort, seed=21)
    xd = synth.normal(n, dt, seed=22)
    vd = synth.normal(m, dt, seed=23)
    yd = dev(xd)
    A.adpar_jvp_scatter(dev(is_), dev(vd), yd)
    ref = oracle.scatter_jvp(n, is_, vd, xd)
    np.testing.assert_array_equal(yd.cpu().numpy().astype(np.float64), ref)


# ---------------------------------------------------------------- map_acc
@pytest.mark.parametrize("dt", DTS)
@pytest.mark.parametrize("gname,na,width", [("gather", 4096, 1), ("scale", 1 << 16, 1), ("sqdist_row", 256, 32)])
def test_jvp_map_acc_vs_oracle(A, oracle, dt, gname, na, width):
    nj = 200003 if width == 1 else 20011
    g = synth.rng(na + width)
    as_ = g.standard_normal(na * width).astype(dt)
    is_ = g.integers(-3, na + 3, size=nj).astype(np.int32)  # a few out of range
    ws = g.standard_normal(nj * width).astype(dt)
    asd = g.standard_normal(na * width).astype(dt)
    wsd = g.standard_normal(nj * width).astype(dt) if gname != "gather" else None
    got = A.adpar_jvp_map_acc(gname, dev(as_), dev(is_), dev(asd), ws=dev(ws) if gname != "gather" else None,
                              wsdot=None if wsd is None else dev(wsd), width=width).cpu().numpy()
    ref = oracle.map_acc_jvp(gname, as_, is_, asd, ws=ws, wsdot=wsd, width=width)
    if gname == "gather":
        np.testing.assert_array_equal(got.astype(np.float64), ref)
    else:
        assert rel_l2(got, ref) < tol(dt)
    oor = (is_ < 0) | (is_ >= na)
    assert np.all(got[oor] == 0)


# ------------------------------------------------ k-means forward over reverse
def test_kmeans_fwd_rev_vs_oracle(A, oracle):
    N, d, k = 1 << 15, 32, 256
    X, Cm = synth.kmeans(N, d, k, seed=31)
    Cd = synth.normal(k * d, np.float32, seed=32).reshape(k, d)
    ydot, Gd = A.adpar_kmeans_fwd_rev(dev(X), dev(Cm), dev(Cd), ybar=0.75)
    rydot, rGd = oracle.kmeans_fwd_rev(X, Cm, Cd, 0.75)
    assert rel_l2(Gd.cpu().numpy(), rGd) < 1e-5
    assert abs(float(ydot.item()) - rydot) <= 1e-4 * abs(rydot)


def test_kmeans_hessdiag_by_fwd_rev_full_size(A):
    """At the benchmark size (N = 2^20, d = 32, k = 256) the Hessian diagonal
    by forward over reverse equals the closed form 2 ybar cnt_k."""
    N, d, k = 1 << 20, 32, 256
    X, Cm = synth.kmeans(N, d, k)
    Xt, Ct = dev(X), dev(Cm)
    H = A.adpar_kmeans_hessdiag_fwd_rev(Xt, Ct, ybar=1.0)
    yb = torch.ones(1, device="cuda")
    out = A.adpar_kmeans_vjp(Xt, Ct, ybar=yb, want_argmin=True)
    Hc = torch.empty_like(Ct)
    A.adpar_kmeans_hessdiag(k, yb, out["work"], Hdiag=Hc)
    cnt = np.bincount(out["argmin"].cpu().numpy(), minlength=k)
    np.testing.assert_allclose(H.cpu().numpy(), 2.0 * cnt[:, None] * np.ones((1, d)), rtol=1e-6)
    np.testing.assert_allclose(H.cpu().numpy(), Hc.cpu().numpy(), rtol=1e-6)


# ------------------------------------------------------- autograd, forward AD
@pytest.fixture(scope="module")
def AG():
    from paper_2202_10297_gb300 import adpar, autograd
    adpar.lib()
    return autograd


def _gc(fn, inputs):
    return torch.autograd.gradcheck(fn, inputs, eps=1e-6, atol=1e-7, rtol=1e-6, check_forward_ad=True,
                                    check_backward_ad=True, check_undefined_grad=False, check_batched_grad=False)


@pytest.mark.parametrize("op", ["add", "mul", "min", "max"])
def test_forward_ad_reduce_gradcheck(AG, op):
    g = synth.rng(41)
    a = torch.from_numpy(g.uniform(0.5, 1.5, 37) * np.sign(g.standard_normal(37))).cuda().requires_grad_()
    assert _gc(lambda x: AG.reduce(op, x), (a,))


@pytest.mark.parametrize("op", ["add", "mul", "min", "max"])
def test_forward_ad_reduce_by_index_gradcheck(AG, op):
    g = synth.rng(42)
    n, m = 60, 5
    v = torch.from_numpy(g.uniform(0.5, 1.5, n) * np.sign(g.standard_normal(n))).cuda().requires_grad_()
    ix = torch.from_numpy(g.integers(-1, m + 1, size=n).astype(np.int32)).cuda()
    assert _gc(lambda x: AG.reduce_by_index(op, x, ix, m), (v,))


def test_forward_ad_scatter_gradcheck(AG):
    g = synth.rng(43)
    n, m = 40, 12
    xs = torch.from_numpy(g.standard_normal(n)).cuda().requires_grad_()
    vs = torch.from_numpy(g.standard_normal(m)).cuda().requires_grad_()
    is_ = torch.from_numpy(g.permutation(n)[:m].astype(np.int32)).cuda()
    assert _gc(lambda x, v: AG.scatter(x, is_, v), (xs, vs))


@pytest.mark.parametrize("gname,width", [("gather", 1), ("scale", 1), ("sqdist_row", 4)])
def test_forward_ad_map_acc_gradcheck(AG, gname, width):
    g = synth.rng(44)
    na, nj = 6, 25
    as_ = torch.from_numpy(g.standard_normal(na * width)).cuda().requires_grad_()
    is_ = torch.from_numpy(g.integers(0, na, size=nj).astype(np.int32)).cuda()
    if gname == "gather":
        assert _gc(lambda a: AG.map_acc(gname, a, is_, width=width), (as_,))
    else:
        ws = torch.from_numpy(g.standard_normal(nj * width)).cuda().requires_grad_()
        assert _gc(lambda a, w: AG.map_acc(gname, a, is_, ws=w, width=width), (as_, ws))


def test_forward_ad_kmeans_loss_and_hvp(AG, oracle):
    """The k-means loss in forward mode (dual tensors in C) and the
    Hessian-vector product by forward over reverse, against the oracle."""
    import torch.autograd.forward_ad as fwAD
    N, d, k = 4096, 32, 64
    X, Cm = synth.kmeans(N, d, k, seed=45)
    Cd = synth.normal(k * d, np.float32, seed=46).reshape(k, d)
    Xt, Ct, Cdt = dev(X), dev(Cm), dev(Cd)
    with fwAD.dual_level():
        loss = AG.kmeans_loss(Xt, fwAD.make_dual(Ct, Cdt))
        ydot = fwAD.unpack_dual(loss).tangent
    rydot, rGd = oracle.kmeans_fwd_rev(X, Cm, Cd, 1.0)
    assert abs(float(ydot.item()) - rydot) <= 1e-4 * abs(rydot)
    assert rel_l2(AG.kmeans_hvp(Xt, Ct, Cdt).cpu().numpy(), rGd) < 1e-5
