"""GPU parity of reduce_by_index (Sec. 5.1.2), scatter (Sec. 5.3) and map with
accumulators (Sec. 5.4) against the FP64 oracle, through the C ABI.

Bin indices (argidx), zero counts and lowest zero indices are compared
bit-exactly; values within 1e-4 (FP32) / 1e-12 (FP64) relative L2.
Scatter is pure data movement and is compared bit-exactly.
"""
import math

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


CASES = [(1000, 7, "uniform"), (100003, 256, "uniform"), (100003, 256, "zipf"),
         (200001, 1 << 16, "uniform"), (200001, 1 << 16, "zipf"), (300007, 20000, "zipf")]


@pytest.mark.parametrize("n,m,dist", CASES)
@pytest.mark.parametrize("itype", [np.int32, np.int64])
def test_hist_add(A, oracle, n, m, dist, itype):
    vals, inds, hsbar = synth.hist(n, m, dist, itype=itype, seed=n + m)
    out = A.adpar_vjp_hist("add", dev(inds), m, dev(hsbar), vals=dev(vals), want_hs=True)
    vb, hs, _ = oracle.hist_vjp("add", vals, inds, m, hsbar)
    np.testing.assert_array_equal(out["valsbar"].cpu().numpy(), vb)  # a gather: exact
    assert rel_l2(out["hs"].cpu().numpy(), hs) < 1e-5


@pytest.mark.parametrize("n,m,dist", CASES)
@pytest.mark.parametrize("op", ["max", "min"])
def test_hist_minmax_f32(A, oracle, n, m, dist, op):
    vals, inds, hsbar = synth.hist(n, m, dist, seed=n + 2 * m)
    vals = (np.round(vals * 4) / 4).astype(np.float32)  # forced ties
    out = A.adpar_vjp_hist(op, dev(inds), m, dev(hsbar), vals=dev(vals), want_hs=True, want_argidx=True)
    vb, hs, arg = oracle.hist_vjp(op, vals, inds, m, hsbar)
    np.testing.assert_array_equal(out["argidx"].cpu().numpy(), arg)
    np.testing.assert_array_equal(out["valsbar"].cpu().numpy(), vb)
    np.testing.assert_array_equal(out["hs"].cpu().numpy()[arg >= 0], hs[arg >= 0])


@pytest.mark.parametrize("op", ["max", "min"])
def test_hist_minmax_f64_and_accumulate(A, oracle, op):
    n, m = 100003, 300
    vals, inds, hsbar = synth.hist(n, m, "zipf", seed=5)
    vals = np.round(vals.astype(np.float64) * 8) / 8
    hsbar = hsbar.astype(np.float64)
    out = A.adpar_vjp_hist(op, dev(inds), m, dev(hsbar), vals=dev(vals), want_argidx=True)
    vb, hs, arg = oracle.hist_vjp(op, vals, inds, m, hsbar)
    np.testing.assert_array_equal(out["argidx"].cpu().numpy(), arg)
    np.testing.assert_array_equal(out["valsbar"].cpu().numpy(), vb)
    base = synth.normal(n, np.float64, seed=6)
    vbt = dev(base)
    A.adpar_vjp_hist(op, dev(inds), m, dev(hsbar), vals=dev(vals), valsbar=vbt, accumulate=True)
    vb2, _, _ = oracle.hist_vjp(op, vals, inds, m, hsbar, valsbar=base)
    assert rel_l2(vbt.cpu().numpy(), vb2) < 1e-12


@pytest.mark.parametrize("n,m,dist", [(1000, 7, "uniform"), (100003, 256, "zipf"), (200001, 1 << 16, "uniform"),
                                      (150001, 5000, "zipf")])
def test_hist_prod(A, oracle, n, m, dist):
    vals, inds, hsbar = synth.hist(n, m, dist, seed=n + 3 * m)
    g = synth.rng(n)
    vals = (g.uniform(0.5, 1.5, n) * np.sign(vals)).astype(np.float32)
    # a few bins with exactly one and two zeros
    for b, k in ((1, 1), (2, 2), (3, 1)):
        members = np.flatnonzero(inds == b)
        vals[members[:k]] = 0
    ref = oracle.hist_prod_vjp(vals, inds, m, hsbar)
    out = A.adpar_vjp_hist("mul", dev(inds), m, dev(hsbar), vals=dev(vals), want_aux=True)
    aux = out["aux"]
    np.testing.assert_array_equal(aux["nzero"], ref["nzero"])
    np.testing.assert_array_equal(aux["first_zero"], ref["first_zero"])
    ok = np.isfinite(ref["lognz"])
    err = np.abs(aux["log_abs_nz"][ok] - ref["lognz"][ok]) / np.maximum(1, np.abs(ref["lognz"][ok]))
    assert err.max() < 1e-12
    np.testing.assert_array_equal(aux["sign"], ref["signnz"])
    # values (most underflow to 0 in FP32, exactly like the correctly rounded oracle values)
    got = out["valsbar"].cpu().numpy()
    refv = ref["valsbar"].astype(np.float32)
    assert rel_l2(got, refv) < 1e-4 or (np.abs(refv).max() == 0 and np.abs(got).max() == 0)
    lg = A.adpar_vjp_hist("mul", dev(inds), m, dev(hsbar), vals=dev(vals), logdomain=True, want_sign=True)
    gl = lg["valsbar"].cpu().numpy().astype(np.float64)
    fin = np.isfinite(ref["log"])
    np.testing.assert_array_equal(np.isfinite(gl), fin)
    assert np.all(np.abs(gl[fin] - ref["log"][fin]) <= 1e-5 * np.maximum(1, np.abs(ref["log"][fin])))
    np.testing.assert_array_equal(lg["sign"].cpu().numpy(), ref["sign"])


def test_hist_prod_representable_values(A, oracle):
    """Few elements per bin: the products stay in range, so values are compared."""
    n, m = 20000, 5000
    vals, inds, hsbar = synth.hist(n, m, "uniform", seed=77)
    g = synth.rng(78)
    vals = (g.uniform(0.5, 1.5, n) * np.sign(vals)).astype(np.float32)
    vals[:5] = 0
    ref = oracle.hist_prod_vjp(vals, inds, m, hsbar)
    out = A.adpar_vjp_hist("mul", dev(inds), m, dev(hsbar), vals=dev(vals), want_hs=True)
    assert rel_l2(out["valsbar"].cpu().numpy(), ref["valsbar"]) < 1e-5


def test_hist_prod_f32_accumulate_subnormal_and_hsbar_zero(A, oracle):
    """FP32 values, few elements per bin (products in range): accumulation into
    existing adjoints, subnormal FP32 inputs, bins with one zero, bins whose
    hsbar is 0, and int64 indices -- values within the FP32 tolerance."""
    n, m = 30000, 4000
    vals, inds, hsbar = synth.hist(n, m, "uniform", seed=91)
    g = synth.rng(92)
    vals = (g.uniform(0.5, 1.5, n) * np.sign(vals)).astype(np.float32)
    vals[10:20] = (np.float32(3e-39) * np.sign(vals[10:20])).astype(np.float32)  # subnormal
    vals[30:33] = 0
    hsbar = hsbar.copy()
    hsbar[::7] = 0
    base = synth.normal(n, np.float32, seed=93)
    ref = oracle.hist_prod_vjp(vals, inds, m, hsbar, valsbar=base)
    vbt = dev(base)
    A.adpar_vjp_hist("mul", dev(inds.astype(np.int64)), m, dev(hsbar), vals=dev(vals), valsbar=vbt,
                     accumulate=True)
    got = vbt.cpu().numpy()
    assert rel_l2(got, ref["valsbar"]) < 1e-5
    # elements of bins with hsbar 0 (or out of range) keep their old adjoint exactly
    inr = (inds >= 0) & (inds < m)
    keep = ~inr | (hsbar[np.clip(inds, 0, m - 1)] == 0)
    np.testing.assert_array_equal(got[keep], base[keep])


def test_hist_all_out_of_range_and_one_bin(A, oracle):
    n = 5000
    vals = synth.normal(n, np.float32, seed=1)
    inds = np.full(n, -5, np.int32)
    inds[::2] = 10
    hsbar = np.ones(3, np.float32)
    for op in ("add", "max", "mul"):
        out = A.adpar_vjp_hist(op, dev(inds), 3, dev(hsbar), vals=dev(vals))
        assert np.all(out["valsbar"].cpu().numpy() == 0)
    inds1 = np.zeros(n, np.int32)
    out = A.adpar_vjp_hist("max", dev(inds1), 1, dev(hsbar[:1]), vals=dev(vals), want_argidx=True)
    assert out["argidx"].item() == int(np.argmax(vals))


@pytest.mark.parametrize("sort", [False, True])
@pytest.mark.parametrize("dt", [np.float32, np.float64])
def test_scatter(A, oracle, sort, dt):
    n, m = 1 << 20, 1 << 17
    is_, ysbar, xs_saved = synth.scatter(n, m, sort=sort, seed=4)
    ysbar = ysbar.astype(dt)
    xs_saved = xs_saved.astype(dt)
    ys = synth.normal(n, dt, seed=5)
    yb_t, ys_t = dev(ysbar), dev(ys)
    xb, vb = A.adpar_vjp_scatter(dev(is_), yb_t, ys=ys_t, xs_saved=dev(xs_saved))
    rxb, rvb, rys = oracle.scatter_vjp(n, is_, ysbar, ys=ys, xs_saved=xs_saved)
    np.testing.assert_array_equal(vb.cpu().numpy(), rvb)
    np.testing.assert_array_equal(xb.cpu().numpy(), rxb)
    np.testing.assert_array_equal(ys_t.cpu().numpy(), rys)


def test_scatter_out_of_range_and_accumulate(A, oracle):
    n = 1000
    is_ = np.array([3, -1, 999, 1000, 5], np.int64)
    ysbar = synth.normal(n, np.float32, seed=9)
    vs0 = np.arange(5, dtype=np.float32)
    xb, vb = A.adpar_vjp_scatter(dev(is_), dev(ysbar), vsbar=dev(vs0), accumulate=True)
    rxb, rvb, _ = oracle.scatter_vjp(n, is_, ysbar, vsbar=vs0)
    # the FP64 sum of two FP32 numbers is exact; rounded to FP32 it is the FP32 add
    np.testing.assert_array_equal(vb.cpu().numpy(), rvb.astype(np.float32))
    np.testing.assert_array_equal(xb.cpu().numpy(), rxb)


@pytest.mark.parametrize("g,width,na", [("gather", 1, 300), ("gather", 1, 1 << 20), ("scale", 1, 1000),
                                        ("scale", 1, 1 << 18), ("sqdist_row", 8, 256), ("sqdist_row", 32, 4096)])
def test_map_acc(A, oracle, g, width, na):
    nj = 200003
    as_, is_, ws, xsbar = synth.map_acc(nj, na, width=width, seed=na + width)
    ab, wb = A.adpar_vjp_map_acc(g, dev(as_), dev(is_), dev(xsbar), ws=None if g == "gather" else dev(ws),
                                 width=width, want_wsbar=g != "gather")
    rab, rwb = oracle.map_acc_vjp(g, as_, is_, xsbar, ws=None if g == "gather" else ws, width=width)
    assert rel_l2(ab.cpu().numpy(), rab) < 1e-5
    if g != "gather":
        assert rel_l2(wb.cpu().numpy(), rwb) < 1e-5
