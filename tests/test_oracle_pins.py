"""Pins of the FP64 oracle against what arXiv 2202.10297 and mathematics fix.

The oracle computes every adjoint by a sequential tape sweep.  These tests
check it against independent statements of the same numbers: the paper's
fixed cases (tests/golden/fixed_cases.json), closed forms, brute force on
tiny inputs, central finite differences of multilinear functions (exact up
to rounding), forward-mode dual numbers (Sec. 3) and library routines.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_2202_10297_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fixed_cases.json")


@pytest.fixture(scope="module")
def golden():
    with open(GOLDEN) as f:
        return json.load(f)


# ---------------------------------------------------------------- fixed cases
def test_golden_prod_reduce(oracle, golden):
    for c in golden["prod_reduce"]:
        r = oracle.prod_reduce_vjp(c["a"], c["ybar"])
        np.testing.assert_array_equal(r["abar"], c["abar"], err_msg=c["cite"])
        assert r["nzero"] == c["nzero"] and r["first_zero"] == c["first_zero"]


def test_golden_minmax_reduce(oracle, golden):
    for c in golden["minmax_reduce"]:
        y, ab, arg = oracle.reduce_vjp(c["op"], c["a"], c["ybar"])
        assert y == c["y"] and arg == c["argidx"], c["cite"]
        np.testing.assert_array_equal(ab, c["abar"])


def test_golden_scan(oracle, golden):
    for c in golden["scan"]:
        if c["op"] == "linrec":
            ab, bb, ya, yb = oracle.scan_vjp("linrec", c["a"], c["ybar_a"], c["b"], c["ybar_b"])
            np.testing.assert_array_equal(ab, c["abar"], err_msg=c["cite"])
            np.testing.assert_array_equal(bb, c["bbar"])
            np.testing.assert_array_equal(ya, c["ys_a"])
            np.testing.assert_array_equal(yb, c["ys_b"])
        else:
            ab, _, _, _ = oracle.scan_vjp(c["op"], c["a"], c["ybar"])
            np.testing.assert_array_equal(ab, c["abar"], err_msg=c["cite"])


def test_golden_hist(oracle, golden):
    for c in golden["hist"]:
        vb, hs, arg = oracle.hist_vjp(c["op"], c["vals"], c["inds"], c["m"], c["hsbar"])
        np.testing.assert_array_equal(vb, c["valsbar"], err_msg=c["cite"])
        if "argidx" in c:
            np.testing.assert_array_equal(arg, c["argidx"])


def test_golden_scatter(oracle, golden):
    for c in golden["scatter"]:
        xb, vb, yr = oracle.scatter_vjp(c["n"], c["is"], c["ysbar"], ys=c["ys"],
                                        xs_saved=c["xs_saved"])
        np.testing.assert_array_equal(vb, c["vsbar"], err_msg=c["cite"])
        np.testing.assert_array_equal(xb, c["xsbar"])
        np.testing.assert_array_equal(yr, c["ys_restored"])


def test_golden_map_acc(oracle, golden):
    for c in golden["map_acc"]:
        ab, _ = oracle.map_acc_vjp(c["g"], c["as"], c["is"], c["xsbar"])
        np.testing.assert_array_equal(ab, c["asbar"], err_msg=c["cite"])


def test_golden_kmeans(oracle, golden):
    for c in golden["kmeans"]:
        X = np.array(c["X"])
        Cm = np.array(c["C"])
        loss, arg, mind, cb = oracle.kmeans(X, Cm, c["ybar"])
        np.testing.assert_array_equal(arg, c["argmin"], err_msg=c["cite"])
        np.testing.assert_array_equal(mind, c["mind"])
        assert loss == c["loss"]
        np.testing.assert_array_equal(cb, c["Cbar"])
        H = oracle.kmeans_hessdiag(X, Cm, ybar=c["ybar"])
        np.testing.assert_array_equal(H, c["hessdiag"])


# ------------------------------------------------------------- product reduce
def _prod_brute(a, ybar):
    """d(prod a)/d a_i = product of all other elements (O(n^2))."""
    n = len(a)
    return np.array([ybar * np.prod(np.delete(a, i)) for i in range(n)])


@pytest.mark.parametrize("nz", [0, 1, 2, 3])
def test_prod_reduce_brute_force(oracle, nz):
    g = synth.rng(11 + nz)
    for n in (1, 2, 7, 33, 64):
        a = g.uniform(0.5, 1.5, n)
        if nz:
            a[g.choice(n, size=min(nz, n), replace=False)] = 0.0
        ybar = g.normal()
        r = oracle.prod_reduce_vjp(a, ybar)
        np.testing.assert_allclose(r["abar"], _prod_brute(a, ybar), rtol=1e-13, atol=0)
        assert r["nzero"] == int((a == 0).sum())
        zs = np.flatnonzero(a == 0)
        assert r["first_zero"] == (int(zs[0]) if zs.size else -1)


def test_prod_reduce_finite_differences(oracle):
    """The product is linear in each a_i, so a central difference is exact up to rounding."""
    g = synth.rng(5)
    a = g.uniform(0.5, 1.5, 24)
    a[7] = 0.0
    r = oracle.prod_reduce_vjp(a, 1.0)
    h = 0.25
    fd = np.empty_like(a)
    for i in range(a.size):
        ap, am = a.copy(), a.copy()
        ap[i] += h
        am[i] -= h
        fd[i] = (np.prod(ap) - np.prod(am)) / (2 * h)
    np.testing.assert_allclose(r["abar"], fd, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("nz", [0, 1, 2])
def test_prod_reduce_log_domain_closed_form(oracle, nz):
    """n = 65536 underflows FP64; ln|abar_i| = sum_{j != i} ln|a_j| + ln|ybar| (math.fsum)."""
    a, zpos = synth.prod_reduce(65536, nz)
    ybar = -1.5
    r = oracle.prod_reduce_vjp(a, ybar)
    la = np.log(np.abs(np.where(a == 0, 1.0, a)))
    total = math.fsum(la[a != 0])
    assert abs(r["lognz"] - total) <= 1e-12 * abs(total)
    assert r["y"] == 0.0  # the full product (about 1e-1287) rounds to zero
    np.testing.assert_array_equal(r["abar"], np.zeros_like(a))  # correctly rounded values
    if nz == 0:
        expect = total - la + math.log(1.5)
        np.testing.assert_allclose(r["log"], expect, rtol=1e-12)
        np.testing.assert_array_equal(r["sign"], -np.sign(a).astype(np.int8))
    elif nz == 1:
        i0 = zpos[0]
        assert abs(r["log"][i0] - (total + math.log(1.5))) <= 1e-12 * abs(total)
        assert r["sign"][i0] == -1
        assert np.all(np.isneginf(np.delete(r["log"], i0)))
    else:
        assert np.all(np.isneginf(r["log"])) and np.all(r["sign"] == 0)


def test_prod_reduce_representable_value_mode(oracle):
    """A representable case: values scaled so the product stays in range."""
    a, _ = synth.prod_reduce(1024, 0)
    a = a * math.exp(0.04523)
    r = oracle.prod_reduce_vjp(a, 1.0)
    y = np.prod(a)
    assert 1e-30 < abs(y) < 1e30
    np.testing.assert_allclose(r["abar"], y / a, rtol=1e-12)


def test_prod_reduce_equals_hist_with_one_bin(oracle):
    g = synth.rng(9)
    a = g.uniform(0.5, 1.5, 300)
    a[17] = 0
    r = oracle.prod_reduce_vjp(a, 0.75)
    h = oracle.hist_prod_vjp(a, np.zeros(300, np.int64), 1, [0.75])
    np.testing.assert_array_equal(r["abar"], h["valsbar"])
    np.testing.assert_array_equal(r["log"], h["log"])
    assert h["nzero"][0] == 1 and h["first_zero"][0] == 17


# ------------------------------------------------------------ min/max reduce
@pytest.mark.parametrize("op", ["min", "max"])
def test_minmax_reduce_first_index_ties(oracle, op):
    g = synth.rng(3)
    for n in (1, 2, 5, 64, 1000):
        a = np.round(g.normal(size=n) * 2) / 8  # quantised: many exact ties
        y, ab, arg = oracle.reduce_vjp(op, a, 2.5)
        ref = int(np.argmax(a) if op == "max" else np.argmin(a))  # numpy: first occurrence
        assert arg == ref and y == a[ref]
        e = np.zeros(n)
        e[ref] = 2.5
        np.testing.assert_array_equal(ab, e)


def test_add_reduce_broadcast(oracle):
    a = synth.normal(100, np.float64, seed=1)
    y, ab, _ = oracle.reduce_vjp("add", a, 0.5)
    assert abs(y - math.fsum(a)) < 1e-12
    np.testing.assert_array_equal(ab, np.full(100, 0.5))


# ---------------------------------------------------------------------- scans
def test_add_scan_suffix_sums(oracle):
    yb = synth.normal(5000, np.float64, seed=2)
    a = synth.normal(5000, np.float64, seed=3)
    ab, _, ys, _ = oracle.scan_vjp("add", a, yb)
    np.testing.assert_allclose(ab, np.cumsum(yb[::-1])[::-1], rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(ys, np.cumsum(a), rtol=1e-10, atol=1e-10)


@pytest.mark.parametrize("op", ["min", "max"])
def test_minmax_scan_brute_force(oracle, op):
    """abar: each ybar_i goes to the first arg-extremum of a[0..i]."""
    g = synth.rng(4)
    for n in (1, 2, 3, 17, 64):
        a = np.round(g.normal(size=n) * 2) / 4
        yb = g.normal(size=n)
        ab, _, _, _ = oracle.scan_vjp(op, a, yb)
        ref = np.zeros(n)
        for i in range(n):
            k = int(np.argmax(a[: i + 1]) if op == "max" else np.argmin(a[: i + 1]))
            ref[k] += yb[i]
        np.testing.assert_allclose(ab, ref, rtol=1e-13, atol=1e-13)


def test_mul_scan_brute_force(oracle):
    """d rs_i / d a_k = prod_{j <= i, j != k} a_j, so abar_k = sum_{i >= k} ybar_i * that."""
    g = synth.rng(6)
    for n in (1, 2, 9, 32):
        a = g.uniform(0.5, 1.5, n)
        if n > 4:
            a[3] = 0.0
        yb = g.normal(size=n)
        ab, _, ys, _ = oracle.scan_vjp("mul", a, yb)
        ref = np.zeros(n)
        for k in range(n):
            for i in range(k, n):
                ref[k] += yb[i] * np.prod(np.delete(a[: i + 1], k))
        np.testing.assert_allclose(ab, ref, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(ys, np.cumprod(a), rtol=1e-13)


def _linrec_forward(a, b):
    A = np.cumprod(a)
    B = np.empty_like(b)
    acc = 0.0
    for i in range(b.size):
        acc = a[i] * acc + b[i]
        B[i] = acc
    return A, B


def test_linrec_scan_forward_mode_dual_numbers(oracle):
    """Full Jacobian by 2n JVPs (dual numbers, Sec. 3), then J^T ybar."""
    g = synth.rng(7)
    for n in (1, 2, 5, 40):
        a = g.uniform(0.9, 1.0, n)
        b = g.normal(size=n)
        ya = g.normal(size=n)
        yb = g.normal(size=n)
        # tangent seeds: columns 0..n-1 perturb a, n..2n-1 perturb b
        da = np.zeros((n, 2 * n))
        db = np.zeros((n, 2 * n))
        da[np.arange(n), np.arange(n)] = 1.0
        db[np.arange(n), n + np.arange(n)] = 1.0
        A = B = None
        dA = dB = None
        JA = np.zeros((n, 2 * n))
        JB = np.zeros((n, 2 * n))
        for i in range(n):
            if i == 0:
                A, B, dA, dB = a[0], b[0], da[0].copy(), db[0].copy()
            else:
                dA = da[i] * A + a[i] * dA
                dB = da[i] * B + a[i] * dB + db[i]
                A, B = a[i] * A, a[i] * B + b[i]
            JA[i], JB[i] = dA, dB
        vjp = ya @ JA + yb @ JB
        ab, bb, ys_a, ys_b = oracle.scan_vjp("linrec", a, ya, b, yb)
        np.testing.assert_allclose(ab, vjp[:n], rtol=1e-12, atol=1e-13)
        np.testing.assert_allclose(bb, vjp[n:], rtol=1e-12, atol=1e-13)
        A_ref, B_ref = _linrec_forward(a, b)
        np.testing.assert_allclose(ys_a, A_ref, rtol=1e-13)
        np.testing.assert_allclose(ys_b, B_ref, rtol=1e-12, atol=1e-14)


def test_linrec_scan_finite_differences(oracle):
    """A and B are multilinear in (a, b): central differences are exact up to rounding."""
    g = synth.rng(8)
    n = 30
    a = g.uniform(0.9, 1.0, n)
    b = g.normal(size=n)
    ya = g.normal(size=n)
    yb = g.normal(size=n)

    def L(a_, b_):
        A, B = _linrec_forward(a_, b_)
        return float(ya @ A + yb @ B)

    ab, bb, _, _ = oracle.scan_vjp("linrec", a, ya, b, yb)
    h = 0.125
    for k in range(n):
        e = np.zeros(n)
        e[k] = h
        fa = (L(a + e, b) - L(a - e, b)) / (2 * h)
        fb = (L(a, b + e) - L(a, b - e)) / (2 * h)
        assert abs(fa - ab[k]) <= 1e-10 * (1 + abs(fa))
        assert abs(fb - bb[k]) <= 1e-10 * (1 + abs(fb))


def test_linrec_closed_form(oracle):
    """b_bar_k = sum_{i >= k} ybar_B_i prod_{j=k+1..i} a_j (explicit O(n^2))."""
    g = synth.rng(12)
    n = 50
    a = g.uniform(0.9, 1.0, n)
    b = g.normal(size=n)
    ya = g.normal(size=n)
    yb = g.normal(size=n)
    _, bb, _, _ = oracle.scan_vjp("linrec", a, ya, b, yb)
    ref = np.array([sum(yb[i] * np.prod(a[k + 1: i + 1]) for i in range(k, n)) for k in range(n)])
    np.testing.assert_allclose(bb, ref, rtol=1e-12)


# ------------------------------------------------ general reduce rule (Sec. 5.1.1)
def test_reduce_general_linrec_finite_differences(oracle):
    """y = (A_n, B_n) of the linear recurrence is multilinear in (a, b):
    central differences of the plain forward loop are exact up to rounding."""
    g = synth.rng(21)
    n = 40
    a = g.uniform(0.9, 1.1, n)
    b = g.normal(size=n)
    ya, yb = 0.7, -1.3

    def L(a_, b_):
        A, B = _linrec_forward(a_, b_)
        return ya * A[-1] + yb * B[-1]

    (yA, yB), ab, bb = oracle.reduce_general_vjp("linrec", a, ya, b=b, ybar_b=yb)
    A, B = _linrec_forward(a, b)
    assert abs(yA - A[-1]) <= 1e-13 * abs(A[-1]) and abs(yB - B[-1]) <= 1e-12 * (1 + abs(B[-1]))
    h = 0.125
    for k in range(n):
        e = np.zeros(n)
        e[k] = h
        fa = (L(a + e, b) - L(a - e, b)) / (2 * h)
        fb = (L(a, b + e) - L(a, b - e)) / (2 * h)
        assert abs(fa - ab[k]) <= 1e-10 * (1 + abs(fa))
        assert abs(fb - bb[k]) <= 1e-10 * (1 + abs(fb))


@pytest.mark.parametrize("op", ["add", "mul", "min", "max", "linrec"])
def test_reduce_general_is_scan_with_last_cotangent(oracle, op):
    """A reduce is the last output of the inclusive scan, so its VJP equals the
    scan VJP with ybar zero everywhere but the last position."""
    g = synth.rng(22)
    n = 57
    if op in ("min", "max"):
        a = np.round(g.normal(size=n) * 4) / 4  # ties
    elif op == "mul":
        a = g.uniform(0.5, 1.5, n)
        a[[5, 40]] = 0.0
    else:
        a = g.uniform(0.9, 1.1, n)
    b = g.normal(size=n)
    ya = np.zeros(n)
    yb = np.zeros(n)
    ya[-1], yb[-1] = 0.8, 1.7
    if op == "linrec":
        sab, sbb, _, _ = oracle.scan_vjp("linrec", a, ya, b, yb)
        _, ab, bb = oracle.reduce_general_vjp("linrec", a, 0.8, b=b, ybar_b=1.7)
        np.testing.assert_allclose(bb, sbb, rtol=1e-13, atol=1e-15)
    else:
        sab, _, _, _ = oracle.scan_vjp(op, a, ya)
        _, ab, _ = oracle.reduce_general_vjp(op, a, 0.8)
    np.testing.assert_allclose(ab, sab, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("op", ["add", "min", "max", "mul"])
def test_reduce_general_matches_plain_reduce_definitions(oracle, op):
    """+ broadcasts ybar; min/max put it at the lowest index of the extremum;
    * gives prod_{j != i} a_j * ybar (brute force, no division)."""
    g = synth.rng(23)
    n = 33
    a = np.round(g.normal(size=n) * 3) / 3 if op in ("min", "max") else g.uniform(0.5, 1.5, n)
    (y,), ab, _ = oracle.reduce_general_vjp(op, a, 2.5)
    if op == "add":
        assert abs(y - a.sum()) <= 1e-12 * (1 + abs(a.sum()))
        np.testing.assert_array_equal(ab, np.full(n, 2.5))
    elif op == "mul":
        ref = np.array([np.prod(np.delete(a, i)) * 2.5 for i in range(n)])
        np.testing.assert_allclose(ab, ref, rtol=1e-12)
    else:
        i0 = int(np.argmax(a) if op == "max" else np.argmin(a))  # numpy: first index on ties
        ref = np.zeros(n)
        ref[i0] = 2.5
        np.testing.assert_array_equal(ab, ref)
        assert y == a[i0]


def test_reduce_general_empty_and_accumulate(oracle):
    (yA, yB), ab, bb = oracle.reduce_general_vjp("linrec", np.zeros(0), 1.0, b=np.zeros(0), ybar_b=1.0)
    assert (yA, yB) == (1.0, 0.0) and ab.size == 0 and bb.size == 0
    _, ab, _ = oracle.reduce_general_vjp("add", [1.0, 2.0], 3.0, abar=[10.0, -1.0])
    np.testing.assert_array_equal(ab, [13.0, 2.0])


# ------------------------------------------------------- forward mode (JVP)
@pytest.mark.parametrize("op", ["add", "mul", "min", "max", "linrec"])
def test_scan_jvp_vjp_duality(oracle, op):
    """<ybar, J xdot> = <J^T ybar, xdot> against the (separately pinned) VJP."""
    g = synth.rng(31)
    n = 45
    if op in ("min", "max"):
        a = g.normal(size=n)  # no ties: the derivative is defined
    elif op == "mul":
        a = g.uniform(0.5, 1.5, n)
    else:
        a = g.uniform(0.9, 1.1, n)
    b = g.normal(size=n)
    ad, bd = g.normal(size=n), g.normal(size=n)
    ya, yb = g.normal(size=n), g.normal(size=n)
    if op == "linrec":
        _, _, yda, ydb = oracle.scan_jvp(op, a, ad, b, bd)
        vab, vbb, _, _ = oracle.scan_vjp(op, a, ya, b, yb)
        lhs = ya @ yda + yb @ ydb
        rhs = vab @ ad + vbb @ bd
    else:
        _, _, yda, _ = oracle.scan_jvp(op, a, ad)
        vab, _, _, _ = oracle.scan_vjp(op, a, ya)
        lhs, rhs = ya @ yda, vab @ ad
    assert abs(lhs - rhs) <= 1e-12 * (1 + abs(lhs))


def test_scan_jvp_linrec_finite_differences(oracle):
    """A, B are multilinear: the central difference along (adot, bdot) is exact up to rounding."""
    g = synth.rng(32)
    n = 30
    a = g.uniform(0.9, 1.1, n)
    b = g.normal(size=n)
    ad, bd = g.normal(size=n), g.normal(size=n)
    ya, yb, yda, ydb = oracle.scan_jvp("linrec", a, ad, b, bd)
    A, B = _linrec_forward(a, b)
    np.testing.assert_allclose(ya, A, rtol=1e-13)
    np.testing.assert_allclose(yb, B, rtol=1e-12, atol=1e-14)
    # the tangent is a polynomial of degree <= n in h: use exact-ish small h on both sides
    h = 1e-4
    Ap, Bp = _linrec_forward(a + h * ad, b + h * bd)
    Am, Bm = _linrec_forward(a - h * ad, b - h * bd)
    np.testing.assert_allclose(yda, (Ap - Am) / (2 * h), rtol=1e-6, atol=1e-8)
    np.testing.assert_allclose(ydb, (Bp - Bm) / (2 * h), rtol=1e-6, atol=1e-8)


def test_scan_jvp_add_and_max_definitions(oracle):
    g = synth.rng(33)
    n = 50
    a = np.round(g.normal(size=n) * 4) / 4  # ties: the earlier element keeps the record
    ad = g.normal(size=n)
    _, _, yd, _ = oracle.scan_jvp("add", a, ad)
    np.testing.assert_allclose(yd, np.cumsum(ad), rtol=1e-13, atol=1e-14)
    _, _, yd, _ = oracle.scan_jvp("max", a, ad)
    arg = np.array([int(np.argmax(a[: i + 1])) for i in range(n)])  # first index of the running max
    np.testing.assert_array_equal(yd, ad[arg])


def test_scan_accumulates(oracle):
    """Adjoints are added into the given arrays (Eq. rewrite-adj, +=)."""
    yb = np.array([1.0, 2.0, 3.0])
    ab, _, _, _ = oracle.scan_vjp("add", [0.0, 0.0, 0.0], yb, abar=[100.0, 0.0, -1.0])
    np.testing.assert_array_equal(ab, [106.0, 5.0, 2.0])


# --------------------------------------------------------------- histograms
def test_hist_add_is_gather(oracle):
    vals, inds, hsbar = synth.hist(20000, 97, "zipf", seed=1)
    vb, hs, _ = oracle.hist_vjp("add", vals, inds, 97, hsbar)
    ok = (inds >= 0) & (inds < 97)
    ref = np.where(ok, hsbar.astype(np.float64)[np.clip(inds, 0, 96)], 0.0)
    np.testing.assert_array_equal(vb, ref)
    ref_hs = np.zeros(97)
    np.add.at(ref_hs, inds[ok], vals[ok].astype(np.float64))
    np.testing.assert_allclose(hs, ref_hs, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("op", ["min", "max"])
def test_hist_minmax_brute_force(oracle, op):
    g = synth.rng(13)
    n, m = 3000, 37
    vals = np.round(g.normal(size=n) * 4) / 4  # ties
    inds = g.integers(-3, m + 3, size=n)
    hsbar = g.normal(size=m)
    vb, hs, arg = oracle.hist_vjp(op, vals, inds, m, hsbar)
    ref = np.zeros(n)
    for b in range(m):
        members = np.flatnonzero(inds == b)
        if members.size == 0:
            assert arg[b] == -1
            continue
        v = vals[members]
        k = members[int(np.argmax(v) if op == "max" else np.argmin(v))]
        assert arg[b] == k and hs[b] == vals[k]
        ref[k] += hsbar[b]
    np.testing.assert_array_equal(vb, ref)


def test_hist_prod_brute_force(oracle):
    g = synth.rng(14)
    n, m = 200, 6
    vals = g.uniform(0.5, 1.5, n) * np.where(g.random(n) < 0.5, -1, 1)
    inds = g.integers(-1, m + 1, size=n)
    vals[np.flatnonzero(inds == 2)[:1]] = 0.0  # bin 2: one zero
    vals[np.flatnonzero(inds == 3)[:2]] = 0.0  # bin 3: two zeros
    hsbar = g.normal(size=m)
    r = oracle.hist_prod_vjp(vals, inds, m, hsbar)
    ref = np.zeros(n)
    for i in range(n):
        b = inds[i]
        if 0 <= b < m:
            members = np.flatnonzero(inds == b)
            ref[i] = hsbar[b] * np.prod(vals[members[members != i]])
    np.testing.assert_allclose(r["valsbar"], ref, rtol=1e-12, atol=1e-300)
    assert r["nzero"][2] == 1 and r["nzero"][3] == 2
    assert r["first_zero"][2] == np.flatnonzero(inds == 2)[0]


def test_hist_minmax_equal_reduce_with_one_bin(oracle):
    a = np.round(synth.normal(500, np.float64, seed=5) * 3) / 3
    for op in ("min", "max"):
        y, ab, arg = oracle.reduce_vjp(op, a, 1.25)
        vb, hs, harg = oracle.hist_vjp(op, a, np.zeros(500, np.int64), 1, [1.25])
        assert arg == harg[0] and y == hs[0]
        np.testing.assert_array_equal(ab, vb)


# ------------------------------------------------------------------- scatter
def test_scan_wide_matrec_primal_fibonacci(oracle):
    """The companion matrix [[1, 1], [1, 0]] with h_0 = (1, 0) makes the
    affine-map scan the Fibonacci recurrence: h_i = (F_{i+1}, F_i) exactly,
    and the matrix part is the matrix power [[F_{i+1}, F_i], [F_i, F_{i-1}]]."""
    n = 30
    a = np.tile([1.0, 1.0, 1.0, 0.0, 0.0, 0.0], (n, 1))
    a[0, 4:] = [1.0, 0.0]
    _, ys = oracle.scan_wide_vjp("matrec2", a, np.zeros((n, 6)))
    F = [0, 1]
    while len(F) < n + 3:
        F.append(F[-1] + F[-2])
    for i in range(n):
        assert list(ys[i, 4:]) == [F[i + 1], F[i]]
        assert list(ys[i, :4]) == [F[i + 2], F[i + 1], F[i + 1], F[i]]


def test_scan_wide_matrec_finite_differences(oracle):
    """Every output of the matrix recurrence is linear in each single input
    scalar, so central differences of a plain loop of 2x2 matrix products are
    exact up to rounding for every component of every element."""
    g = synth.rng(51)
    n = 12
    a = np.concatenate([np.eye(2).ravel() + 0.4 * g.normal(size=(n, 4)), g.normal(size=(n, 2))], axis=1)
    yb = g.normal(size=(n, 6))

    def loss(x):
        P = x[0, :4].reshape(2, 2).copy()
        h = x[0, 4:].copy()
        tot = yb[0, :4] @ P.ravel() + yb[0, 4:] @ h
        for i in range(1, n):
            M = x[i, :4].reshape(2, 2)
            P = M @ P
            h = M @ h + x[i, 4:]
            tot += yb[i, :4] @ P.ravel() + yb[i, 4:] @ h
        return tot

    ab, _ = oracle.scan_wide_vjp("matrec2", a, yb)
    step = 0.125
    for i in range(n):
        for c in range(6):
            e = np.zeros_like(a)
            e[i, c] = step
            fd = (loss(a + e) - loss(a - e)) / (2 * step)
            assert abs(fd - ab[i, c]) <= 1e-10 * (1 + abs(fd)), (i, c, fd, ab[i, c])


def test_scan_wide_matrec_diagonal_is_two_linrecs(oracle):
    """With diagonal matrices the recurrence splits into two scalar linear
    recurrences (a = M00, b = v0) and (a = M11, b = v1); with cotangents only
    on (P00, h0, P11, h1) their adjoints are the separately pinned LINREC
    sweep's."""
    g = synth.rng(52)
    n = 40
    a0, a1 = g.uniform(0.8, 1.2, n), g.uniform(0.8, 1.2, n)
    b0, b1 = g.normal(size=n), g.normal(size=n)
    y = g.normal(size=(4, n))
    a = np.zeros((n, 6))
    a[:, 0], a[:, 3], a[:, 4], a[:, 5] = a0, a1, b0, b1
    yb = np.zeros((n, 6))
    yb[:, 0], yb[:, 4], yb[:, 3], yb[:, 5] = y[0], y[1], y[2], y[3]
    ab, _ = oracle.scan_wide_vjp("matrec2", a, yb)
    ra0, rb0, _, _ = oracle.scan_vjp("linrec", a0, y[0], b0, y[1])
    ra1, rb1, _, _ = oracle.scan_vjp("linrec", a1, y[2], b1, y[3])
    for got, ref in ((ab[:, 0], ra0), (ab[:, 4], rb0), (ab[:, 3], ra1), (ab[:, 5], rb1)):
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-14)


def test_scan_wide_linrec_equals_linrec_scan(oracle):
    """The width-2 element (a, b) with the full 2x2 Jacobians is the linear
    recurrence of the scalar-coefficient sweep; accumulation adds on."""
    g = synth.rng(53)
    n = 37
    a, b = g.uniform(0.9, 1.1, n), g.normal(size=n)
    ya, yb = g.normal(size=n), g.normal(size=n)
    base = g.normal(size=(n, 2))
    ab, ys = oracle.scan_wide_vjp("linrec", np.stack([a, b], 1), np.stack([ya, yb], 1), abar=base)
    ra, rb, rya, ryb = oracle.scan_vjp("linrec", a, ya, b, yb)
    np.testing.assert_allclose(ab[:, 0] - base[:, 0], ra, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(ab[:, 1] - base[:, 1], rb, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(ys[:, 0], rya, rtol=1e-14)
    np.testing.assert_allclose(ys[:, 1], ryb, rtol=1e-14)
    ab, _ = oracle.scan_wide_vjp("matrec2", np.ones((1, 6)), np.arange(6.0).reshape(1, 6))
    np.testing.assert_array_equal(ab, np.arange(6.0).reshape(1, 6))  # n = 1: abar = ybar


def _bins_of(inds, m):
    return [np.flatnonzero(inds == k) for k in range(m)]


@pytest.mark.parametrize("op", ["add", "mul", "min", "max"])
def test_hist_general_definitions(oracle, op):
    """General-rule reduce_by_index against each operator's definition, bin
    by bin: + gathers hsbar; * is the product of the bin's other elements
    (brute force, zeros included); min/max put hsbar at the lowest index of
    the bin's extremum (numpy's first-index argmax); out-of-range elements
    get nothing; hs is the bin's reduction and empty bins hold e."""
    g = synth.rng(41)
    n, m = 300, 13
    inds = g.integers(-2, m + 2, n)
    if op in ("min", "max"):
        v = np.round(g.normal(size=n) * 3) / 3  # many ties
    elif op == "mul":
        v = g.uniform(0.5, 1.5, n)
        first = [np.flatnonzero(inds == k) for k in (2, 5)]
        v[first[0][:1]] = 0.0   # one zero in bin 2
        v[first[1][:2]] = 0.0   # two zeros in bin 5
    else:
        v = g.normal(size=n)
    inds[inds == 7] = -1        # bin 7 empty
    hsbar = g.normal(size=m)
    vb, _, hs, _ = oracle.hist_general_vjp(op, v, inds, m, hsbar)
    ref = np.zeros(n)
    neutral = {"add": 0.0, "mul": 1.0, "min": np.inf, "max": -np.inf}[op]
    for k, idx in enumerate(_bins_of(inds, m)):
        if idx.size == 0:
            assert hs[k] == neutral
            continue
        x = v[idx]
        if op == "add":
            ref[idx] = hsbar[k]
            assert abs(hs[k] - x.sum()) <= 1e-12 * (1 + np.abs(x).sum())
        elif op == "mul":
            ref[idx] = [np.prod(np.delete(x, j)) * hsbar[k] for j in range(x.size)]
            assert abs(hs[k] - np.prod(x)) <= 1e-12 * abs(np.prod(x)) + 1e-300
        else:
            j = int(np.argmax(x) if op == "max" else np.argmin(x))
            ref[idx[j]] = hsbar[k]
            assert hs[k] == x[j]
    if op == "mul":
        np.testing.assert_allclose(vb, ref, rtol=1e-12, atol=0)
    else:
        np.testing.assert_allclose(vb, ref, rtol=1e-13, atol=0)
    assert np.all(vb[(inds < 0) | (inds >= m)] == 0)


@pytest.mark.parametrize("op", ["add", "min", "max"])
def test_hist_general_agrees_with_special_rule_oracle(oracle, op):
    """The general rule and the special rules of Sec. 5.1.2 (a separate tape
    sweep with scalar derivatives) give the same adjoint and bins."""
    g = synth.rng(42)
    n, m = 500, 9
    inds = g.integers(-1, m + 1, n)
    v = np.round(g.normal(size=n) * 2) / 2
    hsbar = g.normal(size=m)
    vb, _, hs, _ = oracle.hist_general_vjp(op, v, inds, m, hsbar)
    vb2, hs2, _ = oracle.hist_vjp(op, v, inds, m, hsbar)
    np.testing.assert_allclose(vb, vb2, rtol=1e-14, atol=0)
    np.testing.assert_allclose(hs, hs2, rtol=1e-14, atol=0)


def test_hist_general_linrec_finite_differences(oracle):
    """LINREC bins are (A, B) of each bin's subsequence in index order; the
    loss sum_k hsbar_A[k] A_k + hsbar_B[k] B_k is multilinear in (a, b), so
    central differences of the plain per-bin forward loop are exact up to
    rounding."""
    g = synth.rng(43)
    n, m = 60, 5
    a = g.uniform(0.8, 1.2, n)
    b = g.normal(size=n)
    inds = g.integers(-1, m + 1, n)
    ha, hb = g.normal(size=m), g.normal(size=m)

    def L(a_, b_):
        tot = 0.0
        for k, idx in enumerate(_bins_of(inds, m)):
            if idx.size == 0:
                tot += ha[k] * 1.0
                continue
            A, B = _linrec_forward(a_[idx], b_[idx])
            tot += ha[k] * A[-1] + hb[k] * B[-1]
        return tot

    ab, bb, hsA, hsB = oracle.hist_general_vjp("linrec", a, inds, m, ha, b=b, hsbar_b=hb)
    for k, idx in enumerate(_bins_of(inds, m)):
        if idx.size:
            A, B = _linrec_forward(a[idx], b[idx])
            assert abs(hsA[k] - A[-1]) <= 1e-13 and abs(hsB[k] - B[-1]) <= 1e-12 * (1 + abs(B[-1]))
        else:
            assert (hsA[k], hsB[k]) == (1.0, 0.0)
    h = 0.125
    for i in range(n):
        e = np.zeros(n)
        e[i] = h
        fa = (L(a + e, b) - L(a - e, b)) / (2 * h)
        fb = (L(a, b + e) - L(a, b - e)) / (2 * h)
        assert abs(fa - ab[i]) <= 1e-10 * (1 + abs(fa))
        assert abs(fb - bb[i]) <= 1e-10 * (1 + abs(fb))


def test_hist_general_linrec_keeps_index_order(oracle):
    """LINREC does not commute: reversing the order of one bin's elements
    changes that bin (and only that bin), so the sweep must combine each
    bin in index order."""
    a = np.array([2.0, 3.0, 0.5, 4.0])
    b = np.array([1.0, -1.0, 2.0, 0.25])
    inds = np.array([0, 1, 0, 1])
    _, _, hsA, hsB = oracle.hist_general_vjp("linrec", a, inds, 2, np.ones(2), b=b, hsbar_b=np.ones(2))
    # bin 0: (2,1) then (0.5,2) -> (1, 0.5*1 + 2); bin 1: (3,-1) then (4,0.25) -> (12, -4 + 0.25)
    np.testing.assert_array_equal(hsA, [1.0, 12.0])
    np.testing.assert_array_equal(hsB, [2.5, -3.75])


def test_hist_general_one_bin_is_reduce_and_accumulates(oracle):
    """With every index in bin 0 the rule is the general reduce; ADPAR-style
    accumulation adds onto the given adjoint and leaves skipped elements."""
    g = synth.rng(44)
    n = 31
    a, b = g.uniform(0.9, 1.1, n), g.normal(size=n)
    ab, bb, hsA, hsB = oracle.hist_general_vjp("linrec", a, np.zeros(n, np.int64), 1, [0.6], b=b,
                                               hsbar_b=[-1.1])
    (yA, yB), rab, rbb = oracle.reduce_general_vjp("linrec", a, 0.6, b=b, ybar_b=-1.1)
    np.testing.assert_allclose(ab, rab, rtol=1e-14, atol=0)
    np.testing.assert_allclose(bb, rbb, rtol=1e-14, atol=0)
    assert abs(hsA[0] - yA) <= 1e-15 and abs(hsB[0] - yB) <= 1e-14
    vb, _, _, _ = oracle.hist_general_vjp("add", [1.0, 2.0, 3.0], [0, 5, 1], 2, [10.0, 20.0],
                                          valsbar=[1.0, 1.0, 1.0])
    np.testing.assert_array_equal(vb, [11.0, 1.0, 21.0])


def test_scatter_closed_form(oracle):
    n, m = 4096, 1000
    is_, ysbar, xs_saved = synth.scatter(n, m, seed=3)
    ys = synth.normal(n, np.float64, seed=4)
    xb, vb, yr = oracle.scatter_vjp(n, is_, ysbar, ys=ys, xs_saved=xs_saved)
    assert np.unique(is_).size == m
    np.testing.assert_array_equal(vb, ysbar.astype(np.float64)[is_])
    ref = ysbar.astype(np.float64).copy()
    ref[is_] = 0.0
    np.testing.assert_array_equal(xb, ref)
    ref_y = ys.copy()
    ref_y[is_] = xs_saved
    np.testing.assert_array_equal(yr, ref_y)


# ------------------------------------------------------------------- map_acc
def test_map_acc_gather_add_at(oracle):
    as_, is_, ws, xsbar = synth.map_acc(5000, 300)
    ab, _ = oracle.map_acc_vjp("gather", as_, is_, xsbar)
    ref = np.zeros(300)
    np.add.at(ref, is_, xsbar.astype(np.float64))
    np.testing.assert_allclose(ab, ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("g,width", [("scale", 1), ("sqdist_row", 4)])
def test_map_acc_finite_differences(oracle, g, width):
    """sum_j xsbar_j g(as[is_j], ws_j) is quadratic at most: central differences are exact."""
    as_, is_, ws, xsbar = synth.map_acc(40, 7, width=width, seed=21)
    as_ = as_.astype(np.float64)
    ws = ws.astype(np.float64)

    def L(a_, w_):
        A = a_.reshape(-1, width)[is_]
        W = w_.reshape(-1, width)
        x = (A * W)[:, 0] if g == "scale" else ((W - A) ** 2).sum(1)
        return float(xsbar.astype(np.float64) @ x)

    ab, wb = oracle.map_acc_vjp(g, as_, is_, xsbar, ws=ws, width=width)
    h = 0.5
    for k in range(as_.size):
        e = np.zeros(as_.size)
        e[k] = h
        assert abs((L(as_ + e, ws) - L(as_ - e, ws)) / (2 * h) - ab[k]) < 1e-11
    for k in range(ws.size):
        e = np.zeros(ws.size)
        e[k] = h
        assert abs((L(as_, ws + e) - L(as_, ws - e)) / (2 * h) - wb[k]) < 1e-11


# ------------------------------------------------------------------- k-means
def test_kmeans_closed_form_and_fd(oracle):
    X, Cm = synth.kmeans(300, 5, 8, seed=2)
    X = X.astype(np.float64)
    Cm = Cm.astype(np.float64)
    loss, arg, mind, cb = oracle.kmeans(X, Cm, 1.5)
    D = ((X[:, None, :] - Cm[None, :, :]) ** 2).sum(-1)
    np.testing.assert_array_equal(arg, np.argmin(D, axis=1))
    assert abs(loss - D.min(1).sum()) < 1e-9
    ref = np.zeros_like(Cm)
    for k in range(8):
        sel = arg == k
        ref[k] = 2 * 1.5 * (sel.sum() * Cm[k] - X[sel].sum(0))
    np.testing.assert_allclose(cb, ref, rtol=1e-11, atol=1e-11)
    # finite differences (no argmin changes for a small step away from ties)
    gap = np.sort(D, 1)[:, 1] - D.min(1)
    assert gap.min() > 1e-4
    h = 1e-6
    for (k, j) in [(0, 0), (3, 2), (7, 4)]:
        Cp, Cn = Cm.copy(), Cm.copy()
        Cp[k, j] += h
        Cn[k, j] -= h
        fd = 1.5 * (oracle.kmeans(X, Cp)[0] - oracle.kmeans(X, Cn)[0]) / (2 * h)
        assert abs(fd - cb[k, j]) < 1e-5 * (1 + abs(fd))


def test_kmeans_hessdiag_is_derivative_of_gradient(oracle):
    """The Hessian diagonal in C equals central differences of the oracle's
    own gradient (Cbar) along each coordinate of C: with the steps far from
    any argmin tie the gradient is affine in C, so the differences are exact
    up to rounding.  Also the closed form 2 ybar cnt_k against argmin counts."""
    g = synth.rng(61)
    N, d, k = 400, 4, 5
    X = g.normal(size=(N, d))
    Cm = g.normal(size=(k, d)) * 1.5
    H = oracle.kmeans_hessdiag(X, Cm, ybar=0.7)
    _, arg, mind, _ = oracle.kmeans(X, Cm)
    # the step must not move any point across a tie
    dist = ((X[:, None, :] - Cm[None, :, :]) ** 2).sum(-1)
    srt = np.sort(dist, axis=1)
    step = 1e-4
    assert (srt[:, 1] - srt[:, 0]).min() > 10 * step * (np.abs(X).max() + np.abs(Cm).max())
    for c in range(k):
        for j in range(d):
            e = np.zeros_like(Cm)
            e[c, j] = step
            gp = oracle.kmeans(X, Cm + e, ybar=0.7)[3]
            gm = oracle.kmeans(X, Cm - e, ybar=0.7)[3]
            fd = (gp[c, j] - gm[c, j]) / (2 * step)
            assert abs(fd - H[c, j]) <= 1e-6 * (1 + abs(fd))
    cnt = np.bincount(arg, minlength=k)
    np.testing.assert_array_equal(H, 2 * 0.7 * cnt[:, None] * np.ones((1, d)))


# ------------------------------------------------------------ forward mode
# The dual-number sweeps (Sec. 3) are pinned by brute force and closed forms
# on small inputs, by central differences where the function is multilinear
# or quadratic (exact up to rounding), and by the duality
# <ybar, J xdot> = <J^T ybar, xdot> against the reverse sweeps pinned above.
@pytest.mark.parametrize("op", ["add", "min", "max"])
def test_reduce_jvp_closed_form_and_duality(oracle, op):
    g = synth.rng(101)
    a = np.round(g.normal(size=57) * 4) / 4  # forced ties
    ad = g.normal(size=57)
    y, yd = oracle.reduce_jvp(op, a, ad)
    if op == "add":
        assert y == a.sum() or abs(y - a.sum()) < 1e-12
        assert abs(yd - ad.sum()) < 1e-12
    else:
        k = int(np.argmax(a) if op == "max" else np.argmin(a))  # numpy: first index
        assert y == a[k] and yd == ad[k]
    ybar = 1.7
    _, ab, _ = oracle.reduce_vjp(op, a, ybar)
    assert abs(ybar * yd - np.dot(ab, ad)) < 1e-12 * (1 + abs(ybar * yd))
    # n = 0: the neutral element and a zero tangent
    y0, yd0 = oracle.reduce_jvp(op, np.zeros(0), np.zeros(0))
    assert yd0 == 0.0


@pytest.mark.parametrize("nz", [0, 1, 2])
def test_prod_reduce_jvp_brute_force_fd_and_duality(oracle, nz):
    g = synth.rng(102 + nz)
    n = 40
    a = g.uniform(0.5, 1.5, n)
    a[g.choice(n, nz, replace=False)] = 0.0
    ad = g.normal(size=n)
    r = oracle.prod_reduce_jvp(a, ad)
    # brute force: sum_i prod_{j != i} a_j adot_i
    ref = sum(np.prod(np.delete(a, i)) * ad[i] for i in range(n))
    assert abs(r["ydot"] - ref) <= 1e-13 * max(1e-300, abs(ref)) + 1e-300
    if nz >= 2:
        assert r["ydot"] == 0.0 and r["sign"] == 0
    else:
        assert r["sign"] == np.sign(ref) and abs(r["log"] - np.log(abs(ref))) < 1e-12
    # central differences along adot: even orders cancel, the third-order
    # terms are O(h^2)
    h = 1e-5
    fd = (np.prod(a + h * ad) - np.prod(a - h * ad)) / (2 * h)
    assert abs(fd - ref) <= 1e-6 * (abs(ref) + 1e-3)
    # duality with the reverse sweep, in the log domain for long products
    a2 = g.uniform(0.5, 1.5, 5000)
    ad2 = g.normal(size=5000)
    rj = oracle.prod_reduce_jvp(a2, ad2)
    rv = oracle.prod_reduce_vjp(a2, 1.0)
    # <1, J adot> = sum_i abar_i adot_i with abar_i = exp(log_i) sign_i: sum in
    # scaled form around the largest term
    lg = rv["log"]
    top = lg.max()
    s = np.sum(rv["sign"] * np.exp(lg - top) * ad2)
    assert rj["sign"] == np.sign(s)
    assert abs(rj["log"] - (top + np.log(abs(s)))) < 1e-10


@pytest.mark.parametrize("op", ["add", "min", "max"])
def test_hist_jvp_brute_force_and_duality(oracle, op):
    g = synth.rng(110)
    n, m = 500, 13
    vals = np.round(g.normal(size=n) * 3) / 3
    vd = g.normal(size=n)
    inds = g.integers(-2, m + 2, size=n)
    hs, hd = oracle.hist_jvp(op, vals, vd, inds, m)
    for b in range(m):
        sel = np.flatnonzero(inds == b)
        if sel.size == 0:
            assert hd[b] == 0.0
            continue
        if op == "add":
            assert abs(hd[b] - vd[sel].sum()) < 1e-12 and abs(hs[b] - vals[sel].sum()) < 1e-12
        else:
            v = vals[sel]
            k = sel[int(np.argmax(v) if op == "max" else np.argmin(v))]  # first index in the bin
            assert hs[b] == vals[k] and hd[b] == vd[k]
    hsbar = g.normal(size=m)
    vb, _, _ = oracle.hist_vjp(op, vals, inds, m, hsbar)
    assert abs(np.dot(hsbar, hd) - np.dot(vb, vd)) < 1e-11


def test_hist_prod_jvp_brute_force(oracle):
    g = synth.rng(111)
    n, m = 300, 7
    vals = g.uniform(0.5, 1.5, n) * np.sign(g.normal(size=n))
    inds = g.integers(-1, m + 1, size=n)
    vals[np.flatnonzero(inds == 2)[:1]] = 0.0   # one zero in bin 2
    vals[np.flatnonzero(inds == 3)[:2]] = 0.0   # two in bin 3
    vd = g.normal(size=n)
    r = oracle.hist_prod_jvp(vals, vd, inds, m)
    for b in range(m):
        sel = np.flatnonzero(inds == b)
        v, t = vals[sel], vd[sel]
        ref = sum(np.prod(np.delete(v, i)) * t[i] for i in range(v.size))
        assert abs(r["hsdot"][b] - ref) <= 1e-12 * abs(ref) + 1e-300, b
        assert r["sign"][b] == np.sign(ref)
    assert r["hsdot"][3] == 0.0


def test_scatter_jvp_closed_form(oracle):
    g = synth.rng(112)
    n, m = 50, 20
    is_ = g.permutation(n + 10)[:m] - 5  # some out of range, no duplicates
    vd = g.normal(size=m)
    xd = g.normal(size=n)
    out = oracle.scatter_jvp(n, is_, vd, xd)
    ref = xd.copy()
    for j, k in enumerate(is_):
        if 0 <= k < n:
            ref[k] = vd[j]
    np.testing.assert_array_equal(out, ref)


@pytest.mark.parametrize("gname,width", [("gather", 1), ("scale", 1), ("sqdist_row", 3)])
def test_map_acc_jvp_fd_and_duality(oracle, gname, width):
    g = synth.rng(113)
    na, nj = 9, 40
    as_ = g.normal(size=na * width)
    ws = g.normal(size=nj * width)
    is_ = g.integers(-1, na + 1, size=nj)
    asd = g.normal(size=na * width)
    wsd = g.normal(size=nj * width) if gname != "gather" else None
    xd = oracle.map_acc_jvp(gname, as_, is_, asd, ws=ws, wsdot=wsd, width=width)

    def F(a, w):
        out = np.zeros(nj)
        for j in range(nj):
            i = is_[j]
            if not (0 <= i < na):
                continue
            if gname == "gather":
                out[j] = a[i]
            elif gname == "scale":
                out[j] = a[i] * w[j]
            else:
                out[j] = ((w[j * width:(j + 1) * width] - a[i * width:(i + 1) * width]) ** 2).sum()
        return out
    h = 0.5  # F is at most quadratic: central differences are exact up to rounding
    wdir = wsd if wsd is not None else np.zeros_like(ws)
    fd = (F(as_ + h * asd, ws + h * wdir) - F(as_ - h * asd, ws - h * wdir)) / (2 * h)
    np.testing.assert_allclose(xd, fd, rtol=1e-12, atol=1e-12)
    xsbar = g.normal(size=nj)
    ab, wb = oracle.map_acc_vjp(gname, as_, is_, xsbar, ws=ws, width=width)
    lhs = np.dot(xsbar, xd)
    rhs = np.dot(ab, asd) + (np.dot(wb, wsd) if wsd is not None else 0.0)
    assert abs(lhs - rhs) < 1e-11


def test_kmeans_fwd_rev_is_the_derivative_of_the_gradient(oracle):
    """Forward over reverse: the tangent of the oracle's own gradient along
    Cdot equals central differences of that gradient (affine in C away from
    argmin ties, so exact up to rounding); the loss's tangent equals central
    differences of the loss; with Cdot = 1 it is the Hessian diagonal."""
    g = synth.rng(114)
    N, d, k = 300, 3, 4
    X = g.normal(size=(N, d))
    Cm = g.normal(size=(k, d)) * 1.5
    Cd = g.normal(size=(k, d))
    ybar = 0.8
    ydot, Gd = oracle.kmeans_fwd_rev(X, Cm, Cd, ybar)
    h = 1e-5
    lp, ap, _, gp = oracle.kmeans(X, Cm + h * Cd, ybar)
    lm, am, _, gm = oracle.kmeans(X, Cm - h * Cd, ybar)
    _, a0, _, _ = oracle.kmeans(X, Cm, ybar)
    # the steps move no point across an argmin tie
    np.testing.assert_array_equal(ap, a0)
    np.testing.assert_array_equal(am, a0)
    np.testing.assert_allclose(Gd, (gp - gm) / (2 * h), rtol=1e-6, atol=1e-6)
    assert abs(ydot - (lp - lm) / (2 * h)) <= 1e-6 * (1 + abs(ydot))
    _, Hd = oracle.kmeans_fwd_rev(X, Cm, np.ones((k, d)), ybar)
    np.testing.assert_allclose(Hd, oracle.kmeans_hessdiag(X, Cm, ybar=ybar), rtol=1e-13)
