"""Full-size GPU parity against the FP64 oracle for the reduce_by_index,
scatter and batched workloads, at the sizes the benchmark times them.

* reduce_by_index (Sec. 5.1.2): n = 2^27 FP32 values N(0,1) into
  m in {256, 2^16, 2^22} bins, uniform and Zipf(1.1), 1 % of the indices out
  of range; + (a gather: bit-exact), max (argidx and adjoints bit-exact) and
  * (zero counts, lowest zeros and signs bit-exact, ln|nonzero product|
  within 1e-12, log-domain adjoints within the FP32 output's precision).
* scatter (Sec. 5.3): 2^26 FP32 cotangents gathered out of a 2^28
  destination through a duplicate-free index set, random and sorted:
  bit-exact (pure data movement).
* batch: the seeded 4096-segment plan (lengths 2^U[8,20], FP32/FP64 mixed,
  product reduce with 0/1/2 zeros then the linear-recurrence scan), run as
  one persistent launch; every 16th segment against the oracle.
"""
import numpy as np
import pytest
import torch

from paper_2202_10297_gb300 import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

HIST_N = 1 << 27


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


@pytest.mark.parametrize("m,dist", [(256, "uniform"), (256, "zipf"), (1 << 16, "uniform"), (1 << 16, "zipf"),
                                    (1 << 22, "uniform"), (1 << 22, "zipf")])
def test_hist_full_size(A, oracle, m, dist):
    vals, inds, hsbar = synth.hist(HIST_N, m, dist, seed=synth.SEED_BASE + 2)
    v, ix, hb = dev(vals), dev(inds), dev(hsbar)
    inr = (inds >= 0) & (inds < m)
    assert 0.009 < 1 - inr.mean() < 0.011  # 1 % out of range

    # +: a gather
    out = A.adpar_vjp_hist("add", ix, m, hb, vals=v)
    vb, _, _ = oracle.hist_vjp("add", vals, inds, m, hsbar)
    np.testing.assert_array_equal(out["valsbar"].cpu().numpy(), vb)
    del out, vb

    # max: per-bin argidx (lowest index on ties) and the adjoint bit-exact
    out = A.adpar_vjp_hist("max", ix, m, hb, vals=v, want_argidx=True)
    vb, _, arg = oracle.hist_vjp("max", vals, inds, m, hsbar)
    np.testing.assert_array_equal(out["argidx"].cpu().numpy(), arg)
    np.testing.assert_array_equal(out["valsbar"].cpu().numpy(), vb)
    del out, vb, arg

    # *: the per-bin product record, and the log-domain adjoints
    ref = oracle.hist_prod_vjp(vals, inds, m, hsbar)
    out = A.adpar_vjp_hist("mul", ix, m, hb, vals=v, want_aux=True)
    aux = out["aux"]
    np.testing.assert_array_equal(aux["nzero"], ref["nzero"])
    np.testing.assert_array_equal(aux["first_zero"], ref["first_zero"])
    np.testing.assert_array_equal(aux["sign"], ref["signnz"])
    ok = np.isfinite(ref["lognz"])
    err = np.abs(aux["log_abs_nz"][ok] - ref["lognz"][ok]) / np.maximum(1, np.abs(ref["lognz"][ok]))
    assert err.max() < 1e-12
    # the hot bin (most members): the longest product, checked on its own
    counts = np.bincount(inds[inr], minlength=m)
    hot = int(np.argmax(counts))
    assert abs(aux["log_abs_nz"][hot] - ref["lognz"][hot]) <= 1e-12 * abs(ref["lognz"][hot])
    # values: correctly rounded FP32 (these long products underflow to 0)
    got = out["valsbar"].cpu().numpy()
    refv = ref["valsbar"].astype(np.float32)
    assert rel_l2(got, refv) < 1e-4 or (np.abs(refv).max() == 0 and np.abs(got).max() == 0)
    del out
    lg = A.adpar_vjp_hist("mul", ix, m, hb, vals=v, logdomain=True, want_sign=True)
    gl = lg["valsbar"].cpu().numpy().astype(np.float64)
    fin = np.isfinite(ref["log"])
    np.testing.assert_array_equal(np.isfinite(gl), fin)
    # an FP32 output of a logarithm of magnitude L carries about L * 2^-24
    assert np.all(np.abs(gl[fin] - ref["log"][fin]) <= 1e-6 * np.maximum(1, np.abs(ref["log"][fin])))
    np.testing.assert_array_equal(lg["sign"].cpu().numpy(), ref["sign"])


@pytest.mark.parametrize("sort", [False, True])
def test_scatter_full_size(A, oracle, sort):
    n, m = 1 << 28, 1 << 26
    is_, ysbar, _ = synth.scatter(n, m, sort=sort, seed=synth.SEED_BASE + 2)
    yt = dev(ysbar)
    xs, vs = A.adpar_vjp_scatter(dev(is_), yt)
    xb, vb, _ = oracle.scatter_vjp(n, is_, ysbar)
    np.testing.assert_array_equal(vs.cpu().numpy().astype(np.float64), vb)
    np.testing.assert_array_equal(xs.cpu().numpy().astype(np.float64), xb)


def test_batch_4096_segments_against_oracle(oracle):
    from paper_2202_10297_gb300 import adpar as A
    from paper_2202_10297_gb300 import batch as B
    A.lib()
    lens, dts, zs = synth.batch_plan(4096, seed=synth.SEED_BASE + 3)
    assert lens.min() >= 256 and lens.max() <= 1 << 20
    checked = set(range(0, 4096, 16))
    gen = torch.Generator(device="cuda")
    gen.manual_seed(5)
    segs, host = [], {}
    for i, (L, dt, z) in enumerate(zip(lens, dts, zs)):
        L, npdt = int(L), (np.float64 if dt else np.float32)
        if i in checked:
            # config-1 product inputs (U[0.5, 1.5) with z zeros) and config-2a
            # linear-recurrence inputs, seeded per segment
            x, _ = synth.prod_reduce(L, int(z), dtype=npdt, seed=synth.SEED_BASE + 100 + i)
            a, b, ya, yb = synth.linrec(L, npdt, seed=synth.SEED_BASE + 10000 + i)
            yp = float(synth.rng(i).normal())
            host[i] = dict(x=x, a=a, b=b, ya=ya, yb=yb, yp=yp)
            s = dict(x=dev(x), a=dev(a), b=dev(b), ybar_a=dev(ya), ybar_b=dev(yb), ybar_prod=yp, aux=True)
        else:
            # the other segments fill the launch; their results are not compared
            tdt = torch.float64 if dt else torch.float32
            x = torch.rand(L, dtype=tdt, device="cuda", generator=gen) + 0.5
            a = torch.rand(L, dtype=tdt, device="cuda", generator=gen) * 0.1 + 0.9
            s = dict(x=x, a=a, b=torch.randn(L, dtype=tdt, device="cuda", generator=gen),
                     ybar_a=torch.randn(L, dtype=tdt, device="cuda", generator=gen),
                     ybar_b=torch.randn(L, dtype=tdt, device="cuda", generator=gen), ybar_prod=1.0, aux=True)
        segs.append(s)
    bt = B.Batch(segs)
    g = bt.graph()
    g.replay()
    torch.cuda.synchronize()
    assert bt.status() == A.OK
    recs = bt.aux_records()
    for i in sorted(checked):
        h, s = host[i], segs[i]
        L = len(h["x"])
        f64 = h["x"].dtype == np.float64
        tol = 1e-12 if f64 else 1e-4
        tiny = np.finfo(np.float64 if f64 else np.float32).smallest_subnormal
        ref = oracle.prod_reduce_vjp(h["x"], h["yp"])
        assert recs[i]["nzero"] == ref["nzero"] and recs[i]["first_zero"] == ref["first_zero"], i
        if ref["nzero"] == 0:
            assert recs[i]["sign"] == ref["signnz"], i
            assert abs(recs[i]["log_abs_nz"] - ref["lognz"]) <= 1e-12 * max(1.0, abs(ref["lognz"])), i
        got = s["xbar"].cpu().numpy().astype(np.float64)
        refv = ref["abar"].astype(h["x"].dtype).astype(np.float64)  # correctly rounded to the output type
        assert np.linalg.norm(got - refv) <= tol * np.linalg.norm(refv) + 2 * tiny * np.sqrt(L), (i, L, f64)
        rab, rbb, _, _ = oracle.scan_vjp("linrec", h["a"], h["ya"], h["b"], h["yb"])
        assert rel_l2(s["abar"].cpu().numpy(), rab) < tol, (i, L, f64)
        assert rel_l2(s["bbar"].cpu().numpy(), rbb) < tol, (i, L, f64)
