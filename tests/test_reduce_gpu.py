"""GPU parity of the reduce VJP (Sec. 5.1, 5.1.1) against the FP64 oracle, through the C ABI.

* rule: zero count and lowest zero index bit-exact; ln|p_nz| and every
ln|abar_i| within 1e-12 relative (the products underflow FP64, Sec. 5.1.1's
y is about 1e-1287 at n = 65536); signs bit-exact; value mode equal to the
correctly rounded oracle values (0 there), and within 1e-12 (FP64) / 1e-4
(FP32) relative L2 on a representable case.
min/max: argidx and y bit-exact, ties to the lowest index.
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


def check_log(got_log, got_sign, ref):
    fin = np.isfinite(ref["log"])
    np.testing.assert_array_equal(np.isfinite(got_log), fin)
    err = np.abs(got_log[fin] - ref["log"][fin]) / np.maximum(1.0, np.abs(ref["log"][fin]))
    assert err.size == 0 or err.max() < 1e-12, err.max()
    np.testing.assert_array_equal(got_sign, ref["sign"])


@pytest.mark.parametrize("nz", [0, 1, 2])
def test_prod_reduce_config_logdomain(A, oracle, nz):
    """n = 65536 FP64 from U[0.5,1.5) with 0/1/2 zeros, ybar = 1 (the latency-bound workload)."""
    a, zpos = synth.prod_reduce(65536, nz)
    ref = oracle.prod_reduce_vjp(a, 1.0)
    out = A.adpar_vjp_reduce("mul", dev(a), 1.0, logdomain=True, want_sign=True, want_aux=True, want_y=True)
    aux = out["aux"]
    assert aux.nzero == ref["nzero"] and aux.first_zero == ref["first_zero"]
    assert abs(aux.log_abs_nz - ref["lognz"]) <= 1e-12 * abs(ref["lognz"])
    assert aux.sign == ref["signnz"]
    assert out["y"].item() == ref["y"] == 0.0
    check_log(out["abar"].cpu().numpy(), out["sign"].cpu().numpy(), ref)
    # value mode: every contribution underflows to exactly the oracle's value
    val = A.adpar_vjp_reduce("mul", dev(a), 1.0)["abar"].cpu().numpy()
    np.testing.assert_array_equal(val, ref["abar"])


@pytest.mark.parametrize("dt", [np.float32, np.float64])
@pytest.mark.parametrize("nz", [0, 1, 2, 3])
@pytest.mark.parametrize("n", [1, 2, 3, 7, 1000, 4097, 100003, (1 << 18) + 1, 1000003])
def test_prod_reduce_sizes(A, oracle, dt, nz, n):
    """Sizes from 1 to past 2^20: one and many blocks in the reduce and the map."""
    g = synth.rng(n * 10 + nz)
    a = g.uniform(0.5, 1.5, n) * np.where(g.random(n) < 0.3, -1.0, 1.0)
    if n < 200:  # representable products: check values too
        pass
    else:
        a = a * math.exp(-np.mean(np.log(np.abs(a))))  # keep the product near 1
    if nz:
        a[g.choice(n, size=min(nz, n), replace=False)] = 0.0
    a = a.astype(dt)
    ybar = -0.75
    ref = oracle.prod_reduce_vjp(a, ybar)
    out = A.adpar_vjp_reduce("mul", dev(a), ybar, want_aux=True)
    tol = 1e-12 if dt == np.float64 else 1e-4
    assert rel_l2(out["abar"].cpu().numpy(), ref["abar"]) < tol
    assert out["aux"].nzero == ref["nzero"] and out["aux"].first_zero == ref["first_zero"]
    lg = A.adpar_vjp_reduce("mul", dev(a), ybar, logdomain=True, want_sign=True)
    got = lg["abar"].cpu().numpy().astype(np.float64)
    if dt == np.float64:
        check_log(got, lg["sign"].cpu().numpy(), ref)
    else:
        fin = np.isfinite(ref["log"])
        np.testing.assert_array_equal(np.isfinite(got), fin)
        assert np.all(np.abs(got[fin] - ref["log"][fin]) <= 1e-5 * np.maximum(1, np.abs(ref["log"][fin])))
        np.testing.assert_array_equal(lg["sign"].cpu().numpy(), ref["sign"])


@pytest.mark.parametrize("n", [65536, 1 << 20])
def test_prod_reduce_clears_status_of_a_dirty_workspace(A, n):
    """The workspace needs no initialisation: a call leaves its status word ok
    even in a workspace full of stale bytes."""
    a, _ = synth.prod_reduce(n, 1)
    work = torch.full((A.adpar_workspace_size(A.RULE_REDUCE, A.OP_MUL, A.F64, n),), 0xFF, dtype=torch.uint8,
                      device="cuda")
    A.adpar_vjp_reduce("mul", dev(a), 1.0, work=work)
    torch.cuda.synchronize()
    assert A.adpar_workspace_status(work) == A.OK


def test_prod_reduce_accumulate(A, oracle):
    for nz in (0, 1, 2):
        a, _ = synth.prod_reduce(1024, nz, seed=5)
        a = a * math.exp(0.04523)
        base = synth.normal(1024, np.float64, seed=6)
        ref = oracle.prod_reduce_vjp(a, 2.0, abar=base)
        ab = dev(base)
        A.adpar_vjp_reduce("mul", dev(a), 2.0, abar=ab, accumulate=True)
        assert rel_l2(ab.cpu().numpy(), ref["abar"]) < 1e-12


@pytest.mark.parametrize("dt", [np.float32, np.float64])
@pytest.mark.parametrize("op", ["min", "max"])
@pytest.mark.parametrize("n", [1, 2, 5, 4096, 4099, 1000003])
def test_minmax_reduce_ties(A, oracle, op, dt, n):
    g = synth.rng(n + 17)
    a = (np.round(g.standard_normal(n) * 4) / 4).astype(dt)  # many exact ties
    out = A.adpar_vjp_reduce(op, dev(a), 1.5, want_y=True, want_argidx=True)
    y, ab, arg = oracle.reduce_vjp(op, a, 1.5)
    assert out["argidx"].item() == arg
    assert out["y"].item() == y
    np.testing.assert_array_equal(out["abar"].cpu().numpy(), ab)


def test_minmax_reduce_accumulate_and_empty(A, oracle):
    a = synth.normal(5000, np.float32, seed=3)
    base = synth.normal(5000, np.float32, seed=4)
    ab = dev(base)
    A.adpar_vjp_reduce("max", dev(a), 2.0, abar=ab, accumulate=True)
    _, ref, _ = oracle.reduce_vjp("max", a, 2.0, abar=base)
    np.testing.assert_allclose(ab.cpu().numpy(), ref, rtol=1e-6)
    e = torch.empty(0, device="cuda")
    out = A.adpar_vjp_reduce("max", e, 1.0, want_argidx=True, want_y=True)
    assert out["argidx"].item() == -1 and out["y"].item() == -math.inf


@pytest.mark.parametrize("dt", [np.float32, np.float64])
def test_add_reduce(A, oracle, dt):
    n = 77777
    a = synth.normal(n, dt, seed=9)
    out = A.adpar_vjp_reduce("add", dev(a), 0.25, want_y=True)
    y, ab, _ = oracle.reduce_vjp("add", a, 0.25)
    np.testing.assert_array_equal(out["abar"].cpu().numpy(), ab)
    assert abs(out["y"].item() - y) <= (1e-4 if dt == np.float32 else 1e-12) * np.abs(a).sum()


@pytest.mark.slow
def test_argmax_full_size(A, oracle):
    """2^28 FP32 N(0,1): argmax index bit-exact, lowest index on ties."""
    n = 1 << 28
    a = synth.normal(n, np.float32, seed=synth.SEED_BASE + 1)
    out = A.adpar_vjp_reduce("max", dev(a), 1.0, want_argidx=True, want_y=True)
    assert out["argidx"].item() == int(np.argmax(a))
    assert out["y"].item() == float(a.max())
