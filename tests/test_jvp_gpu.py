"""GPU parity of the forward-mode (JVP) scan rule against the FP64 oracle's
dual-number loop, through the C ABI: every operator, FP32 and FP64, sizes
spanning several tiles with ragged tails, the primal outputs alongside, and
the duality <ybar, J xdot> = <J^T ybar, xdot> against the GPU VJP.

Tolerances (relative L2): FP32 1e-4 (1e-3 beyond 2^24), FP64 1e-12.
"""
import numpy as np
import pytest
import torch

from paper_2202_10297_gb300 import synth

pytestmark = pytest.mark.gpu

SIZES = [1, 2, 7, 1000, 4095, 4096, 4097, 3 * 8192 + 5, 100001]


def rel_l2(x, ref):
    x = np.asarray(x, np.float64)
    ref = np.asarray(ref, np.float64)
    d = np.linalg.norm(ref)
    return float(np.linalg.norm(x - ref) / (d if d > 0 else 1.0))


def tol(dt, n=0):
    return 1e-12 if dt == np.float64 else (1e-3 if n > (1 << 24) else 1e-4)


@pytest.fixture(scope="module")
def A():
    from paper_2202_10297_gb300 import adpar
    adpar.lib()
    return adpar


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def inputs(op, n, dt, seed):
    g = synth.rng(seed)
    b = bd = None
    if op == "linrec":
        a, b, _, _ = synth.linrec(n, dt, seed=seed)
        bd = g.standard_normal(n).astype(dt)
    elif op == "mul":
        a = g.uniform(0.9, 1.1, n).astype(dt)
    elif op in ("min", "max"):
        a = (np.round(g.standard_normal(n) * 8) / 8).astype(dt)  # ties: the earlier element keeps the record
    else:
        a = g.standard_normal(n).astype(dt)
    ad = g.standard_normal(n).astype(dt)
    return a, b, ad, bd


@pytest.mark.parametrize("dt", [np.float32, np.float64])
@pytest.mark.parametrize("op", ["add", "mul", "min", "max", "linrec"])
@pytest.mark.parametrize("n", SIZES)
def test_jvp_scan_vs_oracle(A, oracle, op, dt, n):
    a, b, ad, bd = inputs(op, n, dt, seed=n * 3 + len(op))
    yd_a, yd_b, ys_a, ys_b = A.adpar_jvp_scan(op, dev(a), dev(ad), b=None if b is None else dev(b),
                                              bdot=None if bd is None else dev(bd), want_ys=True)
    ra, rb, rda, rdb = oracle.scan_jvp(op, a, ad, b, bd)
    assert rel_l2(yd_a.cpu().numpy(), rda) < tol(dt, n), (op, n, rel_l2(yd_a.cpu().numpy(), rda))
    assert rel_l2(ys_a.cpu().numpy(), ra) < tol(dt, n)
    if op == "linrec":
        assert rel_l2(yd_b.cpu().numpy(), rdb) < tol(dt, n)
        assert rel_l2(ys_b.cpu().numpy(), rb) < tol(dt, n)
    if op in ("min", "max"):
        np.testing.assert_array_equal(yd_a.cpu().numpy(), rda.astype(dt))  # a selected tangent, exactly


@pytest.mark.parametrize("op", ["mul", "linrec"])
def test_jvp_vjp_duality_on_gpu(A, op):
    """<ybar, J xdot> = <J^T ybar, xdot> with both sides from the library (FP64)."""
    n = 50021
    dt = np.float64
    a, b, ad, bd = inputs(op, n, dt, seed=5)
    g = synth.rng(6)
    ya, yb = g.standard_normal(n), g.standard_normal(n)
    w2 = op == "linrec"
    yd_a, yd_b, _, _ = A.adpar_jvp_scan(op, dev(a), dev(ad), b=dev(b) if w2 else None, bdot=dev(bd) if w2 else None)
    ab, bb, _ = A.adpar_vjp_scan(op, dev(a), dev(ya), b=dev(b) if w2 else None, ybar_b=dev(yb) if w2 else None)
    lhs = float(ya @ yd_a.cpu().numpy()) + (float(yb @ yd_b.cpu().numpy()) if w2 else 0.0)
    rhs = float(ab.cpu().numpy() @ ad) + (float(bb.cpu().numpy() @ bd) if w2 else 0.0)
    assert abs(lhs - rhs) <= 1e-10 * (1 + abs(lhs))


def test_jvp_scan_empty_and_errors(A):
    e = torch.empty(0, device="cuda")
    yd, _, _, _ = A.adpar_jvp_scan("add", e, e)
    assert yd.numel() == 0
    x = torch.zeros(9, device="cuda")
    with pytest.raises(A.AdparError):
        A.adpar_jvp_scan("add", x[1:], x[1:])  # not 16-byte aligned


@pytest.mark.slow
def test_jvp_linrec_full_size(A, oracle):
    n = 1 << 26
    a, b, ad, bd = inputs("linrec", n, np.float32, seed=synth.SEED_BASE + 1)
    yd_a, yd_b, _, _ = A.adpar_jvp_scan("linrec", dev(a), dev(ad), b=dev(b), bdot=dev(bd))
    _, _, rda, rdb = oracle.scan_jvp("linrec", a, ad, b, bd)
    assert rel_l2(yd_a.cpu().numpy(), rda) < 1e-3
    assert rel_l2(yd_b.cpu().numpy(), rdb) < 1e-3
