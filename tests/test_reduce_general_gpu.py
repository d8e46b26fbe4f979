"""GPU parity of the general reduce rule (Sec. 5.1.1: l_i and r_i from two
exclusive scans, then d(l_i (.) a_i (.) r_i)/d a_i) against the FP64 oracle's
plain tape sweep, through the C ABI: every operator (LINREC has no special
rule), FP32 and FP64, sizes spanning several tiles with ragged tails, the
recomputed y, accumulation, n = 0, and agreement with the special rules.

Tolerances (relative L2): FP32 1e-4, FP64 1e-12; min/max positions exact.
"""
import numpy as np
import pytest
import torch

from paper_2202_10297_gb300 import synth

pytestmark = pytest.mark.gpu

SIZES = [1, 2, 7, 1000, 2047, 2048, 2049, 8192 + 3, 3 * 8192 + 5, 100001]


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


def inputs(op, n, dt, seed):
    g = synth.rng(seed)
    b = None
    if op == "linrec":
        a, b, _, _ = synth.linrec(n, dt, seed=seed)
    elif op == "mul":
        # geometric mean near 1, so the products of all other elements stay in range
        a = (g.uniform(0.5, 1.5, n) * np.exp(0.04523)).astype(dt)
        if n > 20:
            a[g.choice(n, size=1, replace=False)] = 0
    elif op in ("min", "max"):
        a = (np.round(g.standard_normal(n) * 8) / 8).astype(dt)  # ties
    else:
        a = g.standard_normal(n).astype(dt)
    return a, b


@pytest.mark.parametrize("dt", [np.float32, np.float64])
@pytest.mark.parametrize("op", ["add", "mul", "min", "max", "linrec"])
@pytest.mark.parametrize("n", SIZES)
def test_reduce_general_vs_oracle(A, oracle, op, dt, n):
    if op == "mul" and dt == np.float32 and n > 5000:
        pytest.skip("products of 10^4+ FP32 factors leave the FP32 range")
    a, b = inputs(op, n, dt, seed=n * 5 + len(op))
    ya, yb = 0.75, -1.25
    ab, bb, y = A.adpar_vjp_reduce_general(op, dev(a), ya, b=None if b is None else dev(b), ybar_b=yb)
    ry, rab, rbb = oracle.reduce_general_vjp(op, a, ya, b=b, ybar_b=yb)
    got = ab.cpu().numpy()
    assert rel_l2(got, rab) < tol(dt), (op, n, rel_l2(got, rab))
    yv = y.cpu().numpy()
    assert rel_l2(yv, np.array(ry)) < tol(dt)
    if op == "linrec":
        assert rel_l2(bb.cpu().numpy(), rbb) < tol(dt)
    if op in ("min", "max"):
        np.testing.assert_array_equal(got != 0, rab != 0)  # the lowest index of the extremum, exactly


@pytest.mark.parametrize("op", ["add", "max", "linrec"])
def test_reduce_general_accumulates(A, oracle, op):
    n = 20011
    dt = np.float64
    a, b = inputs(op, n, dt, seed=3)
    base = synth.normal(n, dt, seed=4)
    base_b = base[::-1].copy()
    ab0 = dev(base)
    bb0 = dev(base_b) if op == "linrec" else None
    A.adpar_vjp_reduce_general(op, dev(a), 1.5, b=None if b is None else dev(b), ybar_b=0.5, abar=ab0, bbar=bb0,
                               accumulate=True)
    _, rab, rbb = oracle.reduce_general_vjp(op, a, 1.5, b=b, ybar_b=0.5, abar=base,
                                            bbar=base_b if op == "linrec" else None)
    assert rel_l2(ab0.cpu().numpy(), rab) < 1e-12
    if op == "linrec":
        assert rel_l2(bb0.cpu().numpy(), rbb) < 1e-12


def test_reduce_general_empty_gives_neutral(A):
    e = torch.empty(0, dtype=torch.float64, device="cuda")
    _, _, y = A.adpar_vjp_reduce_general("linrec", e, 1.0, b=e, ybar_b=1.0)
    assert y.cpu().tolist() == [1.0, 0.0]
    _, _, y = A.adpar_vjp_reduce_general("max", torch.empty(0, device="cuda"), 1.0)
    assert y.item() == float("-inf")


@pytest.mark.parametrize("op", ["add", "max", "min", "mul"])
def test_reduce_general_agrees_with_special_rules(A, op):
    """Where a special rule exists (Sec. 5.1.1), the general rule gives the same adjoint."""
    n = 50021
    a, _ = inputs(op, n, np.float64, seed=9)
    at = dev(a)
    g, _, _ = A.adpar_vjp_reduce_general(op, at, 2.0)
    sp = A.adpar_vjp_reduce(op, at, 2.0)
    s = sp["abar"] if isinstance(sp, dict) else sp[0]
    assert rel_l2(g.cpu().numpy(), s.cpu().numpy()) < 1e-12


@pytest.mark.slow
def test_reduce_general_linrec_full_size(A, oracle):
    """n = 2^26 FP32 pairs (the linear-recurrence benchmark size)."""
    n = 1 << 26
    a, b, _, _ = synth.linrec(n, np.float32, seed=synth.SEED_BASE + 1)
    ab, bb, y = A.adpar_vjp_reduce_general("linrec", dev(a), 0.5, b=dev(b), ybar_b=1.0)
    ry, rab, rbb = oracle.reduce_general_vjp("linrec", a, 0.5, b=b, ybar_b=1.0)
    assert rel_l2(ab.cpu().numpy(), rab) < 1e-3
    assert rel_l2(bb.cpu().numpy(), rbb) < 1e-3


@pytest.mark.parametrize("dt", [np.float32, np.float64])
@pytest.mark.parametrize("n", [1, 31, 33, 2049, 4097, 3 * 4096 + 5, 100001, (1 << 20) + 3])
@pytest.mark.parametrize("minimal", [False, True])
def test_reduce_general_linrec_both_workspaces(A, oracle, dt, n, minimal):
    """LINREC by the general rule on per-thread runs (full workspace: run
    carries and products, the product of the later a from a reverse scan of
    the runs' products) and on the scan engine (the minimal size), ragged
    sizes around run and tile edges, against the oracle."""
    a, b = inputs("linrec", n, dt, seed=n * 7 + 3)
    ya, yb = -0.5, 1.75
    code = A.F64 if dt == np.float64 else A.F32
    flags = A.RULE_REDUCE_GENERAL | (A.WS_MINIMAL if minimal else 0)
    work = A.workspace(A.adpar_workspace_size(flags, A.OP_LINREC, code, n))
    ab, bb, y = A.adpar_vjp_reduce_general("linrec", dev(a), ya, b=dev(b), ybar_b=yb, work=work)
    assert A.adpar_workspace_status(work) == A.OK
    ry, rab, rbb = oracle.reduce_general_vjp("linrec", a, ya, b=b, ybar_b=yb)
    assert rel_l2(ab.cpu().numpy(), rab) < tol(dt)
    assert rel_l2(bb.cpu().numpy(), rbb) < tol(dt)
    assert rel_l2(y.cpu().numpy(), np.array(ry)) < tol(dt)
