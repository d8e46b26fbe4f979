"""GPU parity of the vectorised scan VJP (Sec. 5.2: a scan over d-vectors with
an elementwise operator is d independent column scans) against the FP64
oracle applied column by column (the paper's transpose / map / transpose
rule), through the C ABI: every operator, FP32 and FP64, shapes with ragged
chunk and column tails, accumulation, ADD without the input, empty shapes.

Tolerances (relative L2): FP32 1e-4, FP64 1e-12; min/max positions exact.
"""
import numpy as np
import pytest
import torch

from paper_2202_10297_gb300 import synth

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1), (33, 7), (100, 256), (1000, 300), (4101, 129)]


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


def inputs(op, n, d, dt, seed):
    g = synth.rng(seed)
    b = yb = None
    if op == "linrec":
        a = g.uniform(0.9, 1.0, (n, d)).astype(dt)
        b = g.standard_normal((n, d)).astype(dt)
        yb = g.standard_normal((n, d)).astype(dt)
    elif op == "mul":
        a = g.uniform(0.9, 1.1, (n, d)).astype(dt)
    elif op in ("min", "max"):
        a = (np.round(g.standard_normal((n, d)) * 8) / 8).astype(dt)  # ties
    else:
        a = g.standard_normal((n, d)).astype(dt)
    ya = g.standard_normal((n, d)).astype(dt)
    return a, b, ya, yb


def oracle_columns(oracle, op, a, b, ya, yb, abar=None, bbar=None):
    n, d = ya.shape
    ra, rb = np.zeros((n, d)), np.zeros((n, d))
    for j in range(d):
        x, y, z = oracle.scan_vjp(op, a[:, j], ya[:, j], None if b is None else b[:, j],
                                  None if yb is None else yb[:, j],
                                  abar=None if abar is None else abar[:, j],
                                  bbar=None if bbar is None else bbar[:, j])[:3]
        ra[:, j] = x
        if y is not None:
            rb[:, j] = y
    return ra, rb


@pytest.mark.parametrize("dt", [np.float32, np.float64])
@pytest.mark.parametrize("op", ["add", "mul", "min", "max", "linrec"])
@pytest.mark.parametrize("shape", SHAPES)
def test_scan_vec_vs_oracle(A, oracle, op, dt, shape):
    n, d = shape
    a, b, ya, yb = inputs(op, n, d, dt, seed=n * 7 + d + len(op))
    ab, bb, work = A.adpar_vjp_scan_vec(op, dev(a), dev(ya), b=None if b is None else dev(b),
                                        ybar_b=None if yb is None else dev(yb))
    torch.cuda.synchronize()
    assert A.adpar_workspace_status(work) == A.OK
    ra, rb = oracle_columns(oracle, op, a, b, ya, yb)
    tol = 1e-12 if dt == np.float64 else 1e-4
    got = ab.cpu().numpy()
    assert rel_l2(got, ra) < tol, (op, shape, rel_l2(got, ra))
    if op == "linrec":
        assert rel_l2(bb.cpu().numpy(), rb) < tol
    if op in ("min", "max"):
        np.testing.assert_array_equal(got != 0, ra != 0)


@pytest.mark.parametrize("op", ["max", "linrec"])
def test_scan_vec_accumulates(A, oracle, op):
    n, d = 777, 65
    a, b, ya, yb = inputs(op, n, d, np.float64, seed=11)
    base = synth.normal(n * d, np.float64, seed=12).reshape(n, d)
    ab0 = dev(base)
    bb0 = dev(base[::-1].copy()) if op == "linrec" else None
    A.adpar_vjp_scan_vec(op, dev(a), dev(ya), b=None if b is None else dev(b), ybar_b=None if yb is None else dev(yb),
                         abar=ab0, bbar=bb0, accumulate=True)
    ra, rb = oracle_columns(oracle, op, a, b, ya, yb, abar=base,
                            bbar=base[::-1].copy() if op == "linrec" else None)
    assert rel_l2(ab0.cpu().numpy(), ra) < 1e-12
    if op == "linrec":
        assert rel_l2(bb0.cpu().numpy(), rb) < 1e-12


def test_scan_vec_add_needs_no_input_and_empty(A, oracle):
    n, d = 300, 40
    _, _, ya, _ = inputs("add", n, d, np.float32, seed=13)
    ab, _, _ = A.adpar_vjp_scan_vec("add", None, dev(ya))
    ref = np.flip(np.cumsum(np.flip(ya.astype(np.float64), 0), 0), 0)  # suffix sums down each column
    assert rel_l2(ab.cpu().numpy(), ref) < 1e-6
    e = torch.empty((0, 5), device="cuda")
    ab, _, _ = A.adpar_vjp_scan_vec("add", None, e)
    assert ab.numel() == 0
