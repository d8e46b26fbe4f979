"""GPU parity of the scan VJP over wide elements (Sec. 5.2 with the general
d x d lin_o: the return sweep scans affine maps (d, C) with a D x D matrix C)
against the FP64 oracle's tape sweep with full D x D Jacobians, through the
C ABI: the 2x2 matrix linear recurrence (D = 6) and the linear recurrence as
a D = 2 element, FP32 and FP64, sizes spanning several tiles with ragged
tails, the recomputed scan, accumulation, n = 0, and agreement with the
scalar-coefficient LINREC kernels of adpar_vjp_scan.

Tolerances (relative L2): FP32 1e-4, FP64 1e-12.
"""
import numpy as np
import pytest
import torch

from paper_2202_10297_gb300 import synth

pytestmark = pytest.mark.gpu

SIZES = [1, 2, 3, 511, 512, 513, 4097, 100003]


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


def inputs(op, n, dt, seed):
    """Contractive elements: LINREC a in [0.9, 1]; 2x2 matrices 0.95 I plus a
    small random part (spectral radius below 1), so long scans stay bounded."""
    g = synth.rng(seed)
    if op == "linrec":
        a = np.stack([g.uniform(0.9, 1.0, n), g.standard_normal(n)], 1)
    else:
        M = 0.95 * np.eye(2).ravel() + 0.03 * g.standard_normal((n, 4))
        a = np.concatenate([M, g.standard_normal((n, 2))], 1)
    yb = g.standard_normal(a.shape)
    return a.astype(dt), yb.astype(dt)


@pytest.mark.parametrize("full", [False, True])
@pytest.mark.parametrize("dt", [np.float32, np.float64])
@pytest.mark.parametrize("op", ["linrec", "matrec2"])
@pytest.mark.parametrize("n", SIZES)
def test_scan_wide_matches_oracle(A, O, op, dt, n, full):
    """Both forms of the lin_o: blockwise C = I (x) N where the operator
    allows it (the default) and the full d x d matrix (ADPAR_FULL_LIN_O)."""
    a, yb = inputs(op, n, dt, seed=n % 89 + 3)
    ab, ys = A.adpar_vjp_scan_wide(op, dev(a), dev(yb), want_ys=True, full_lin_o=full)
    torch.cuda.synchronize()
    rab, rys = O.scan_wide_vjp(op, a, yb)
    assert rel_l2(ab.cpu().numpy(), rab) <= tol(dt), rel_l2(ab.cpu().numpy(), rab)
    assert rel_l2(ys.cpu().numpy(), rys) <= tol(dt)


@pytest.mark.parametrize("dt", [np.float32, np.float64])
def test_scan_wide_accumulates(A, O, dt):
    a, yb = inputs("matrec2", 30001, dt, seed=5)
    base = synth.rng(6).standard_normal(a.shape).astype(dt)
    ab, _ = A.adpar_vjp_scan_wide("matrec2", dev(a), dev(yb), abar=dev(base), accumulate=True)
    rab, _ = O.scan_wide_vjp("matrec2", a, yb, abar=base)
    assert rel_l2(ab.cpu().numpy(), rab) <= tol(dt)


def test_scan_wide_linrec_equals_scalar_rule(A):
    """D = 2 through full 2x2 Jacobians vs the library's scalar-coefficient
    LINREC kernels on the same data."""
    n = 1 << 20
    a, b, ya, yb = synth.linrec(n, np.float64, seed=synth.SEED_BASE + 1)
    ab, _ = A.adpar_vjp_scan_wide("linrec", dev(np.stack([a, b], 1)), dev(np.stack([ya, yb], 1)))
    sa, sb, _ = A.adpar_vjp_scan("linrec", dev(a), dev(ya), b=dev(b), ybar_b=dev(yb))
    ab = ab.cpu().numpy()
    assert rel_l2(ab[:, 0], sa.cpu().numpy()) <= 1e-12 and rel_l2(ab[:, 1], sb.cpu().numpy()) <= 1e-12


def test_scan_wide_edges(A):
    e = torch.empty(0, 6, device="cuda")
    ab, _ = A.adpar_vjp_scan_wide("matrec2", e, e)
    assert ab.numel() == 0
    L = A.lib()
    d = A.OpDesc(A.OP_MATREC2, A.F32, 2)  # MATREC2 needs width 6
    assert L.adpar_vjp_scan_wide(d, 4, None, None, None, None, 0, None, 0, None) == 1
    d = A.OpDesc(A.OP_MAX, A.F32, 1)  # not a wide operator
    assert L.adpar_vjp_scan_wide(d, 4, None, None, None, None, 0, None, 0, None) == 1


@pytest.mark.parametrize("full", [False, True])
def test_scan_wide_full_size_matrec(A, O, full):
    """The benchmark's case, n = 2^24 2x2-matrix elements FP32, against the
    oracle on every output, with both forms of the lin_o."""
    n = 1 << 24
    a, yb = inputs("matrec2", n, np.float32, seed=synth.SEED_BASE + 7)
    ab, ys = A.adpar_vjp_scan_wide("matrec2", dev(a), dev(yb), want_ys=True, full_lin_o=full)
    rab, rys = O.scan_wide_vjp("matrec2", a, yb)
    assert rel_l2(ab.cpu().numpy(), rab) <= 1e-4 and rel_l2(ys.cpu().numpy(), rys) <= 1e-4
