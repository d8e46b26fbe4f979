"""GPU parity of the k-means cost and gradient (Sec. 7.4, squared distances).

The argmin from the TF32 tensor-core distances is certified, so it must
equal the FP64 oracle's argmin (lowest k on ties) bit-exactly on every
point; the loss within 1e-5 and Cbar within 1e-4 relative L2.
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


@pytest.fixture(scope="module")
def A():
    from paper_2202_10297_gb300 import adpar
    adpar.lib()
    return adpar


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def run_and_check(A, oracle, X, Cm, ybar=1.5):
    out = A.adpar_kmeans_vjp(dev(X), dev(Cm), ybar=ybar, want_argmin=True)
    loss, arg, _, cb = oracle.kmeans(X, Cm, ybar)
    assert A.adpar_workspace_status(out["work"]) == A.OK
    np.testing.assert_array_equal(out["argmin"].cpu().numpy(), arg)
    assert abs(out["loss"].item() - loss) <= 1e-5 * abs(loss)
    assert rel_l2(out["Cbar"].cpu().numpy(), cb) < 1e-4


@pytest.mark.parametrize("N,k", [(1, 32), (127, 32), (128, 64), (1000, 256), (4096 + 7, 256), (50001, 128),
                                 (20000, 256)])
def test_kmeans_small(A, oracle, N, k):
    X, Cm = synth.kmeans(N, 32, k, seed=N + k)
    run_and_check(A, oracle, X, Cm)


def test_kmeans_forced_ties(A, oracle):
    """Duplicate centroids tie exactly: the lower k must win, as in the oracle."""
    X, Cm = synth.kmeans(3000, 32, 64, seed=3)
    Cm[40] = Cm[7]
    Cm[63] = Cm[0]
    X[:100] = Cm[7]  # points sitting on a duplicated centroid
    X[100:110] = 0.5 * (Cm[1] + Cm[2])  # equidistant from two centroids
    run_and_check(A, oracle, X, Cm)


def test_kmeans_forward_only_and_accumulate(A, oracle):
    X, Cm = synth.kmeans(5000, 32, 96, seed=4)
    out = A.adpar_kmeans_vjp(dev(X), dev(Cm), want_grad=False)
    loss, _, _, cb = oracle.kmeans(X, Cm, 2.0)
    assert abs(out["loss"].item() - loss) <= 1e-5 * abs(loss)
    base = synth.normal(96 * 32, np.float32, seed=5).reshape(96, 32)
    cbt = dev(base)
    A.adpar_kmeans_vjp(dev(X), dev(Cm), ybar=2.0, Cbar=cbt, accumulate=True)
    assert rel_l2(cbt.cpu().numpy(), base + cb) < 1e-4


def test_kmeans_empty(A):
    X = torch.zeros(0, 32, device="cuda")
    Cm = torch.randn(64, 32, device="cuda")
    out = A.adpar_kmeans_vjp(X, Cm)
    assert out["loss"].item() == 0.0
    assert torch.all(out["Cbar"] == 0)


@pytest.mark.slow
def test_kmeans_full_size(A, oracle):
    """N = 2^20, d = 32, k = 256 (the workload size): every argmin bit-exact."""
    X, Cm = synth.kmeans(1 << 20, 32, 256, seed=synth.SEED_BASE + 4)
    run_and_check(A, oracle, X, Cm, ybar=1.0)


@pytest.mark.parametrize("N,k", [(1000, 32), (20000, 256), (50001, 128)])
def test_kmeans_hessdiag(A, oracle, N, k):
    """Hessian diagonal in C (argmins held fixed) from the gradient call's
    counts: exactly 2 ybar cnt_k, as the FP64 oracle gives it (the certified
    argmin matches the oracle's, and counts are exact integers in FP32)."""
    X, Cm = synth.kmeans(N, 32, k, seed=N + 2 * k)
    out = A.adpar_kmeans_vjp(dev(X), dev(Cm), ybar=1.5)
    H = A.adpar_kmeans_hessdiag(k, 1.5, out["work"])
    ref = oracle.kmeans_hessdiag(X, Cm, ybar=1.5)
    np.testing.assert_array_equal(H.cpu().numpy(), ref.astype(np.float32))
    base = torch.ones(k, 32, device="cuda")
    H2 = A.adpar_kmeans_hessdiag(k, 1.5, out["work"], Hdiag=base, accumulate=True)
    np.testing.assert_array_equal(H2.cpu().numpy(), ref.astype(np.float32) + 1)
