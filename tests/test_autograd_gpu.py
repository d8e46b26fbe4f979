"""torch.autograd wrappers: gradcheck in FP64 against finite differences, and
FP32 gradients against the FP64 oracle.  Also checks the memory policy:
the forward passes save only their inputs (no tape of intermediates)."""
import numpy as np
import pytest
import torch
from torch.autograd import gradcheck

from paper_2202_10297_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def AG():
    from paper_2202_10297_gb300 import adpar, autograd
    adpar.lib()
    return autograd


def t64(x, grad=True):
    return torch.tensor(np.asarray(x, np.float64), device="cuda", requires_grad=grad)


def rel_l2(x, ref):
    x = np.asarray(x, np.float64)
    ref = np.asarray(ref, np.float64)
    d = np.linalg.norm(ref)
    return float(np.linalg.norm(x - ref) / (d if d > 0 else 1.0))


@pytest.mark.parametrize("op", ["add", "mul", "max", "min"])
def test_gradcheck_scan(AG, op):
    g = synth.rng(1)
    a = g.uniform(0.6, 1.4, 37) if op == "mul" else g.permutation(37).astype(np.float64) + g.uniform(0, 0.5, 37)
    assert gradcheck(lambda x: AG.scan(op, x), (t64(a),), eps=1e-6, atol=1e-8, nondet_tol=1e-12)


def test_gradcheck_linrec(AG):
    g = synth.rng(2)
    a = t64(g.uniform(0.9, 1.0, 29))
    b = t64(g.standard_normal(29))
    assert gradcheck(lambda x, y: AG.scan("linrec", x, y), (a, b), eps=1e-6, atol=1e-8)


@pytest.mark.parametrize("op", ["add", "mul", "max", "min"])
def test_forward_ad_scan_gradcheck(AG, op):
    """Forward mode through the Function's jvp (the library's dual-number scan),
    checked by torch against numerical directional derivatives."""
    g = synth.rng(3)
    a = g.uniform(0.6, 1.4, 37) if op == "mul" else g.permutation(37).astype(np.float64) + g.uniform(0, 0.5, 37)
    assert gradcheck(lambda x: AG.scan(op, x), (t64(a),), eps=1e-6, atol=1e-8, nondet_tol=1e-12,
                     check_forward_ad=True, check_backward_ad=False, check_undefined_grad=False,
                     check_batched_grad=False)


def test_forward_ad_linrec_vs_oracle(AG, oracle):
    """torch.autograd.forward_ad dual tensors through scan("linrec") give the
    oracle's dual-number tangents (FP64, several tiles)."""
    import torch.autograd.forward_ad as fwAD
    g = synth.rng(4)
    n = 20011
    a = g.uniform(0.9, 1.0, n)
    b, ad, bd = g.standard_normal(n), g.standard_normal(n), g.standard_normal(n)
    with fwAD.dual_level():
        da = fwAD.make_dual(t64(a, False), t64(ad, False))
        db = fwAD.make_dual(t64(b, False), t64(bd, False))
        ya, yb = AG.scan("linrec", da, db)
        ta, tb = fwAD.unpack_dual(ya).tangent, fwAD.unpack_dual(yb).tangent
    _, _, rda, rdb = oracle.scan_jvp("linrec", a, ad, b, bd)
    assert rel_l2(ta.cpu().numpy(), rda) < 1e-12
    assert rel_l2(tb.cpu().numpy(), rdb) < 1e-12


@pytest.mark.parametrize("op,zeros", [("add", 0), ("mul", 0), ("mul", 1), ("mul", 2), ("max", 0), ("min", 0)])
def test_gradcheck_reduce(AG, op, zeros):
    g = synth.rng(3)
    a = g.uniform(0.6, 1.4, 41)
    if op in ("max", "min"):
        a = g.permutation(41) + g.uniform(0, 0.5, 41)
    a[:zeros] = 0.0
    assert gradcheck(lambda x: AG.reduce(op, x), (t64(a),), eps=1e-6, atol=1e-8)


@pytest.mark.parametrize("op", ["add", "mul", "max", "min"])
def test_gradcheck_reduce_by_index(AG, op):
    g = synth.rng(4)
    n, m = 60, 7
    vals = g.uniform(0.6, 1.4, n) if op == "mul" else g.permutation(n) + g.uniform(0, 0.5, n)
    inds = torch.tensor(g.integers(-1, m + 1, n), dtype=torch.int32, device="cuda")
    # the + and * forwards combine bins with atomics, so their FP64 rounding
    # order varies between calls: ~1e-14 / (2 eps) of finite-difference noise
    assert gradcheck(lambda v: AG.reduce_by_index(op, v, inds, m), (t64(vals),), eps=1e-6, atol=1e-6,
                     nondet_tol=1e-12)


def test_gradcheck_scatter(AG):
    g = synth.rng(5)
    is_ = torch.tensor(synth.permutation_prefix(50, 12, seed=6), dtype=torch.int64, device="cuda")
    xs, vs = t64(g.standard_normal(50)), t64(g.standard_normal(12))
    assert gradcheck(lambda x, v: AG.scatter(x, is_, v), (xs, vs), eps=1e-6, atol=1e-8)


@pytest.mark.parametrize("gfun,width", [("gather", 1), ("scale", 1), ("sqdist_row", 3)])
def test_gradcheck_map_acc(AG, gfun, width):
    g = synth.rng(7)
    na, nj = 9, 40
    as_ = t64(g.standard_normal(na * width))
    is_ = torch.tensor(g.integers(0, na, nj), dtype=torch.int32, device="cuda")
    if gfun == "gather":
        f = lambda a: AG.map_acc(gfun, a, is_)
        args = (as_,)
    else:
        ws = t64(g.standard_normal(nj * width))
        f = lambda a, w: AG.map_acc(gfun, a, is_, w, width)
        args = (as_, ws)
    assert gradcheck(f, args, eps=1e-6, atol=1e-6, nondet_tol=1e-12)  # atomic sums: see above


def test_kmeans_autograd_vs_oracle(AG, oracle):
    X, Cm = synth.kmeans(30000, 32, 256, seed=9)
    Xt = torch.from_numpy(X).cuda()
    Ct = torch.from_numpy(Cm).cuda().requires_grad_(True)
    loss = AG.kmeans_loss(Xt, Ct)
    (0.5 * loss).backward()
    rl, _, _, rcb = oracle.kmeans(X, Cm, 0.5)
    assert abs(loss.item() - rl / 0.5 * 0.5) <= 1e-5 * abs(rl)
    assert rel_l2(Ct.grad.cpu().numpy(), rcb) < 1e-4


def test_fp32_scan_grad_vs_oracle(AG, oracle):
    a, b, ya, yb = synth.linrec(100003, np.float32, seed=10)
    at = torch.from_numpy(a).cuda().requires_grad_(True)
    bt = torch.from_numpy(b).cuda().requires_grad_(True)
    A_, B_ = AG.scan("linrec", at, bt)
    ((A_ * torch.from_numpy(ya).cuda()).sum() + (B_ * torch.from_numpy(yb).cuda()).sum()).backward()
    rab, rbb, _, _ = oracle.scan_vjp("linrec", a, ya, b, yb)
    assert rel_l2(at.grad.cpu().numpy(), rab) < 1e-4
    assert rel_l2(bt.grad.cpu().numpy(), rbb) < 1e-4


def test_forward_saves_only_inputs(AG):
    """Primal recomputation, not storage: every saved tensor is an input."""
    g = synth.rng(11)
    a = torch.tensor(g.uniform(0.9, 1.0, 5000), device="cuda", requires_grad=True)
    b = torch.tensor(g.standard_normal(5000), device="cuda", requires_grad=True)
    inds = torch.tensor(g.integers(0, 30, 5000), dtype=torch.int32, device="cuda")
    packed = []

    def pack(t):
        packed.append(t.data_ptr())
        return t

    with torch.autograd.graph.saved_tensors_hooks(pack, lambda t: t):
        A_, B_ = AG.scan("linrec", a, b)
        y = AG.reduce("mul", a)
        h = AG.reduce_by_index("max", b, inds, 30)
    allowed = {a.data_ptr(), b.data_ptr(), inds.data_ptr()}
    assert packed and set(packed) <= allowed
    (A_.sum() + B_.sum() + y + h.sum()).backward()
    assert a.grad is not None and b.grad is not None


def test_primal_operators(oracle):
    """The forward operators of the autograd layer against the oracle's primal."""
    from paper_2202_10297_gb300 import adpar as A
    g = synth.rng(12)
    a = g.uniform(0.5, 1.5, 10007)
    at = torch.tensor(a, device="cuda")
    for op in ("add", "max", "min"):
        y, arg = A.adpar_reduce(op, at, want_argidx=op != "add")
        ry, _, rarg = oracle.reduce_vjp(op, a, 1.0)
        assert abs(y.item() - ry) <= 1e-12 * max(1.0, abs(ry))
        if op != "add":
            assert arg.item() == rarg
    y, _ = A.adpar_reduce("mul", at[:500])
    assert abs(y.item() - np.prod(a[:500])) <= 1e-12 * abs(np.prod(a[:500]))
    vals, inds, hsbar = synth.hist(20000, 64, "zipf", seed=13)
    for op in ("add", "max"):
        hs, _ = A.adpar_hist(op, torch.from_numpy(vals).cuda(), torch.from_numpy(inds).cuda(), 64)
        _, rhs, rarg = oracle.hist_vjp(op, vals, inds, 64, hsbar)
        assert rel_l2(hs.cpu().numpy()[rarg >= 0] if op == "max" else hs.cpu().numpy(),
                      rhs[rarg >= 0] if op == "max" else rhs) < 1e-5
    as_, is_, ws, _ = synth.map_acc(5000, 40, width=4, seed=14)
    xs = A.adpar_map_acc("sqdist_row", torch.from_numpy(as_).cuda(), torch.from_numpy(is_).cuda(),
                         ws=torch.from_numpy(ws).cuda(), width=4)
    ref = ((ws.reshape(-1, 4).astype(np.float64) - as_.reshape(-1, 4).astype(np.float64)[is_]) ** 2).sum(1)
    assert rel_l2(xs.cpu().numpy(), ref) < 1e-5
    n, m = 4096, 1000
    is2, _, _ = synth.scatter(n, m, seed=15)
    xs0 = synth.normal(n, np.float32, seed=16)
    vs = synth.normal(m, np.float32, seed=17)
    ys = torch.from_numpy(xs0.copy()).cuda()
    saved = torch.empty(m, device="cuda")
    A.adpar_scatter(torch.from_numpy(is2).cuda(), torch.from_numpy(vs).cuda(), ys, xs_saved=saved)
    ref = xs0.copy()
    ref[is2] = vs
    np.testing.assert_array_equal(ys.cpu().numpy(), ref)
    np.testing.assert_array_equal(saved.cpu().numpy(), xs0[is2])


def test_gradcheck_reduce_by_index_linrec_general_rule():
    """torch's gradcheck of the general reduce_by_index rule (LINREC bins,
    out-of-range indices included) in FP64."""
    from paper_2202_10297_gb300 import autograd as AG
    g = torch.Generator().manual_seed(7)
    n, m = 300, 7
    a = (0.9 + 0.2 * torch.rand(n, generator=g, dtype=torch.float64)).cuda().requires_grad_()
    b = torch.randn(n, generator=g, dtype=torch.float64).cuda().requires_grad_()
    inds = torch.randint(-1, m + 1, (n,), generator=g).to(torch.int32).cuda()
    assert torch.autograd.gradcheck(lambda x, y: AG.reduce_by_index("linrec", x, inds, m, b=y), (a, b),
                                    eps=1e-6, atol=1e-7, rtol=1e-6)


@pytest.mark.parametrize("op", ["linrec", "matrec2"])
def test_gradcheck_scan_wide(op):
    """torch's gradcheck of the wide-element scan (block and full lin_o give
    the same numbers) in FP64."""
    from paper_2202_10297_gb300 import autograd as AG
    g = torch.Generator().manual_seed(8)
    n = 700
    if op == "linrec":
        a = torch.stack([0.9 + 0.1 * torch.rand(n, generator=g, dtype=torch.float64),
                         torch.randn(n, generator=g, dtype=torch.float64)], 1)
    else:
        M = torch.eye(2, dtype=torch.float64).reshape(1, 4) * 0.95 + 0.03 * torch.randn(n, 4, generator=g,
                                                                                      dtype=torch.float64)
        a = torch.cat([M, torch.randn(n, 2, generator=g, dtype=torch.float64)], 1)
    a = a.cuda().requires_grad_()
    assert torch.autograd.gradcheck(lambda x: AG.scan_wide(op, x), (a,), eps=1e-6, atol=1e-7, rtol=1e-6)
