"""The batched form (one persistent launch for many uneven instances) gives
what the plain per-call entry points give, segment by segment: products'
zero counts and lowest zero indices bit-exact, values within the FP32/FP64
tolerances; also against the oracle, under every compiled tile variant and
scheduling order, and when replayed from a CUDA graph."""
import numpy as np
import pytest
import torch

from paper_2202_10297_gb300 import synth

pytestmark = pytest.mark.gpu

LENS = [1, 2, 7, 255, 256, 1023, 1024, 1025, 2047, 2048, 2049, 4095, 4096, 4097, 8191, 8193, 16385, 70001,
        123457, 0, 33, 300000]


def rel_l2(x, ref):
    x = np.asarray(x, np.float64)
    ref = np.asarray(ref, np.float64)
    d = np.linalg.norm(ref)
    return float(np.linalg.norm(x - ref) / (d if d > 0 else 1.0))


def tol(dt, n):
    return 1e-12 if dt == np.float64 else (1e-3 if n > (1 << 24) else 1e-4)


@pytest.fixture(scope="module")
def M():
    from paper_2202_10297_gb300 import adpar, batch
    adpar.lib()
    return adpar, batch


def make_segments(lens, seed=0):
    g = synth.rng(seed)
    segs, host = [], []
    for i, L in enumerate(lens):
        dt = np.float64 if (g.random() < 0.5) else np.float32
        x = g.uniform(0.5, 1.5, L)
        z = int(g.integers(0, 3))
        if L and z:
            x[g.choice(L, size=min(z, L), replace=False)] = 0
        x = x * np.exp(-np.mean(np.log(np.abs(np.where(x == 0, 1, x))))) if L else x  # keep values in range
        a, b, ya, yb = synth.linrec(max(L, 1), dt, seed=seed * 1000 + i)
        h = dict(x=x.astype(dt), a=a[:L], b=b[:L], ybar_a=ya[:L], ybar_b=yb[:L], ybar_prod=float(g.normal()))
        host.append(h)
        segs.append({k: (torch.from_numpy(np.ascontiguousarray(v)).cuda() if isinstance(v, np.ndarray) else v)
                     for k, v in h.items()} | {"aux": True})
    return segs, host


def check_against_plain(A, segs, recs):
    for i, s in enumerate(segs):
        L = s["x"].numel()
        if L == 0:
            continue
        dt = np.float64 if s["x"].dtype == torch.float64 else np.float32
        r = A.adpar_vjp_reduce("mul", s["x"], s["ybar_prod"], want_aux=True)
        assert recs[i]["nzero"] == r["aux"].nzero and recs[i]["first_zero"] == r["aux"].first_zero
        assert rel_l2(s["xbar"].cpu().numpy(), r["abar"].cpu().numpy()) < tol(dt, L), i
        ab, bb, _ = A.adpar_vjp_scan("linrec", s["a"], s["ybar_a"], b=s["b"], ybar_b=s["ybar_b"])
        assert rel_l2(s["abar"].cpu().numpy(), ab.cpu().numpy()) < tol(dt, L), i
        assert rel_l2(s["bbar"].cpu().numpy(), bb.cpu().numpy()) < tol(dt, L), i


@pytest.mark.parametrize("variant", [0, 1, 2])
@pytest.mark.parametrize("order", [0, 1])
def test_batch_equals_plain_calls(M, variant, order):
    A, B = M
    segs, _ = make_segments(LENS, seed=variant * 2 + order)
    bt = B.Batch(segs, config=(variant, 2, order, 0))
    bt.run()
    torch.cuda.synchronize()
    assert bt.status() == A.OK
    check_against_plain(A, segs, bt.aux_records())


def test_batch_against_oracle(M, oracle):
    A, B = M
    segs, host = make_segments([1, 1000, 5000, 20011], seed=42)
    bt = B.Batch(segs)
    bt.run()
    recs = bt.aux_records()
    for i, (s, h) in enumerate(zip(segs, host)):
        L = len(h["x"])
        dt = h["x"].dtype.type
        ref = oracle.prod_reduce_vjp(h["x"], h["ybar_prod"])
        assert recs[i]["nzero"] == ref["nzero"] and recs[i]["first_zero"] == ref["first_zero"]
        assert rel_l2(s["xbar"].cpu().numpy(), ref["abar"]) < tol(dt, L)
        rab, rbb, _, _ = oracle.scan_vjp("linrec", h["a"], h["ybar_a"], h["b"], h["ybar_b"])
        assert rel_l2(s["abar"].cpu().numpy(), rab) < tol(dt, L)
        assert rel_l2(s["bbar"].cpu().numpy(), rbb) < tol(dt, L)


def test_batch_graph_replay(M):
    A, B = M
    segs, _ = make_segments(LENS, seed=7)
    bt = B.Batch(segs, config=(0, 2, 1, 0))
    bt.run()
    torch.cuda.synchronize()
    first = [(s["xbar"].clone(), s["abar"].clone(), s["bbar"].clone()) for s in segs]
    for s in segs:
        for k in ("xbar", "abar", "bbar"):
            s[k].fill_(-7.0)
    g = bt.graph()
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    assert bt.status() == A.OK
    for s, f in zip(segs, first):
        dt = s["x"].dtype
        for k, ref in zip(("xbar", "abar", "bbar"), f):
            assert rel_l2(s[k].cpu().numpy(), ref.cpu().numpy()) < (1e-12 if dt == torch.float64 else 1e-5)


def test_tuner_picks_a_valid_shape(M, tmp_path):
    A, B = M
    segs, _ = make_segments([300, 5000, 40000, 100000] * 8, seed=9)
    bt = B.Batch(segs)
    best, ms, results = B.tune(bt, reps=2, table=str(tmp_path / "t.json"))
    assert ms > 0 and len(results) >= 6
    assert B.tuned_config(segs, table=str(tmp_path / "t.json")) == best
    bt.run()
    torch.cuda.synchronize()
    check_against_plain(A, segs, bt.aux_records())
