"""Serving loop: each request's result is the same alone and in the mix;
admission respects the HBM budget; rejected and failing requests do not
stop the loop; and the concurrent form serves faster than one-at-a-time."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    from paper_2202_10297_gb300 import adpar, serve
    adpar.lib()
    pool = serve.Pool(1 << 16, torch.device("cuda"))
    return serve, pool


def test_same_alone_and_in_the_mix(S):
    serve, pool = S
    reqs = serve.make_requests(80, rate=None, lo=8, hi=16, seed=3)
    srv = serve.Server(budget_bytes=1 << 30, slots=6, max_n=1 << 16, pool=pool)
    st = srv.serve(reqs, keep_outputs=True)
    assert st["done"] == 80 and st["failed"] == 0
    alone = [serve.Request(r.rid, r.op, r.n) for r in reqs]
    serve.serve_plain(alone, pool, serve.Slot(1 << 16, torch.device("cuda")), keep_outputs=True)
    for r, q in zip(reqs, alone):
        for x, y in zip(r.outputs, q.outputs):
            x, y = x.cpu().numpy().astype(np.float64), y.cpu().numpy().astype(np.float64)
            d = np.linalg.norm(y)
            assert np.linalg.norm(x - y) <= 1e-5 * (d if d > 0 else 1.0), (r.op, r.n)


def test_budget_admission_and_rejection(S):
    serve, pool = S
    reqs = serve.make_requests(40, rate=None, lo=10, hi=16, seed=4)
    big = serve.Request(999, "linrec", 1 << 16)  # larger than the budget below
    budget = 2 * (1 << 20) + 200000
    srv = serve.Server(budget_bytes=budget, slots=8, max_n=1 << 16, pool=pool)
    st = srv.serve(reqs + [big])
    assert big.status == "rejected" and st["rejected"] >= 1
    assert srv.peak_resident <= budget
    assert st["done"] == sum(r.bytes() <= budget for r in reqs)


def test_failed_launch_does_not_stop_the_loop(S):
    serve, pool = S
    reqs = serve.make_requests(10, rate=None, lo=8, hi=12, seed=5)
    reqs.append(serve.Request(100, "no_such_op", 1000))
    srv = serve.Server(budget_bytes=1 << 30, slots=4, max_n=1 << 16, pool=pool)
    st = srv.serve(reqs)
    assert st["failed"] == 1 and st["done"] == 10


def test_concurrent_beats_plain(S):
    serve, pool = S
    reqs = serve.make_requests(300, rate=None, lo=10, hi=16, seed=6)
    srv = serve.Server(budget_bytes=1 << 30, slots=8, max_n=1 << 16, pool=pool)
    srv.serve(reqs[:20])  # warm-up
    a = srv.serve([serve.Request(r.rid, r.op, r.n) for r in reqs])
    b = serve.serve_plain([serve.Request(r.rid, r.op, r.n) for r in reqs], pool, serve.Slot(1 << 16, torch.device("cuda")))
    assert a["throughput_rps"] > b["throughput_rps"]
