"""Serving loop on the GPU: every served result matches the FP64 oracle on the
request's own inputs (FP32 and FP64 requests in the mix); each result is the
same alone and in the mix; admission allocates from the arena and never
exceeds it; rejected and failing requests do not stop the loop; and the
concurrent form serves faster than one call at a time."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-4, "f64": 1e-12}


@pytest.fixture(scope="module")
def S():
    from paper_2202_10297_gb300 import adpar, serve
    adpar.lib()
    pool = serve.Pool(1 << 18, torch.device("cuda"), window=1 << 16)
    return serve, pool


def _close(got, ref, tol):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    d = max(np.linalg.norm(ref), 1e-30)
    return np.linalg.norm(got - ref) <= tol * d


def _check_against_oracle(serve, pool, reqs, oracle):
    for r in reqs:
        assert r.status == "done", (r.rid, r.op, r.status, r.error)
        refs = serve.oracle_outputs(r, pool, oracle)
        assert len(refs) == len(r.outputs)
        for got, ref in zip(r.outputs, refs):
            if r.op == "scatter":
                # pure data movement: bit-exact
                np.testing.assert_array_equal(np.asarray(got, np.float64), ref, err_msg=str((r.rid, r.dtype, r.n)))
            else:
                assert _close(got, ref, TOL[r.dtype]), (r.rid, r.op, r.dtype, r.n)
            if r.op in ("max_reduce", "max_scan", "hist_max"):
                # the positions that receive adjoint are index decisions: exact
                np.testing.assert_array_equal(np.asarray(got) != 0, ref != 0, err_msg=str((r.rid, r.op, r.n)))


def test_served_results_match_oracle_small(S, oracle):
    serve, pool = S
    reqs = serve.make_requests(96, rate=None, lo=6, hi=11, seed=3, window=pool.window)
    assert {r.dtype for r in reqs} == {"f32", "f64"} and len({r.op for r in reqs}) == len(serve.OPS)
    srv = serve.Server(budget_bytes=64 << 20, slots=6, max_n=pool.max_n, pool=pool)
    st = srv.serve(reqs, keep_outputs=True)
    assert st["done"] == len(reqs) and st["failed"] == 0
    _check_against_oracle(serve, pool, reqs, oracle)
    assert srv.arena.used == 0 and srv.peak_resident <= srv.budget


def test_served_results_match_oracle_large(S, oracle):
    serve, pool = S
    reqs = serve.make_requests(32, rate=None, lo=14, hi=18, seed=4, window=pool.window)
    srv = serve.Server(budget_bytes=256 << 20, slots=8, max_n=pool.max_n, pool=pool)
    st = srv.serve(reqs, keep_outputs=True)
    assert st["done"] == len(reqs)
    _check_against_oracle(serve, pool, reqs, oracle)


def test_same_alone_and_in_the_mix(S):
    serve, pool = S
    reqs = serve.make_requests(80, rate=None, lo=8, hi=17, seed=5, window=pool.window)
    srv = serve.Server(budget_bytes=256 << 20, slots=8, max_n=pool.max_n, pool=pool)
    st = srv.serve(reqs, keep_outputs=True)
    assert st["done"] == 80 and st["failed"] == 0
    alone = [r.copy() for r in reqs]
    serve.serve_plain(alone, pool, serve.Arena(256 << 20, torch.device("cuda")), keep_outputs=True)
    for r, q in zip(reqs, alone):
        for x, y in zip(r.outputs, q.outputs):
            assert _close(x, y, 1e-5 if r.dtype == "f32" else 1e-13), (r.op, r.dtype, r.n)


def test_budget_admission_and_rejection(S):
    serve, pool = S
    reqs = serve.make_requests(60, rate=None, lo=10, hi=16, seed=6, window=pool.window)
    big = serve.Request(999, "linrec", 1 << 18, dtype="f64")  # larger than the arena below
    budget = 3 * (1 << 20)
    assert big.bytes() > budget
    srv = serve.Server(budget_bytes=budget, slots=8, max_n=pool.max_n, pool=pool)
    st = srv.serve(reqs + [big])
    assert big.status == "rejected" and st["rejected"] == 1
    assert 0 < srv.peak_resident <= srv.budget
    assert st["done"] == len(reqs)
    assert srv.arena.used == 0 and srv.arena.largest_free() == srv.arena.size


def test_failed_launch_does_not_stop_the_loop(S):
    serve, pool = S
    reqs = serve.make_requests(10, rate=None, lo=8, hi=12, seed=7, window=pool.window)
    reqs.append(serve.Request(100, "no_such_op", 1000))
    srv = serve.Server(budget_bytes=64 << 20, slots=4, max_n=pool.max_n, pool=pool)
    st = srv.serve(reqs)
    assert st["failed"] == 1 and st["done"] == 10
    assert srv.arena.used == 0


def test_concurrent_beats_plain():
    from paper_2202_10297_gb300 import serve
    pool = serve.Pool(1 << 22, torch.device("cuda"), window=1 << 20)
    reqs = serve.make_requests(60, rate=None, lo=19, hi=22, seed=8, window=pool.window)
    srv = serve.Server(budget_bytes=2 << 30, slots=8, max_n=pool.max_n, pool=pool)
    srv.serve([r.copy() for r in reqs[:16]])  # warm-up
    arena = serve.Arena(2 << 30, torch.device("cuda"))
    serve.serve_plain([r.copy() for r in reqs[:16]], pool, arena)
    a = srv.serve([r.copy() for r in reqs])
    b = serve.serve_plain([r.copy() for r in reqs], pool, arena)
    print("concurrent %.0f req/s, plain %.0f req/s" % (a["throughput_rps"], b["throughput_rps"]))
    assert a["done"] == b["done"] == len(reqs)
    assert a["throughput_rps"] > 1.1 * b["throughput_rps"]
