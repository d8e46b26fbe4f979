"""Serving loop for VJP requests of mixed operators and sizes.

Requests reference primal inputs and cotangents that stay resident on the
device (a pool generated once).  The server admits waiting requests in
arrival order whenever a slot (a CUDA stream with its own output buffers
and workspace) is free and the request's device bytes fit in what the HBM
budget leaves; admitted requests run concurrently on their slots' streams,
and completions are detected by polling CUDA events, which frees the slot
and the budget for the next request (continuous batching: no request waits
for a batch to drain).  A request larger than the budget or than a slot is
rejected; a request whose launch raises is marked failed and the loop goes
on.  ``serve_plain`` is the one-call-at-a-time form for comparison.

Each request's kernels read only its own inputs and write only its slot,
so its result does not depend on what runs beside it.
"""
import collections
import time

import numpy as np
import torch

from . import adpar as A
from . import synth

OPS = ("prod_reduce", "max_reduce", "linrec", "add_scan", "max_scan", "hist_add", "hist_max", "scatter")
HIST_BINS = 256


class Request:
    __slots__ = ("rid", "op", "n", "arrival", "start", "done", "status", "slot", "event", "outputs", "error")

    def __init__(self, rid, op, n, arrival=0.0):
        self.rid, self.op, self.n, self.arrival = rid, op, int(n), float(arrival)
        self.start = self.done = None
        self.status = "queued"
        self.slot = self.event = self.outputs = self.error = None

    @property
    def latency(self):
        return None if self.done is None else self.done - self.arrival

    def bytes(self):
        """Device bytes the request occupies while it runs (inputs + outputs + workspace)."""
        n = self.n
        per = {"prod_reduce": 8, "max_reduce": 8, "linrec": 24, "add_scan": 8, "max_scan": 12,
               "hist_add": 12, "hist_max": 16, "scatter": 12}.get(self.op, 16)
        return n * per + (1 << 20)


def make_requests(count, rate=None, lo=10, hi=24, seed=synth.SEED_BASE + 5, ops=OPS):
    """Poisson arrivals (rate requests/s; None = all at t = 0), op uniform over
    ``ops``, size 2^U[lo, hi]."""
    g = synth.rng(seed)
    t = 0.0
    reqs = []
    for i in range(count):
        if rate:
            t += g.exponential(1.0 / rate)
        op = ops[int(g.integers(0, len(ops)))]
        n = int(round(2.0 ** g.uniform(lo, hi)))
        reqs.append(Request(i, op, n, t))
    return reqs


class Pool:
    """Device-resident FP32 inputs and cotangents that requests read (first n elements)."""

    def __init__(self, max_n, device, seed=synth.SEED_BASE + 5):
        d = device
        self.max_n = max_n
        self.x_prod = torch.from_numpy(synth.uniform(max_n, 0.5, 1.5, np.float32, seed=seed)).to(d)
        self.x = torch.from_numpy(synth.normal(max_n, np.float32, seed=seed + 1)).to(d)
        self.y = torch.from_numpy(synth.normal(max_n, np.float32, seed=seed + 2)).to(d)
        a, b, ya, yb = synth.linrec(max_n, np.float32, seed=seed + 3)
        self.a, self.b, self.ya, self.yb = (torch.from_numpy(v).to(d) for v in (a, b, ya, yb))
        _, inds, hsbar = synth.hist(max_n, HIST_BINS, "zipf", seed=seed + 4)
        self.inds = torch.from_numpy(inds).to(d)
        self.hsbar = torch.from_numpy(hsbar).to(d)
        # duplicate-free scatter indices for any destination length n: 0, 4, 8, ... (< n for the first n // 4)
        self.idx4 = torch.arange(0, max_n, 4, dtype=torch.int32, device=d)


class Slot:
    def __init__(self, max_n, device):
        self.stream = torch.cuda.Stream(device=device)
        self.out1 = torch.empty(max_n, dtype=torch.float32, device=device)
        self.out2 = torch.empty(max_n, dtype=torch.float32, device=device)
        ws = 0
        for op, code in (("scan", A.OP_LINREC), ("scan", A.OP_MAX), ("scan", A.OP_ADD)):
            ws = max(ws, A.adpar_workspace_size(A.RULE_SCAN, code, A.F32, max_n))
        ws = max(ws, A.adpar_workspace_size(A.RULE_REDUCE, A.OP_MUL, A.F32, max_n),
                 A.adpar_workspace_size(A.RULE_HIST, A.OP_MAX, A.F32, max_n, HIST_BINS))
        self.work = A.workspace(ws, device)
        self.busy = None


def launch(req, slot, pool):
    """Enqueue the request's VJP on the slot's stream (all steps in the library's kernels)."""
    n, s = req.n, slot.stream
    o1, o2, w = slot.out1[:n], slot.out2[:n], slot.work
    with torch.cuda.stream(s):
        if req.op == "prod_reduce":
            A.adpar_vjp_reduce("mul", pool.x_prod[:n], pool.y[:1], abar=o1, work=w, stream=s)
        elif req.op == "max_reduce":
            A.adpar_vjp_reduce("max", pool.x[:n], pool.y[:1], abar=o1, work=w, stream=s)
        elif req.op == "linrec":
            A.adpar_vjp_scan("linrec", pool.a[:n], pool.ya[:n], b=pool.b[:n], ybar_b=pool.yb[:n], abar=o1,
                             bbar=o2, work=w, stream=s)
        elif req.op == "add_scan":
            A.adpar_vjp_scan("add", None, pool.y[:n], abar=o1, work=w, stream=s)
        elif req.op == "max_scan":
            A.adpar_vjp_scan("max", pool.x[:n], pool.y[:n], abar=o1, work=w, stream=s)
        elif req.op == "hist_add":
            A.adpar_vjp_hist("add", pool.inds[:n], HIST_BINS, pool.hsbar, valsbar=o1, work=w, stream=s)
        elif req.op == "hist_max":
            A.adpar_vjp_hist("max", pool.inds[:n], HIST_BINS, pool.hsbar, vals=pool.x[:n], valsbar=o1, work=w,
                             stream=s)
        elif req.op == "scatter":
            m = n // 4
            o1.copy_(pool.y[:n], non_blocking=True)  # the cotangent ysbar becomes xsbar in place
            A.adpar_vjp_scatter(pool.idx4[:m], o1, vsbar=o2[:m], stream=s)
        else:
            raise ValueError("unknown op %r" % req.op)
        ev = torch.cuda.Event()
        ev.record(s)
    return ev


def _collect(req, slot):
    n = req.n
    if req.op == "linrec":
        return slot.out1[:n].clone(), slot.out2[:n].clone()
    if req.op == "scatter":
        return slot.out1[:n].clone(), slot.out2[: n // 4].clone()
    return (slot.out1[:n].clone(),)


class Server:
    def __init__(self, budget_bytes=32 << 30, slots=8, max_n=1 << 24, device="cuda", pool=None):
        self.device = torch.device(device)
        self.budget = int(budget_bytes)
        self.max_n = max_n
        self.pool = pool or Pool(max_n, self.device)
        self.slots = [Slot(max_n, self.device) for _ in range(slots)]
        self.peak_resident = 0

    def serve(self, requests, keep_outputs=False, timeout_s=600.0):
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        queue = collections.deque()
        inflight = []
        resident = 0
        free = list(self.slots)
        torch.cuda.synchronize(self.device)
        t0 = time.perf_counter()
        while pending or queue or inflight:
            now = time.perf_counter() - t0
            if now > timeout_s:
                raise TimeoutError("serving loop exceeded %.0f s" % timeout_s)
            while pending and pending[0].arrival <= now:
                queue.append(pending.popleft())
            # completions free their slot and budget
            still = []
            for req in inflight:
                if req.event.query():
                    req.done = time.perf_counter() - t0
                    req.status = "done"
                    if keep_outputs:
                        req.outputs = _collect(req, req.slot)
                    resident -= req.bytes()
                    free.append(req.slot)
                    req.slot.busy = None
                else:
                    still.append(req)
            inflight = still
            # admission in arrival order
            while queue:
                req = queue[0]
                need = req.bytes()
                if need > self.budget or req.n > self.max_n:
                    queue.popleft()
                    req.status = "rejected"
                    continue
                if not free or resident + need > self.budget:
                    break
                queue.popleft()
                slot = free.pop()
                try:
                    req.start = time.perf_counter() - t0
                    req.event = launch(req, slot, self.pool)
                except Exception as e:  # a failed launch does not stop the loop
                    req.status, req.error = "failed", repr(e)
                    free.append(slot)
                    continue
                req.slot = slot
                slot.busy = req
                resident += need
                self.peak_resident = max(self.peak_resident, resident)
                req.status = "running"
                inflight.append(req)
            if not inflight and not queue and pending:
                time.sleep(max(0.0, min(1e-3, pending[0].arrival - (time.perf_counter() - t0))))
        torch.cuda.synchronize(self.device)
        return summarize(requests, time.perf_counter() - t0)


def serve_plain(requests, pool, slot, keep_outputs=False):
    """One call at a time: wait for the arrival, launch, synchronize."""
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for req in sorted(requests, key=lambda r: r.arrival):
        while time.perf_counter() - t0 < req.arrival:
            pass
        req.start = time.perf_counter() - t0
        ev = launch(req, slot, pool)
        ev.synchronize()
        req.done = time.perf_counter() - t0
        req.status = "done"
        if keep_outputs:
            req.outputs = _collect(req, slot)
    return summarize(requests, time.perf_counter() - t0)


def summarize(requests, makespan):
    done = [r for r in requests if r.status == "done"]
    lat = np.array([r.latency for r in done]) if done else np.zeros(1)
    el = sum(r.n for r in done)
    return {"requests": len(requests), "done": len(done),
            "rejected": sum(r.status == "rejected" for r in requests),
            "failed": sum(r.status == "failed" for r in requests),
            "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "throughput_rps": len(done) / makespan, "elements_per_s": el / makespan, "makespan_s": makespan}
