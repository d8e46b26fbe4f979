"""Serving loop for VJP requests of mixed operators, dtypes and sizes.

Primal inputs and cotangents are resident on the device: every request reads
its own window of seeded device arrays (its own offset, length and dtype;
scatter requests also their own duplicate-free index set).  What a request
writes -- its adjoints, its workspace and, for scatter, its index set and
the cotangent it consumes in place -- is allocated at admission from one
device arena whose size is the HBM budget (``Arena``: first fit over a free
list, 256-byte aligned blocks, neighbours merged on release).  A request is
admitted, in arrival order, when a slot (a CUDA stream) is free and its
block can be allocated; admitted requests run concurrently on their slots'
streams and completions are found by polling CUDA events, which returns the
block to the arena and the slot to the free list (continuous batching: no
request waits for a batch to drain).  A request larger than the whole arena
is rejected; a request whose launch raises is marked failed and the loop
goes on.  ``serve_plain`` is the one-call-at-a-time form for comparison.

Each request's kernels read only its own inputs and write only its own
block, so its result does not depend on what runs beside it.
"""
import bisect
import collections
import math
import time

import numpy as np
import torch

from . import adpar as A
from . import synth

OPS = ("prod_reduce", "max_reduce", "linrec", "add_scan", "max_scan", "hist_add", "hist_max", "scatter")
DTYPES = ("f32", "f64")
HIST_BINS = 256
ALIGN = 256


def _round_up(x, a=ALIGN):
    return (int(x) + a - 1) // a * a


class Arena:
    """First-fit allocator over one buffer of ``nbytes`` (the HBM budget).

    The bookkeeping is host-side: a sorted list of free (offset, length)
    blocks.  ``alloc`` returns an offset or None when no free block is large
    enough (the request then waits); ``release`` returns a block and merges it
    with free neighbours.  ``peak`` is the high-water mark of allocated bytes.
    With ``device`` None no device buffer is made (host logic only)."""

    def __init__(self, nbytes, device=None):
        self.size = int(nbytes) // ALIGN * ALIGN
        self.starts = [0]            # free blocks, sorted by offset
        self.lens = [self.size]
        self.used = 0
        self.peak = 0
        self.buf = None if device is None else torch.empty(self.size, dtype=torch.uint8, device=device)

    def alloc(self, nbytes):
        need = _round_up(max(int(nbytes), 1))
        for i, ln in enumerate(self.lens):
            if ln >= need:
                off = self.starts[i]
                if ln == need:
                    del self.starts[i]
                    del self.lens[i]
                else:
                    self.starts[i] += need
                    self.lens[i] -= need
                self.used += need
                self.peak = max(self.peak, self.used)
                return off
        return None

    def release(self, off, nbytes):
        need = _round_up(max(int(nbytes), 1))
        i = bisect.bisect_left(self.starts, off)
        if (i < len(self.starts) and self.starts[i] < off + need) or \
                (i > 0 and self.starts[i - 1] + self.lens[i - 1] > off):
            raise ValueError("release of a block that overlaps free space")
        self.starts.insert(i, off)
        self.lens.insert(i, need)
        self.used -= need
        if i + 1 < len(self.starts) and self.starts[i] + self.lens[i] == self.starts[i + 1]:
            self.lens[i] += self.lens[i + 1]
            del self.starts[i + 1]
            del self.lens[i + 1]
        if i > 0 and self.starts[i - 1] + self.lens[i - 1] == self.starts[i]:
            self.lens[i - 1] += self.lens[i]
            del self.starts[i]
            del self.lens[i]

    def free_bytes(self):
        return self.size - self.used

    def largest_free(self):
        return max(self.lens) if self.lens else 0

    def view(self, off, numel, dtype):
        """A tensor of ``numel`` elements of ``dtype`` at byte offset ``off``."""
        esz = torch.empty((), dtype=dtype).element_size()
        return self.buf[off:off + numel * esz].view(dtype)


def scatter_indices(n, m, s, o):
    """Duplicate-free indices is_j = (s j + o) mod n, j < m <= n (gcd(s, n) = 1)."""
    return (np.arange(m, dtype=np.int64) * s + o) % n


class Request:
    __slots__ = ("rid", "op", "dtype", "n", "arrival", "off", "sc_s", "sc_o", "start", "done", "status", "slot",
                 "event", "outputs", "error", "block", "nbytes", "views")

    def __init__(self, rid, op, n, arrival=0.0, dtype="f32", off=0, sc_s=1, sc_o=0):
        self.rid, self.op, self.n, self.arrival = rid, op, int(n), float(arrival)
        self.dtype, self.off, self.sc_s, self.sc_o = dtype, int(off), int(sc_s), int(sc_o)
        self.start = self.done = None
        self.status = "queued"
        self.slot = self.event = self.outputs = self.error = self.block = self.views = None
        self.nbytes = None

    def copy(self):
        return Request(self.rid, self.op, self.n, self.arrival, self.dtype, self.off, self.sc_s, self.sc_o)

    @property
    def latency(self):
        return None if self.done is None else self.done - self.arrival

    @property
    def torch_dtype(self):
        return torch.float64 if self.dtype == "f64" else torch.float32

    def layout(self):
        """[(name, numel, torch dtype)] of the arrays the request writes, and
        its workspace bytes: everything it holds in the arena while it runs."""
        n, t = self.n, self.torch_dtype
        dt = A.F64 if self.dtype == "f64" else A.F32
        if self.op == "prod_reduce":
            return [("abar", n, t)], A.adpar_workspace_size(A.RULE_REDUCE, A.OP_MUL, dt, n)
        if self.op == "max_reduce":
            return [("abar", n, t)], A.adpar_workspace_size(A.RULE_REDUCE, A.OP_MAX, dt, n)
        if self.op == "linrec":
            return [("abar", n, t), ("bbar", n, t)], A.adpar_workspace_size(A.RULE_SCAN, A.OP_LINREC, dt, n)
        if self.op == "add_scan":
            return [("abar", n, t)], A.adpar_workspace_size(A.RULE_SCAN, A.OP_ADD, dt, n)
        if self.op == "max_scan":
            return [("abar", n, t)], A.adpar_workspace_size(A.RULE_SCAN, A.OP_MAX, dt, n)
        if self.op in ("hist_add", "hist_max"):
            code = A.OP_ADD if self.op == "hist_add" else A.OP_MAX
            return [("valsbar", n, t)], A.adpar_workspace_size(A.RULE_HIST, code, dt, n, HIST_BINS)
        if self.op == "scatter":
            m = n // 4
            return [("xsbar", n, t), ("vsbar", m, t), ("is", m, torch.int64)], 0
        raise ValueError("unknown op %r" % self.op)

    def bytes(self):
        """Arena bytes of the request's block (every array and the workspace, each 256-byte aligned)."""
        arrays, ws = self.layout()
        esz = {torch.float32: 4, torch.float64: 8, torch.int64: 8}
        return sum(_round_up(k * esz[t]) for _, k, t in arrays) + (_round_up(ws) if ws else 0)


def make_requests(count, rate=None, lo=10, hi=24, seed=synth.SEED_BASE + 5, ops=OPS, dtypes=DTYPES,
                  window=1 << 22):
    """Poisson arrivals (rate requests/s; None = all at t = 0); op uniform over
    ``ops``, dtype uniform over ``dtypes``, size 2^U[lo, hi]; each request's
    inputs start at its own seeded offset (a multiple of 4, below ``window``)
    in the device-resident arrays, and a scatter request gets its own index
    map (s j + o) mod n."""
    g = synth.rng(seed)
    t = 0.0
    reqs = []
    for i in range(count):
        if rate:
            t += g.exponential(1.0 / rate)
        op = ops[int(g.integers(0, len(ops)))]
        dt = dtypes[int(g.integers(0, len(dtypes)))]
        n = int(round(2.0 ** g.uniform(lo, hi)))
        off = 4 * int(g.integers(0, max(1, window // 4)))
        s = 2 * int(g.integers(0, 1 << 30)) + 1
        while math.gcd(s, n) != 1:
            s += 2
        o = int(g.integers(0, n))
        reqs.append(Request(i, op, n, t, dt, off, s, o))
    return reqs


class Pool:
    """Seeded primal inputs and cotangents, host copies (numpy, for checking
    results) and device-resident copies (what requests read), per dtype;
    each array holds ``max_n + window`` elements so that any request window
    fits."""

    def __init__(self, max_n, device, window=1 << 22, dtypes=DTYPES, seed=synth.SEED_BASE + 5):
        self.max_n, self.window = int(max_n), int(window)
        L = self.max_n + self.window
        self.host, self.dev = {}, {}
        for j, dt in enumerate(dtypes):
            npdt = np.float64 if dt == "f64" else np.float32
            s = seed + 10 * j
            a, b, ya, yb = synth.linrec(L, npdt, seed=s + 3)
            _, inds, hsbar = synth.hist(L, HIST_BINS, "zipf", seed=s + 4)
            h = {"x_prod": synth.uniform(L, 0.5, 1.5, npdt, seed=s), "x": synth.normal(L, npdt, seed=s + 1),
                 "y": synth.normal(L, npdt, seed=s + 2), "a": a, "b": b, "ya": ya, "yb": yb, "inds": inds,
                 "hsbar": hsbar.astype(npdt)}
            self.host[dt] = h
            self.dev[dt] = {k: torch.from_numpy(v).to(device) for k, v in h.items()}

    def inputs(self, req, host=False):
        """The request's input windows (device tensors, or host arrays with host=True)."""
        P = (self.host if host else self.dev)[req.dtype]
        w, n = req.off, req.n
        win = {k: P[k][w:w + n] for k in ("x_prod", "x", "y", "a", "b", "ya", "yb", "inds")}
        win["hsbar"] = P["hsbar"]
        win["ybar"] = P["y"][w:w + 1]
        return win


_ESZ = {torch.float32: 4, torch.float64: 8, torch.int64: 8}


def launch(req, stream, pool, arena, off):
    """Enqueue the request's VJP on ``stream``, writing into its arena block
    at ``off`` (every step of the VJP runs in the library's kernels)."""
    arrays, ws = req.layout()
    views, o = {}, off
    for name, k, t in arrays:
        views[name] = arena.view(o, k, t)
        o += _round_up(k * _ESZ[t])
    work = arena.buf[o:o + ws] if ws else None
    req.views = views
    x = pool.inputs(req)
    with torch.cuda.stream(stream):
        if req.op == "prod_reduce":
            A.adpar_vjp_reduce("mul", x["x_prod"], x["ybar"], abar=views["abar"], work=work, stream=stream)
        elif req.op == "max_reduce":
            A.adpar_vjp_reduce("max", x["x"], x["ybar"], abar=views["abar"], work=work, stream=stream)
        elif req.op == "linrec":
            A.adpar_vjp_scan("linrec", x["a"], x["ya"], b=x["b"], ybar_b=x["yb"], abar=views["abar"],
                             bbar=views["bbar"], work=work, stream=stream)
        elif req.op == "add_scan":
            A.adpar_vjp_scan("add", None, x["y"], abar=views["abar"], work=work, stream=stream)
        elif req.op == "max_scan":
            A.adpar_vjp_scan("max", x["x"], x["y"], abar=views["abar"], work=work, stream=stream)
        elif req.op == "hist_add":
            A.adpar_vjp_hist("add", x["inds"], HIST_BINS, x["hsbar"], valsbar=views["valsbar"], work=work,
                             stream=stream)
        elif req.op == "hist_max":
            A.adpar_vjp_hist("max", x["inds"], HIST_BINS, x["hsbar"], vals=x["x"], valsbar=views["valsbar"],
                             work=work, stream=stream)
        elif req.op == "scatter":
            n, m = req.n, req.n // 4
            is_ = views["is"]
            torch.arange(m, out=is_)
            is_.mul_(req.sc_s).add_(req.sc_o).remainder_(n)
            xs = views["xsbar"]
            xs.copy_(x["y"])  # the cotangent ysbar becomes xsbar in place
            A.adpar_vjp_scatter(is_, xs, vsbar=views["vsbar"], stream=stream)
        else:
            raise ValueError("unknown op %r" % req.op)
        ev = torch.cuda.Event()
        ev.record(stream)
    return ev


def _collect(req):
    """Host copies of the request's outputs (after its event has completed)."""
    v = req.views
    if req.op == "linrec":
        return v["abar"].cpu().numpy(), v["bbar"].cpu().numpy()
    if req.op == "scatter":
        return v["xsbar"].cpu().numpy(), v["vsbar"].cpu().numpy()
    return (next(iter(v.values())).cpu().numpy(),)


class Server:
    """Continuous-batching server: ``slots`` CUDA streams over one arena of
    ``budget_bytes``."""

    def __init__(self, budget_bytes=32 << 30, slots=8, max_n=1 << 24, device="cuda", pool=None):
        self.device = torch.device(device)
        self.max_n = max_n
        self.pool = pool or Pool(max_n, self.device)
        self.arena = Arena(budget_bytes, self.device)
        self.budget = self.arena.size
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(slots)]

    @property
    def peak_resident(self):
        return self.arena.peak

    def _finish(self, req, t0, keep_outputs):
        req.done = time.perf_counter() - t0
        req.status = "done"
        if keep_outputs:
            req.outputs = _collect(req)
        self.arena.release(req.block, req.nbytes)
        req.views = None

    def serve(self, requests, keep_outputs=False, timeout_s=600.0):
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        queue = collections.deque()
        inflight = []
        free = list(self.streams)
        torch.cuda.synchronize(self.device)
        t0 = time.perf_counter()
        while pending or queue or inflight:
            now = time.perf_counter() - t0
            if now > timeout_s:
                raise TimeoutError("serving loop exceeded %.0f s" % timeout_s)
            while pending and pending[0].arrival <= now:
                queue.append(pending.popleft())
            # completions return their block and their stream
            still = []
            for req in inflight:
                if req.event.query():
                    self._finish(req, t0, keep_outputs)
                    free.append(req.slot)
                else:
                    still.append(req)
            inflight = still
            # admission in arrival order: a stream and an arena block
            while queue and free:
                req = queue[0]
                try:
                    need = req.bytes()
                except Exception as e:  # an unknown op or size fails alone
                    queue.popleft()
                    req.status, req.error = "failed", repr(e)
                    continue
                if need > self.arena.size or req.n > self.max_n or req.off + req.n > self.max_n + self.pool.window:
                    queue.popleft()
                    req.status = "rejected"
                    continue
                off = self.arena.alloc(need)
                if off is None:
                    break  # waits for a completion to free space
                queue.popleft()
                stream = free.pop()
                req.block, req.nbytes = off, need
                try:
                    req.start = time.perf_counter() - t0
                    req.event = launch(req, stream, self.pool, self.arena, off)
                except Exception as e:  # a failed launch does not stop the loop
                    req.status, req.error = "failed", repr(e)
                    self.arena.release(off, need)
                    free.append(stream)
                    continue
                req.slot = stream
                req.status = "running"
                inflight.append(req)
            if not inflight and not queue and pending:
                time.sleep(max(0.0, min(1e-3, pending[0].arrival - (time.perf_counter() - t0))))
        torch.cuda.synchronize(self.device)
        return summarize(requests, time.perf_counter() - t0)


def serve_plain(requests, pool, arena, keep_outputs=False):
    """One call at a time on one stream: wait for the arrival, allocate, launch, synchronize."""
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for req in sorted(requests, key=lambda r: r.arrival):
        while time.perf_counter() - t0 < req.arrival:
            pass
        req.start = time.perf_counter() - t0
        need = req.bytes()
        off = arena.alloc(need)
        if off is None:
            req.status = "rejected"
            continue
        ev = launch(req, stream, pool, arena, off)
        ev.synchronize()
        req.done = time.perf_counter() - t0
        req.status = "done"
        if keep_outputs:
            req.outputs = _collect(req)
        arena.release(off, need)
        req.views = None
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


def oracle_outputs(req, pool, O):
    """The FP64 oracle's adjoints for the request's own inputs (test helper:
    ``O`` is the oracle module, passed in by the caller)."""
    x = pool.inputs(req, host=True)
    f = lambda v: np.asarray(v, np.float64)  # noqa: E731
    if req.op == "prod_reduce":
        return (O.prod_reduce_vjp(f(x["x_prod"]), float(x["ybar"][0]))["abar"],)
    if req.op == "max_reduce":
        return (O.reduce_vjp("max", f(x["x"]), float(x["ybar"][0]))[1],)
    if req.op == "linrec":
        ab, bb, _, _ = O.scan_vjp("linrec", f(x["a"]), f(x["ya"]), f(x["b"]), f(x["yb"]))
        return ab, bb
    if req.op == "add_scan":
        return (O.scan_vjp("add", np.zeros(req.n), f(x["y"]))[0],)
    if req.op == "max_scan":
        return (O.scan_vjp("max", f(x["x"]), f(x["y"]))[0],)
    if req.op in ("hist_add", "hist_max"):
        op = "add" if req.op == "hist_add" else "max"
        return (O.hist_vjp(op, f(x["x"]), np.asarray(x["inds"], np.int64), HIST_BINS, f(x["hsbar"]))[0],)
    if req.op == "scatter":
        is_ = scatter_indices(req.n, req.n // 4, req.sc_s, req.sc_o)
        xb, vb, _ = O.scatter_vjp(req.n, is_, f(x["y"]))
        return xb, vb
    raise ValueError(req.op)
