"""Batched VJPs (C: adpar_batch_plan / adpar_vjp_batch), CUDA-graph capture
and the autotuner that picks the launch shape.

A :class:`Batch` holds many independent segments, each a product-reduce
VJP followed by a linear-recurrence scan VJP, with its own dtype and
length.  ``run()`` is one persistent launch; ``graph()`` captures it once
in a CUDA graph for replay.  :func:`tune` times the compiled tile variants,
block counts and scheduling orders with CUDA events and writes the winner
to a JSON table.
"""
import ctypes as C
import json
import os
import time

import numpy as np
import torch

from . import adpar as A

_VP = C.c_void_p


class Segment(C.Structure):
    _fields_ = [("x", _VP), ("xbar", _VP), ("a", _VP), ("b", _VP), ("ybar_a", _VP), ("ybar_b", _VP),
                ("abar", _VP), ("bbar", _VP), ("aux", _VP), ("ybar_prod", C.c_double), ("len", C.c_int64),
                ("dtype", C.c_int32), ("reserved", C.c_int32)]


class Config(C.Structure):
    _fields_ = [("variant", C.c_int32), ("ctas_per_sm", C.c_int32), ("order", C.c_int32), ("reserved", C.c_int32)]


assert C.sizeof(Segment) == 96

TUNED_TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned_batch.json")
NUM_VARIANTS = 3


def _bind():
    L = A.lib()
    if not hasattr(L, "_batch_bound"):
        L.adpar_batch_plan_bytes.restype = C.c_size_t
        L.adpar_batch_plan_bytes.argtypes = [C.c_int]
        L.adpar_batch_plan.restype = C.c_int
        L.adpar_batch_plan.argtypes = [C.POINTER(Segment), C.c_int, C.POINTER(Config), _VP, C.c_size_t,
                                       C.POINTER(C.c_size_t)]
        L.adpar_vjp_batch.restype = C.c_int
        L.adpar_vjp_batch.argtypes = [_VP, _VP, _VP, C.c_size_t, _VP]
        L._batch_bound = True
    return L


class Batch:
    """Segments given as dicts of CUDA tensors:
    x, a, b, ybar_a, ybar_b (inputs), xbar, abar, bbar (outputs, allocated if
    missing), ybar_prod (float) and optionally aux=True for the product record.
    """

    def __init__(self, segments, config=None, device=None):
        L = _bind()
        self.device = device or segments[0]["x"].device
        self.segments = segments
        n = len(segments)
        arr = (Segment * max(n, 1))()
        self.aux = torch.zeros(max(n, 1) * A.PROD_AUX_BYTES, dtype=torch.uint8, device=self.device)
        for i, s in enumerate(segments):
            x = s["x"]
            for key in ("xbar", "abar", "bbar"):
                if s.get(key) is None:
                    s[key] = torch.empty_like(x)
            arr[i] = Segment(A._ptr(x), A._ptr(s["xbar"]), A._ptr(s["a"]), A._ptr(s["b"]), A._ptr(s["ybar_a"]),
                             A._ptr(s["ybar_b"]), A._ptr(s["abar"]), A._ptr(s["bbar"]),
                             self.aux.data_ptr() + i * A.PROD_AUX_BYTES if s.get("aux") else None,
                             float(s.get("ybar_prod", 1.0)), x.numel(), A._dtype_code(x), 0)
        self._arr = arr
        self.nseg = n
        self.plan(config)

    def plan(self, config=None):
        L = _bind()
        cfg = config if isinstance(config, Config) else Config(*(config or (0, 2, 1, 0)))
        self.config = cfg
        nbytes = L.adpar_batch_plan_bytes(self.nseg)
        self.plan_host = np.zeros(nbytes, dtype=np.uint8)
        wsb = C.c_size_t(0)
        A._check("adpar_batch_plan", L.adpar_batch_plan(self._arr, self.nseg, C.byref(cfg),
                                                        self.plan_host.ctypes.data, nbytes, C.byref(wsb)))
        self.plan_dev = torch.from_numpy(self.plan_host).to(self.device)
        self.work = A.workspace(wsb.value, self.device)
        self.work_bytes = wsb.value
        self._graph = None

    def run(self, stream=None):
        L = _bind()
        A._check("adpar_vjp_batch", L.adpar_vjp_batch(self.plan_host.ctypes.data, self.plan_dev.data_ptr(),
                                                      self.work.data_ptr(), self.work.numel(), A._stream(stream)))

    def graph(self):
        """The launch captured once in a CUDA graph (replay with .replay())."""
        if self._graph is None:
            s = torch.cuda.Stream(device=self.device)
            s.wait_stream(torch.cuda.current_stream(self.device))
            with torch.cuda.stream(s):
                self.run(stream=s)  # warm-up outside capture
            torch.cuda.current_stream(self.device).wait_stream(s)
            torch.cuda.synchronize(self.device)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=s):
                self.run(stream=s)
            self._graph = g
        return self._graph

    def status(self):
        return A.adpar_workspace_status(self.work)

    def aux_records(self):
        dt = np.dtype([("nzero", "<i8"), ("first_zero", "<i8"), ("exp2", "<i8"), ("mant", "<f8"),
                       ("log_abs_nz", "<f8"), ("sign", "<i4"), ("reserved", "<i4")])
        return np.frombuffer(self.aux.cpu().numpy().tobytes(), dtype=dt)[: self.nseg]


def signature(segments):
    lens = np.array([s["x"].numel() for s in segments], dtype=np.float64)
    f64 = np.mean([s["x"].dtype == torch.float64 for s in segments]) if segments else 0.0
    return "nseg=%d,mean_log2_len=%.1f,f64=%.2f" % (len(segments), float(np.mean(np.log2(np.maximum(lens, 1)))), f64)


def candidates():
    for v in range(NUM_VARIANTS):
        for c in (1, 2, 4):
            for o in (0, 1):
                yield (v, c, o, 0)


def _time(fn, reps):
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(reps):
        fn()
    e.record()
    torch.cuda.synchronize()
    return s.elapsed_time(e) / reps


def tune(batch, reps=5, table=TUNED_TABLE, write=True):
    """Times every candidate launch shape on this batch; keeps and records the best."""
    results = []
    for cand in candidates():
        batch.plan(cand)
        batch.run()
        torch.cuda.synchronize()
        if batch.status() != A.OK:
            continue
        results.append((_time(batch.run, reps), cand))
    results.sort()
    best_ms, best = results[0]
    batch.plan(best)
    if write:
        data = {}
        if os.path.exists(table):
            with open(table) as f:
                data = json.load(f)
        data[signature(batch.segments)] = {
            "variant": best[0], "ctas_per_sm": best[1], "order": best[2], "ms": best_ms,
            "device": torch.cuda.get_device_name(), "when": time.strftime("%Y-%m-%dT%H:%M:%S"),
            "all": [{"config": list(c), "ms": t} for t, c in results]}
        with open(table, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
    return best, best_ms, results


def tuned_config(segments, table=TUNED_TABLE):
    """The recorded best launch shape for a batch like this one, if any."""
    if os.path.exists(table):
        with open(table) as f:
            d = json.load(f).get(signature(segments))
        if d:
            return (d["variant"], d["ctas_per_sm"], d["order"], 0)
    return None
