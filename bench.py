"""Benchmark of the adpar VJP hot path on GB300.

One step = one pass of every VJP of the scan workload over its batch of
synthetic inputs, at the sizes the metric is quoted on:
  * linear-recurrence scan VJP, n = 2^26 pairs, FP32
  * linear-recurrence scan VJP, n = 2^26 pairs, FP64
  * + scan VJP, n = 2^28 FP32
  * max scan VJP, n = 2^28 FP32
Inputs are resident in HBM when the timed region starts and every array is
larger than L2 (no flush needed).  ``value`` is VJP elements/s over the
whole job; the JSON line also carries the HBM roofline of the dominant call,
the VJP/primal time ratio per operator, the oracle CPU baseline, clocks
sampled during the timed region, an end-to-end figure through host
buffers, and (at N = 1, unless --no-rows) ``rows``: one summary measurement
of each other configuration of the hot path (product reduce, reduce_by_index
and scatter, the 4096-segment batch, k-means, serving).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl adpar|reference] [--no-rows]

``--workload NAME`` measures one other row of the hot path instead (one
JSON line each; these are measurements, not the headline line):
  prod     product-reduce VJP, n = 65536 FP64 with 0/1/2 zeros (latency), and
           n = 2^28 FP64 (bandwidth); argmax VJP, n = 2^28 FP32
  hist     reduce_by_index VJPs, n = 2^27 FP32, m in {256, 2^16, 2^22},
           uniform / Zipf(1.1) bins, + / * / max
  hist_general  reduce_by_index VJP by the general rule (radix sort by bin,
           segmented scans): linear recurrence at n = 2^27 FP32 with m in
           {256, 2^16, 2^22}; + and max beside the special rules
  scatter  scatter VJP, 2^26 values into 2^28 (random and sorted indices);
           map-accumulator VJPs at 2^26
  kmeans   k-means loss and C-gradient, N = 2^20, d = 32, k = 256
  batch    4096 segments (product-reduce + linear-recurrence VJPs, lengths
           2^U[8,20], FP32/FP64 mixed): one graph-replayed launch vs 4096
           plain calls
  reduce_general  reduce VJP by the general rule (two exclusive scans): the
           linear recurrence at 2^26 pairs FP32/FP64; general vs special
           rules for +, max and * at 2^28 FP32
  scan_vec vectorised scan VJP (d column scans of row-major [n][d]): linear
           recurrence and max over [2^14, 2^12]
  scan_wide scan VJP over wide elements by the general d x d lin_o: the 2x2
           matrix linear recurrence at n = 2^24 FP32/FP64; the linear
           recurrence as a 2-wide element vs the scalar rule at 2^26
  jvp      forward-mode scan rule: linear recurrence 2^26 FP32/FP64, max scan
           2^28 FP32, against the primal forward scan
  serve    Poisson arrivals of mixed-operator requests sized 2^10..2^24:
           p50/p99 latency and throughput vs one call at a time
  call     one entry point on a small case, --reps times (the profiling
           driver: --call NAME, --log2n L), e.g.
           python bench.py --workload call --call scan-linrec-f64 --log2n 24
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

LOG2_LINREC = 26
LOG2_SCAN = 28

# (name, op, dtype, log2 n, algorithmic bytes per element of the VJP, of the primal)
# VJP bytes: inputs read once + adjoints written once (Sec. 5.2's rule).
#   linrec: a, b, ybar_A, ybar_B in; abar, bbar out   -> 6 arrays
#   add:    ybar in; abar out                         -> 2 arrays
#   max:    a, ybar in; abar out                      -> 3 arrays
# Primal bytes: as in, ys out.
CALLS = [
    ("linrec_f32", "linrec", np.float32, LOG2_LINREC, 24, 16),
    ("linrec_f64", "linrec", np.float64, LOG2_LINREC, 48, 32),
    ("add_f32", "add", np.float32, LOG2_SCAN, 8, 8),
    ("max_f32", "max", np.float32, LOG2_SCAN, 12, 8),
]
# kernel launches of one call: init + (primal pass) + adjoint pass; min/max:
# init + tile extrema + group scan + record-free tiles + tiles with records +
# runs by group + runs across groups
LAUNCHES = {"linrec": 3, "max": 7, "add": 2, "mul": 3, "min": 7}

# FP64 arithmetic of the linear-recurrence VJP per pair, counted on the
# sequential definition (an FMA is 2 flops): forward A_i = a_i A_{i-1} (1)
# and B_i = a_i B_{i-1} + b_i (2); backward rs_bar = ybar + a_{i+1} rs_bar_{i+1}
# for both components (4); abar_i = A_{i-1} rA_i + B_{i-1} rB_i (3).
LINREC_FLOP_PER_PAIR = 10
# FP64 peak of a GB300: 152 SMs x 2 FP64 FMA lanes per clock (one warp
# instruction per 16 cycles per SM) x 2 flops x the maximum SM clock
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
# DRAM bytes per call of the FP64 linear-recurrence VJP (carry pass + reverse
# pass of the runs path), from an ncu capture at n = 2^24 (carry: 268.5 MB
# read + 18.3 MB written; reverse: 563.6 + 245.0 MB) scaled by 4 to 2^26
# (traffic grows in proportion to n)
LINREC_F64_TRAFFIC_PER_CALL = 4 * (268452096 + 18297344 + 563612928 + 244971008)

WORKLOAD = ("scan VJPs: linear-recurrence n=2^26 pairs FP32 and FP64 (a~U[0.9,1], b,ybar~N(0,1)); "
            "+ scan and max scan n=2^28 FP32 N(0,1)")


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """Samples nvidia-smi clocks/throttle reasons while the timed region runs."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value, dist=None, device=None):
    """The maximum of a per-rank number over all ranks (the timing rule)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, max_ms, steps):
    """Units processed by all ranks per second, timed by the slowest rank."""
    return units_per_rank * world * steps / (max_ms / 1000.0)


def make_inputs(scale_log2=0):
    """Host inputs of every call (seeded; see paper_2202_10297_gb300.synth)."""
    from paper_2202_10297_gb300 import synth
    ins = {}
    for name, op, dt, lg, _, _ in CALLS:
        n = 1 << (lg - scale_log2)
        if op == "linrec":
            a, b, ya, yb = synth.linrec(n, dt, seed=synth.SEED_BASE + 1)
            ins[name] = dict(a=a, b=b, ybar_a=ya, ybar_b=yb)
        elif op == "add":
            ins[name] = dict(ybar_a=synth.normal(n, dt, seed=synth.SEED_BASE + 11))
        else:
            ins[name] = dict(a=synth.normal(n, dt, seed=synth.SEED_BASE + 1),
                             ybar_a=synth.normal(n, dt, seed=synth.SEED_BASE + 12))
    return ins


def cpu_baseline(budget_s=12.0):
    """The FP64 oracle, as it stands, on a bounded sample of the same workload (1 core)."""
    from oracle import oracle as O
    sample_log2 = 6  # each call at 1/64 of its size
    ins = make_inputs(sample_log2)
    done_el, spent = 0, 0.0
    reps = 0
    while spent < budget_s and reps < 8:
        for name, op, dt, lg, _, _ in CALLS:
            d = ins[name]
            t0 = time.perf_counter()
            if op == "linrec":
                O.scan_vjp("linrec", d["a"], d["ybar_a"], d["b"], d["ybar_b"])
            elif op == "add":
                O.scan_vjp("add", np.zeros(1, np.float64).repeat(d["ybar_a"].size), d["ybar_a"])
            else:
                O.scan_vjp(op, d["a"], d["ybar_a"])
            spent += time.perf_counter() - t0
            done_el += d["ybar_a"].size
        reps += 1
    return {"value": done_el / spent, "unit": "elements/s", "cores": 1, "kind": "oracle",
            "sample": "each call of the step at 1/64 of its size (2^20 and 2^22 elements), "
                      "%d repetitions, %.1f s of CPU time" % (reps, spent)}


def run_reference(args, ws, rank):
    if rank != 0:
        return 0
    from oracle import oracle as O
    from paper_2202_10297_gb300 import synth  # noqa: F401
    sample_log2 = 6
    ins = make_inputs(sample_log2)
    el_per_step = sum(ins[c[0]]["ybar_a"].size for c in CALLS)

    def step():
        for name, op, dt, lg, _, _ in CALLS:
            d = ins[name]
            if op == "linrec":
                O.scan_vjp("linrec", d["a"], d["ybar_a"], d["b"], d["ybar_b"])
            elif op == "add":
                O.scan_vjp("add", np.zeros(d["ybar_a"].size), d["ybar_a"])
            else:
                O.scan_vjp(op, d["a"], d["ybar_a"])

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    v = el_per_step * args.steps / dt
    line = {"impl": "reference", "metric": "VJP elements/s", "value": v, "unit": "elements/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": "each call at 1/64 of its size",
                       "parallelism": "replicas"},
            "cpu_baseline": {"value": v, "unit": "elements/s", "cores": 1, "kind": "oracle",
                             "sample": "each call of the step at 1/64 of its size"},
            "e2e": {"value": v, "unit": "elements/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_adpar(args, ws, rank, local):
    import torch
    import torch.distributed as dist
    from paper_2202_10297_gb300 import adpar as A

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=dev)
    A.lib()
    stream = torch.cuda.current_stream()

    host = make_inputs()
    # pinned host copies (for the end-to-end figure) and device copies
    pinned = {k: {kk: torch.from_numpy(v).pin_memory() for kk, v in d.items()} for k, d in host.items()}
    devin = {k: {kk: v.to(dev) for kk, v in d.items()} for k, d in pinned.items()}
    del host
    outs, works, prims = {}, {}, {}
    for name, op, dt, lg, _, _ in CALLS:
        d = devin[name]
        ref = d["ybar_a"]
        outs[name] = (torch.empty_like(ref), torch.empty_like(ref) if op == "linrec" else None)
        dtc = A.F64 if dt == np.float64 else A.F32
        works[name] = A.workspace(A.adpar_workspace_size(A.RULE_SCAN, A.OPS[op], dtc, ref.numel()), dev)
        prims[name] = (torch.empty_like(ref), torch.empty_like(ref) if op == "linrec" else None)

    def call(name, op):
        d = devin[name]
        ab, bb = outs[name]
        A.adpar_vjp_scan(op, d.get("a"), d["ybar_a"], b=d.get("b"), ybar_b=d.get("ybar_b"),
                         abar=ab, bbar=bb, work=works[name])

    ev = {c[0]: [] for c in CALLS}

    def step(record):
        for name, op, _, _, _, _ in CALLS:
            if record:
                s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                s.record(stream)
                call(name, op)
                e.record(stream)
                ev[name].append((s, e))
            else:
                call(name, op)

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step(False)
    barrier()
    clk = ClockSampler(local)
    clk.start()
    time.sleep(0.3)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        step(True)
    t1.record(stream)
    barrier()
    clocks = clk.stop()
    ms = max_over_ranks(t0.elapsed_time(t1), dist if ws > 1 else None, dev)
    el_step = sum(1 << c[3] for c in CALLS)
    value = whole_job_rate(el_step, ws, ms, args.steps)

    # per-call averages and the roofline of the dominant call
    hbm, peak_kind = measured_peaks()
    per_call = {}
    for name, op, dt, lg, vb, pb in CALLS:
        t = np.mean([s.elapsed_time(e) for s, e in ev[name]])
        n = 1 << lg
        per_call[name] = {"ms": float(t), "elements_per_s": n / (t / 1000.0),
                          "hbm_frac_of_measured": (vb * n / (t / 1000.0)) / (hbm * 1e9)}
    f64 = per_call["linrec_f64"]
    f64["fp64_tflops"] = LINREC_FLOP_PER_PAIR * (1 << LOG2_LINREC) / (f64["ms"] / 1000.0) / 1e12
    f64["fp64_frac_of_derived_peak"] = f64["fp64_tflops"] / FP64_PEAK_TFLOPS
    dom = max(per_call, key=lambda k: per_call[k]["ms"])
    dcall = [c for c in CALLS if c[0] == dom][0]
    kernel = "adpar_vjp_scan(%s): init + primal pass + adjoint pass" % dom
    # the roofline of every scan row is HBM bandwidth on its algorithmic bytes
    ach = dcall[4] * (1 << dcall[3]) / (per_call[dom]["ms"] / 1000.0) / 1e9
    roofline = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                "traffic": LINREC_F64_TRAFFIC_PER_CALL if dom == "linrec_f64" else None,
                "kernel": kernel, "peak_source": peak_kind,
                "algorithmic_bytes_per_element": dcall[4], "elements_per_launch": 1 << dcall[3]}
    if dom == "linrec_f64":
        # GB300's FP64 rate co-bounds this call: its arithmetic against the
        # derived FP64 peak, beside the HBM fraction
        roofline["fp64_alu"] = {"achieved_tflops": f64["fp64_tflops"], "peak_tflops": FP64_PEAK_TFLOPS,
                                "frac": f64["fp64_frac_of_derived_peak"],
                                "peak_source": "derived (FP64 lanes x SMs x max SM clock)"}

    # primal (forward operator) times for the AD overhead ratio
    for name, op, dt, lg, vb, pb in CALLS:
        d = devin[name]
        ya, yb = prims[name]

        def prim():
            A.adpar_scan(op, d.get("a") if op != "add" else d["ybar_a"], b=d.get("b"), ys_a=ya, ys_b=yb,
                         work=works[name])
        for _ in range(3):
            prim()
        torch.cuda.synchronize()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 10
        s.record(stream)
        for _ in range(reps):
            prim()
        e.record(stream)
        torch.cuda.synchronize()
        tp = s.elapsed_time(e) / reps
        per_call[name]["primal_ms"] = tp
        per_call[name]["vjp_primal_ratio"] = per_call[name]["ms"] / tp

    # end to end through host buffers: copy inputs in, run, read adjoints back
    hout = {name: tuple(None if o is None else torch.empty(o.shape, dtype=o.dtype).pin_memory()
                        for o in outs[name]) for name in outs}
    h2d = sum(t.numel() * t.element_size() for d in pinned.values() for t in d.values())
    d2h = sum(o.numel() * o.element_size() for t in outs.values() for o in t if o is not None)

    # each call on its own stream: its host->device copies, its kernels and its
    # device->host copies are ordered on that stream, and the four calls'
    # transfers and kernels overlap (splitting each copy over more streams
    # measured slower)
    e2e_streams = {name: torch.cuda.Stream(device=dev) for name in outs}

    # The host->device copies (one engine, about 210 GB/s) bound the step;
    # every call's copies in are issued first, then each call's kernels and
    # copies out, which run beside the later copies in.  The calls go in
    # order of their copies out, largest first, so that the last copy in is
    # followed by the smallest kernel and copy out (measured 13-17 G el/s
    # against 11-16 issued call by call in CALLS order, on one box).
    e2e_order = [c for n in ("add_f32", "max_f32", "linrec_f64", "linrec_f32") for c in CALLS if c[0] == n]
    e2e_order += [c for c in CALLS if c not in e2e_order]

    def e2e_step():
        for name, op, _, _, _, _ in e2e_order:
            s_call = e2e_streams[name]
            s_call.wait_stream(stream)
            with torch.cuda.stream(s_call):
                for kk, v in pinned[name].items():
                    devin[name][kk].copy_(v, non_blocking=True)
        for name, op, _, _, _, _ in e2e_order:
            with torch.cuda.stream(e2e_streams[name]):
                call(name, op)
                for o, h in zip(outs[name], hout[name]):
                    if o is not None:
                        h.copy_(o, non_blocking=True)
        for s_call in e2e_streams.values():
            stream.wait_stream(s_call)

    e2e_steps = max(1, min(args.steps, 5))
    e2e_step()
    barrier()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record(stream)
    for _ in range(e2e_steps):
        e2e_step()
    e.record(stream)
    barrier()
    ems = max_over_ranks(s.elapsed_time(e), dist if ws > 1 else None, dev)
    e2e = {"value": whole_job_rate(el_step, ws, ems, e2e_steps), "unit": "elements/s",
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": e2e_steps,
           "streams": len(e2e_streams)}

    # device status words: every bounded wait finished
    status = {name: A.adpar_workspace_status(works[name]) for name in works}
    if any(v != 0 for v in status.values()):
        raise RuntimeError("device-side status not ok: %s" % status)

    if rank == 0:
        line = {"metric": "VJP elements/s", "value": value, "unit": "elements/s", "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32+f64", "data": "synthetic",
                "config": {"workload": WORKLOAD, "elements_per_step": el_step,
                           "l2": "every array larger than L2 (no flush)",
                           "parallelism": "replicas" if ws > 1 else "single GPU"},
                "roofline": roofline, "per_call": per_call,
                "gpu_launches": args.steps * sum(LAUNCHES[c[1]] for c in CALLS),
                "clocks": clocks, "e2e": e2e}
        if ws == 1:
            line["cpu_baseline"] = cpu_baseline()
            if not args.no_rows:
                line["rows"] = default_rows(args)
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


# --------------------------------------------------------------------------
# Per-row measurements (--workload NAME)
# --------------------------------------------------------------------------
def _cuda_ms(fn, reps=10, warm=3):
    """Average device time of fn() in ms (CUDA events on the current stream)."""
    import torch
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(reps):
        fn()
    e.record()
    torch.cuda.synchronize()
    return s.elapsed_time(e) / reps


def _oracle_rate(fn, elements, budget_s=3.0):
    """Elements/s of an oracle call on the host (1 core), repeated for about budget_s."""
    t0 = time.perf_counter()
    reps = 0
    while True:
        fn()
        reps += 1
        dt = time.perf_counter() - t0
        if dt >= budget_s or reps >= 50:
            return elements * reps / dt


def _line(workload, **kw):
    hbm, kind = measured_peaks()
    d = {"workload": workload, "data": "synthetic", "peak_hbm_gbs": hbm, "peak_source": kind}
    d.update(kw)
    return d


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def row_prod(args):
    """Product-reduce VJP (Sec. 5.1.1): the 65536-element FP64 latency case with
    0/1/2 zeros, the 2^28 FP64 bandwidth case; and the argmax VJP at 2^28 FP32."""
    import torch
    from oracle import oracle as O
    from paper_2202_10297_gb300 import adpar as A
    from paper_2202_10297_gb300 import synth
    hbm, _ = measured_peaks()
    cases = {}
    for z in (0, 1, 2):
        a, _ = synth.prod_reduce(65536, z)
        at = _dev(a)
        yb = torch.ones(1, dtype=torch.float64, device="cuda")
        ab = torch.empty_like(at)
        sg = torch.empty(65536, dtype=torch.int8, device="cuda")
        wk = A.workspace(A.adpar_workspace_size(A.RULE_REDUCE, A.OP_MUL, A.F64, 65536), "cuda")
        f_log = lambda: A.adpar_vjp_reduce("mul", at, yb, abar=ab, logdomain=True, want_sign=False, work=wk)
        f_val = lambda: A.adpar_vjp_reduce("mul", at, yb, abar=ab, work=wk)
        f_pri = lambda: A.adpar_reduce("mul", at, work=wk)
        t_log, t_val, t_pri = _cuda_ms(f_log, 200, 20), _cuda_ms(f_val, 200, 20), _cuda_ms(f_pri, 200, 20)
        cases["n65536_z%d" % z] = {"vjp_logdomain_us": 1e3 * t_log, "vjp_value_us": 1e3 * t_val,
                                   "primal_us": 1e3 * t_pri, "vjp_primal_ratio": t_val / t_pri,
                                   "launches_per_call": 3,
                                   "oracle_elements_per_s": _oracle_rate(lambda: O.prod_reduce_vjp(a, 1.0), 65536, 1.0)}
    n = 1 << 28
    big = torch.rand(n, dtype=torch.float64, device="cuda") + 0.5
    abig = torch.empty_like(big)
    wk = A.workspace(A.adpar_workspace_size(A.RULE_REDUCE, A.OP_MUL, A.F64, n), "cuda")
    t = _cuda_ms(lambda: A.adpar_vjp_reduce("mul", big, 1.0, abar=abig, work=wk), 5, 2)
    tp = _cuda_ms(lambda: A.adpar_reduce("mul", big, work=wk), 5, 2)
    cases["n2^28_f64_value"] = {"ms": t, "algorithmic_bytes": 16 * n, "gbs": 16 * n / t / 1e6,
                                "hbm_frac_of_measured": 16 * n / t / 1e6 / hbm, "primal_ms": tp,
                                "vjp_primal_ratio": t / tp}
    del big, abig
    x = torch.randn(n, device="cuda")
    xb = torch.empty_like(x)
    wk = A.workspace(A.adpar_workspace_size(A.RULE_REDUCE, A.OP_MAX, A.F32, n), "cuda")
    t = _cuda_ms(lambda: A.adpar_vjp_reduce("max", x, 1.0, abar=xb, work=wk), 5, 2)
    tp = _cuda_ms(lambda: A.adpar_reduce("max", x, work=wk), 5, 2)
    cases["argmax_n2^28_f32"] = {"ms": t, "algorithmic_bytes": 8 * n, "gbs": 8 * n / t / 1e6,
                                 "hbm_frac_of_measured": 8 * n / t / 1e6 / hbm, "primal_ms": tp,
                                 "vjp_primal_ratio": t / tp}
    return _line("prod", metric="VJP latency / GB/s", cases=cases, oracle_cores=1)


def row_reduce_general(args):
    """Reduce VJP by the general rule (Sec. 5.1: two exclusive scans, then a
    map): the linear recurrence (no special rule) at 2^26 pairs FP32/FP64, and
    the general vs the special rules for +, max and * at 2^28 FP32."""
    import torch
    from oracle import oracle as O
    from paper_2202_10297_gb300 import adpar as A
    from paper_2202_10297_gb300 import synth
    hbm, _ = measured_peaks()
    cases = {}
    n = 1 << LOG2_LINREC
    for dt, code, name in ((np.float32, A.F32, "linrec_f32"), (np.float64, A.F64, "linrec_f64")):
        a, b, _, _ = synth.linrec(n, dt, seed=synth.SEED_BASE + 1)
        at, bt = _dev(a), _dev(b)
        ab, bb = torch.empty_like(at), torch.empty_like(at)
        wk = A.workspace(A.adpar_workspace_size(A.RULE_REDUCE_GENERAL, A.OP_LINREC, code, n), "cuda")
        t = _cuda_ms(lambda: A.adpar_vjp_reduce_general("linrec", at, 1.0, b=bt, ybar_b=1.0, abar=ab, bbar=bb,
                                                         work=wk), 10, 3)
        w = np.dtype(dt).itemsize
        alg = 4 * w * n          # a, b read once; abar, bbar written once
        moved = 6 * w * n        # a, b read by both passes; abar, bbar written
        cases[name] = {"ms": t, "elements_per_s": n / t * 1e3, "algorithmic_bytes": alg,
                       "hbm_frac_of_measured": alg / t / 1e6 / hbm, "bytes_moved_by_design": moved,
                       "design_frac_of_measured": moved / t / 1e6 / hbm}
        del at, bt, ab, bb, wk
    # general vs special rules, FP32 2^28
    n = 1 << LOG2_SCAN
    x = torch.randn(n, device="cuda")
    xm = torch.rand(n, device="cuda") * 0.2 + 0.9
    xb = torch.empty_like(x)
    for op, inp in (("add", x), ("max", x), ("mul", xm)):
        wg = A.workspace(A.adpar_workspace_size(A.RULE_REDUCE_GENERAL, A.OPS[op], A.F32, n), "cuda")
        ws = A.workspace(A.adpar_workspace_size(A.RULE_REDUCE, A.OPS[op], A.F32, n), "cuda")
        tg = _cuda_ms(lambda: A.adpar_vjp_reduce_general(op, inp, 1.0, abar=xb, work=wg), 10, 3)
        tsp = _cuda_ms(lambda: A.adpar_vjp_reduce(op, inp, 1.0, abar=xb, work=ws), 10, 3)
        tp = _cuda_ms(lambda: A.adpar_reduce(op, inp, work=ws), 10, 3)
        cases["%s_f32_2^28" % op] = {"general_ms": tg, "special_ms": tsp, "primal_ms": tp,
                                     "general_over_special": tg / tsp, "general_over_primal": tg / tp,
                                     "special_over_primal": tsp / tp}
    small = synth.linrec(1 << 20, np.float64, seed=synth.SEED_BASE + 1)
    rate = _oracle_rate(lambda: O.reduce_general_vjp("linrec", small[0], 1.0, b=small[1], ybar_b=1.0), 1 << 20, 2.0)
    return _line("reduce_general", metric="general-rule reduce VJP elements/s and % of HBM", cases=cases,
                 cpu_baseline={"value": rate, "unit": "elements/s", "cores": 1, "kind": "oracle",
                               "sample": "linear recurrence, n = 2^20 FP64"})


def row_scan_vec(args):
    """Vectorised scan VJP (Sec. 5.2: a scan over d-vectors = d column scans):
    the linear recurrence over [2^14 rows, 2^12 channels] FP32/FP64 and the
    max scan over the same shape FP32 (2^26 elements each)."""
    import torch
    from paper_2202_10297_gb300 import adpar as A
    hbm, _ = measured_peaks()
    n, d = 1 << 14, 1 << 12
    cases = {}
    g = torch.Generator(device="cuda").manual_seed(20220221 + 6)
    for dt, name in ((torch.float32, "linrec_f32"), (torch.float64, "linrec_f64")):
        a = torch.rand((n, d), device="cuda", dtype=dt, generator=g) * 0.1 + 0.9
        b, ya, yb = (torch.randn((n, d), device="cuda", dtype=dt, generator=g) for _ in range(3))
        ab, bb = torch.empty_like(a), torch.empty_like(a)
        code = A.F64 if dt == torch.float64 else A.F32
        wk = A.workspace(A.adpar_workspace_size(A.RULE_SCAN_VEC, A.OP_LINREC, code, n, d), "cuda")
        t = _cuda_ms(lambda: A.adpar_vjp_scan_vec("linrec", a, ya, b=b, ybar_b=yb, abar=ab, bbar=bb, work=wk), 10, 3)
        w = a.element_size()
        alg = 6 * w * n * d
        cases[name] = {"rows": n, "channels": d, "ms": t, "elements_per_s": n * d / t * 1e3,
                       "algorithmic_bytes": alg, "hbm_frac_of_measured": alg / t / 1e6 / hbm}
        del a, b, ya, yb, ab, bb, wk
    x = torch.randn((n, d), device="cuda", generator=g)
    y = torch.randn((n, d), device="cuda", generator=g)
    xb = torch.empty_like(x)
    wk = A.workspace(A.adpar_workspace_size(A.RULE_SCAN_VEC, A.OP_MAX, A.F32, n, d), "cuda")
    t = _cuda_ms(lambda: A.adpar_vjp_scan_vec("max", x, y, abar=xb, work=wk), 10, 3)
    cases["max_f32"] = {"rows": n, "channels": d, "ms": t, "elements_per_s": n * d / t * 1e3,
                        "algorithmic_bytes": 12 * n * d, "hbm_frac_of_measured": 12 * n * d / t / 1e6 / hbm}
    return _line("scan_vec", metric="vectorised scan VJP elements/s and % of HBM", cases=cases)


def row_jvp(args):
    """Forward-mode (JVP) scan rule: the linear recurrence at 2^26 pairs FP32/FP64
    and the max scan at 2^28 FP32, against the primal forward scan."""
    import torch
    from oracle import oracle as O
    from paper_2202_10297_gb300 import adpar as A
    from paper_2202_10297_gb300 import synth
    hbm, _ = measured_peaks()
    cases = {}
    n = 1 << LOG2_LINREC
    for dt, name in ((np.float32, "linrec_f32"), (np.float64, "linrec_f64")):
        a, b, _, _ = synth.linrec(n, dt, seed=synth.SEED_BASE + 1)
        at, bt = _dev(a), _dev(b)
        ad, bd = torch.randn_like(at), torch.randn_like(at)
        oa, ob = torch.empty_like(at), torch.empty_like(at)
        code = A.F64 if dt == np.float64 else A.F32
        wk = A.workspace(A.adpar_workspace_size(A.RULE_SCAN | A.WS_MINIMAL, A.OP_LINREC, code, n), "cuda")
        t = _cuda_ms(lambda: A.adpar_jvp_scan("linrec", at, ad, b=bt, bdot=bd, ysdot_a=oa, ysdot_b=ob, work=wk), 10, 3)
        tp = _cuda_ms(lambda: A.adpar_scan("linrec", at, b=bt, ys_a=oa, ys_b=ob, work=wk), 10, 3)
        w = np.dtype(dt).itemsize
        alg = 6 * w * n  # a, b, adot, bdot in; ysdot_a, ysdot_b out
        cases[name] = {"ms": t, "elements_per_s": n / t * 1e3, "algorithmic_bytes": alg,
                       "hbm_frac_of_measured": alg / t / 1e6 / hbm, "primal_ms": tp, "jvp_primal_ratio": t / tp}
        del at, bt, ad, bd, oa, ob, wk
    n = 1 << LOG2_SCAN
    x = torch.randn(n, device="cuda")
    xd = torch.randn_like(x)
    o = torch.empty_like(x)
    wk = A.workspace(A.adpar_workspace_size(A.RULE_SCAN | A.WS_MINIMAL, A.OP_MAX, A.F32, n), "cuda")
    t = _cuda_ms(lambda: A.adpar_jvp_scan("max", x, xd, ysdot_a=o, work=wk), 10, 3)
    tp = _cuda_ms(lambda: A.adpar_scan("max", x, ys_a=o, work=wk), 10, 3)
    cases["max_f32_2^28"] = {"ms": t, "elements_per_s": n / t * 1e3, "algorithmic_bytes": 12 * n,
                             "hbm_frac_of_measured": 12 * n / t / 1e6 / hbm, "primal_ms": tp, "jvp_primal_ratio": t / tp}
    small = synth.linrec(1 << 20, np.float64, seed=synth.SEED_BASE + 1)
    sd = np.ones(1 << 20)
    rate = _oracle_rate(lambda: O.scan_jvp("linrec", small[0], sd, small[1], sd), 1 << 20, 2.0)
    return _line("jvp", metric="forward-mode scan elements/s and % of HBM", cases=cases,
                 cpu_baseline={"value": rate, "unit": "elements/s", "cores": 1, "kind": "oracle",
                               "sample": "linear recurrence, n = 2^20 FP64"})


# algorithmic bytes per element of the reduce_by_index VJPs: + reads the
# indices and writes the adjoint (the bins' cotangents stay in L2); max also
# reads the values in the recompute pass and the indices again in the
# adjoint pass; * reads values and indices in both passes
HIST_ALG_BYTES = {"add": 8, "max": 16, "mul": 20}
HIST_CASES = [(m, dist) for m in (256, 1 << 16, 1 << 22) for dist in ("uniform", "zipf")]


def hist_inputs(n=1 << 27, cases=HIST_CASES):
    """Seeded reduce_by_index inputs of every (m, distribution), drawn in parallel threads."""
    import concurrent.futures as cf
    from paper_2202_10297_gb300 import synth
    with cf.ThreadPoolExecutor(max_workers=len(cases)) as ex:
        futs = {c: ex.submit(synth.hist, n, c[0], c[1], seed=synth.SEED_BASE + 2) for c in cases}
        return {c: f.result() for c, f in futs.items()}


def row_hist(args, inputs=None):
    """reduce_by_index VJPs (Sec. 5.1.2), n = 2^27 FP32."""
    import torch
    from oracle import oracle as O
    from paper_2202_10297_gb300 import adpar as A
    from paper_2202_10297_gb300 import synth
    hbm, _ = measured_peaks()
    n = 1 << 27
    alg = HIST_ALG_BYTES
    inputs = inputs or hist_inputs(n)
    cases = {}
    for (m, dist) in HIST_CASES:
        vals, inds, hsbar = inputs[(m, dist)]
        v, ix, hb = _dev(vals), _dev(inds), _dev(hsbar)
        vb = torch.empty_like(v)
        for op in ("add", "max", "mul"):
            wk = A.workspace(A.adpar_workspace_size(A.RULE_HIST, A.OPS[op], A.F32, n, m), "cuda")
            f = lambda: A.adpar_vjp_hist(op, ix, m, hb, vals=v, valsbar=vb, work=wk)
            fp = lambda: A.adpar_hist(op, v, ix, m, work=wk)
            t, tp = _cuda_ms(f, 5, 2), _cuda_ms(fp, 5, 2)
            cases["%s_m%d_%s" % (op, m, dist)] = {
                "ms": t, "elements_per_s": n / t * 1e3, "gbs": alg[op] * n / t / 1e6,
                "hbm_frac_of_measured": alg[op] * n / t / 1e6 / hbm, "primal_ms": tp, "vjp_primal_ratio": t / tp}
        del v, ix, hb, vb
    vals, inds, hsbar = synth.hist(1 << 20, 256, "zipf", seed=1)
    orate = _oracle_rate(lambda: O.hist_vjp("max", vals, inds, 256, hsbar), 1 << 20, 2.0)
    return _line("hist", metric="VJP elements/s and % of HBM", n=n, algorithmic_bytes_per_element=alg,
                 cases=cases, cpu_baseline={"value": orate, "unit": "elements/s", "cores": 1, "kind": "oracle",
                                            "sample": "hist max, n = 2^20, m = 256, Zipf"})


def row_hist_general(args):
    """reduce_by_index VJP by the general rule (Sec. 5.1.2: radix sort by bin,
    forward and reverse segmented scans, map), n = 2^27 FP32; LINREC has no
    special rule, + and max are timed beside the special-rule kernels."""
    import torch
    from oracle import oracle as O
    from paper_2202_10297_gb300 import adpar as A
    from paper_2202_10297_gb300 import synth
    hbm, _ = measured_peaks()
    n = 1 << 27
    # algorithmic bytes per element: (a, b), inds in; (abar, bbar) out
    alg = {"linrec": 20, "add": 12, "max": 12}
    cases = {}
    for op, m, dist in (("linrec", 1 << 16, "zipf"), ("linrec", 256, "uniform"), ("linrec", 1 << 22, "uniform"),
                        ("add", 1 << 16, "zipf"), ("max", 1 << 16, "zipf")):
        vals, inds, hsbar = synth.hist(n, m, dist, seed=synth.SEED_BASE + 2)
        v, ix, hb = _dev(vals), _dev(inds), _dev(hsbar)
        w2 = op == "linrec"
        b = torch.randn(n, device="cuda") if w2 else None
        hbb = torch.randn(m, device="cuda") if w2 else None
        ab = torch.empty_like(v)
        bb = torch.empty_like(v) if w2 else None
        wk = A.workspace(A.adpar_workspace_size(A.RULE_HIST_GENERAL, A.OPS[op], A.F32, n, m), "cuda")
        f = lambda: A.adpar_vjp_hist_general(op, v, ix, m, hb, b=b, hsbar_b=hbb, abar=ab, bbar=bb, work=wk)
        t = _cuda_ms(f, 5, 2)
        c = {"ms": t, "elements_per_s": n / t * 1e3, "gbs": alg[op] * n / t / 1e6,
             "hbm_frac_of_measured": alg[op] * n / t / 1e6 / hbm}
        if not w2:
            wk2 = A.workspace(A.adpar_workspace_size(A.RULE_HIST, A.OPS[op], A.F32, n, m), "cuda")
            c["special_rule_ms"] = _cuda_ms(lambda: A.adpar_vjp_hist(op, ix, m, hb, vals=v, valsbar=ab, work=wk2),
                                            5, 2)
            del wk2
        cases["%s_m%d_%s" % (op, m, dist)] = c
        del v, ix, hb, b, hbb, ab, bb, wk
    vals, inds, hsbar = synth.hist(1 << 20, 1 << 16, "zipf", seed=1)
    g = synth.rng(2)
    bv, hbv = g.standard_normal(1 << 20), g.standard_normal(1 << 16)
    orate = _oracle_rate(lambda: O.hist_general_vjp("linrec", vals, inds, 1 << 16, hsbar, b=bv, hsbar_b=hbv),
                         1 << 20, 2.0)
    return _line("hist_general", metric="VJP elements/s and % of HBM", n=n, algorithmic_bytes_per_element=alg,
                 cases=cases, cpu_baseline={"value": orate, "unit": "elements/s", "cores": 1, "kind": "oracle",
                                            "sample": "hist LINREC, n = 2^20, m = 2^16, Zipf"})


def row_scan_wide(args):
    """Scan VJP over wide elements by the general d x d lin_o (Sec. 5.2): the
    2x2 matrix linear recurrence (D = 6) at n = 2^24 FP32 and FP64, and the
    linear recurrence as a D = 2 element beside the scalar-coefficient rule."""
    import torch
    from oracle import oracle as O
    from paper_2202_10297_gb300 import adpar as A
    from paper_2202_10297_gb300 import synth
    hbm, _ = measured_peaks()
    cases = {}
    n = 1 << 24
    for dt, tdt in ((np.float32, torch.float32), (np.float64, torch.float64)):
        g = synth.rng(synth.SEED_BASE + 7)
        M = 0.95 * np.eye(2).ravel() + 0.03 * g.standard_normal((n, 4))
        a = _dev(np.concatenate([M, g.standard_normal((n, 2))], 1).astype(dt))
        yb = torch.randn(n, 6, dtype=tdt, device="cuda")
        ab = torch.empty_like(a)
        wk = A.workspace(A.adpar_workspace_size(A.RULE_SCAN_WIDE, A.OP_MATREC2, A.F32 if dt == np.float32 else A.F64,
                                                n, 0, width=6), "cuda")
        t = _cuda_ms(lambda: A.adpar_vjp_scan_wide("matrec2", a, yb, abar=ab, work=wk), 5, 2)
        tf = _cuda_ms(lambda: A.adpar_vjp_scan_wide("matrec2", a, yb, abar=ab, work=wk, full_lin_o=True), 3, 1)
        alg = 3 * 6 * np.dtype(dt).itemsize  # a, ybar in; abar out
        cases["matrec2_%s_n2p24" % ("f32" if dt == np.float32 else "f64")] = {
            "ms": t, "elements_per_s": n / t * 1e3, "gbs": alg * n / t / 1e6,
            "hbm_frac_of_measured": alg * n / t / 1e6 / hbm, "full_lin_o_ms": tf}
        del a, yb, ab, wk
    n = 1 << 26
    a, b, ya, ybb = (_dev(v) for v in synth.linrec(n, np.float32, seed=synth.SEED_BASE + 1))
    aw, yw = torch.stack([a, b], 1).contiguous(), torch.stack([ya, ybb], 1).contiguous()
    abw = torch.empty_like(aw)
    wk = A.workspace(A.adpar_workspace_size(A.RULE_SCAN_WIDE, A.OP_LINREC, A.F32, n, 0, width=2), "cuda")
    t = _cuda_ms(lambda: A.adpar_vjp_scan_wide("linrec", aw, yw, abar=abw, work=wk), 5, 2)
    ts = _cuda_ms(lambda: A.adpar_vjp_scan("linrec", a, ya, b=b, ybar_b=ybb), 5, 2)
    cases["linrec_as_d2_f32_n2p26"] = {"ms": t, "scalar_rule_ms": ts, "gbs": 24 * n / t / 1e6,
                                       "hbm_frac_of_measured": 24 * n / t / 1e6 / hbm}
    g = synth.rng(3)
    sa = np.concatenate([0.95 * np.eye(2).ravel() + 0.03 * g.standard_normal((1 << 18, 4)),
                         g.standard_normal((1 << 18, 2))], 1)
    syb = g.standard_normal(sa.shape)
    orate = _oracle_rate(lambda: O.scan_wide_vjp("matrec2", sa, syb), 1 << 18, 2.0)
    return _line("scan_wide", metric="VJP elements/s and % of HBM", cases=cases,
                 cpu_baseline={"value": orate, "unit": "elements/s", "cores": 1, "kind": "oracle",
                               "sample": "2x2 matrix recurrence, n = 2^18"})


def scatter_inputs(n=1 << 28, m=1 << 26):
    """The seeded random and sorted index sets of the scatter VJP, drawn in parallel threads."""
    import concurrent.futures as cf
    from paper_2202_10297_gb300 import synth
    with cf.ThreadPoolExecutor(max_workers=2) as ex:
        futs = {srt: ex.submit(synth.scatter, n, m, sort=srt, seed=synth.SEED_BASE + 2) for srt in (False, True)}
        return {srt: f.result()[0] for srt, f in futs.items()}


def row_scatter(args, inputs=None, map_acc=True):
    """Scatter VJP (Sec. 5.3) and map-accumulator VJPs (Sec. 5.4)."""
    import torch
    from oracle import oracle as O
    from paper_2202_10297_gb300 import adpar as A
    from paper_2202_10297_gb300 import synth
    hbm, _ = measured_peaks()
    n, m = 1 << 28, 1 << 26
    inputs = inputs or scatter_inputs(n, m)
    cases = {}
    for sort in (False, True):
        is_ = inputs[sort]
        it = _dev(is_)
        ysbar = torch.randn(n, device="cuda")
        vsbar = torch.empty(m, device="cuda")
        t = _cuda_ms(lambda: A.adpar_vjp_scatter(it, ysbar, vsbar=vsbar), 5, 2)
        # 16 B per j (is, the gathered ysbar, vsbar, the zeroed ysbar); a random
        # 4-byte access moves a 32-byte sector: 4 + 32 + 4 + 32 = 72 B per j
        cases["sorted" if sort else "random"] = {
            "ms": t, "elements_per_s": m / t * 1e3, "gbs_algorithmic": 16 * m / t / 1e6,
            "hbm_frac_of_measured": 16 * m / t / 1e6 / hbm, "gbs_sector": 72 * m / t / 1e6,
            "sector_frac_of_measured": 72 * m / t / 1e6 / hbm}
        del it, ysbar, vsbar
    nj = 1 << 26
    for g, na, width in (("gather", 1 << 20, 1), ("scale", 1 << 20, 1), ("gather", 4096, 1),
                         ("sqdist_row", 256, 32)) if map_acc else ():
        as_, is_, ws, xsbar = synth.map_acc(nj // width if width > 1 else nj, na, width=width, seed=3)
        at, it, wt, xt = _dev(as_), _dev(is_), _dev(ws), _dev(xsbar)
        asb = torch.empty_like(at)
        wsb = torch.empty_like(wt) if g != "gather" else None
        t = _cuda_ms(lambda: A.adpar_vjp_map_acc(g, at, it, xt, ws=None if g == "gather" else wt, width=width,
                                                 asbar=asb, wsbar=wsb), 5, 2)
        cases["map_acc_%s_na%d_w%d" % (g, na, width)] = {"ms": t, "elements_per_s": it.numel() * width / t * 1e3}
    is_, ys, _ = synth.scatter(1 << 22, 1 << 20, seed=4)
    orate = _oracle_rate(lambda: O.scatter_vjp(1 << 22, is_, ys), 1 << 20, 2.0)
    return _line("scatter", metric="VJP elements/s and % of HBM", cases=cases,
                 cpu_baseline={"value": orate, "unit": "elements/s", "cores": 1, "kind": "oracle",
                               "sample": "scatter, m = 2^20 into n = 2^22"})


def row_kmeans(args):
    """k-means loss and C-gradient (Sec. 7.4), N = 2^20, d = 32, k = 256."""
    import torch
    from oracle import oracle as O
    from paper_2202_10297_gb300 import adpar as A
    from paper_2202_10297_gb300 import synth
    N, d, k = 1 << 20, 32, 256
    X, Cm = synth.kmeans(N, d, k)
    Xt, Ct = _dev(X), _dev(Cm)
    wk = A.workspace(A.adpar_workspace_size(A.RULE_KMEANS, 0, A.F32, N, k), "cuda")
    cb = torch.empty_like(Ct)
    yb = torch.ones(1, device="cuda")
    t_vjp = _cuda_ms(lambda: A.adpar_kmeans_vjp(Xt, Ct, ybar=yb, Cbar=cb, work=wk), 20, 5)
    t_fwd = _cuda_ms(lambda: A.adpar_kmeans_vjp(Xt, Ct, want_grad=False, work=wk), 20, 5)
    hd = torch.empty_like(Ct)

    def grad_and_hessdiag():
        A.adpar_kmeans_vjp(Xt, Ct, ybar=yb, Cbar=cb, work=wk)
        A.adpar_kmeans_hessdiag(k, yb, wk, Hdiag=hd)
    t_gh = _cuda_ms(grad_and_hessdiag, 20, 5)  # the paper's "Jacobian + Hessian diagonal" measurement
    flops = 2.0 * N * k * d
    bf16 = 1933.0
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            bf16 = float(json.load(f)["bf16_tflops"])
    tf32_peak = bf16 * 1.1 / 2.25  # measured bf16 x the nominal tf32/bf16 ratio
    hbm, _ = measured_peaks()
    orate = _oracle_rate(lambda: O.kmeans(X[:2048], Cm, 1.0), 2048, 2.0)
    return _line("kmeans", metric="k-means VJP time", N=N, d=d, k=k, vjp_ms=t_vjp, forward_ms=t_fwd,
                 grad_and_hessdiag_ms=t_gh,
                 vjp_primal_ratio=t_vjp / t_fwd, points_per_s=N / t_vjp * 1e3,
                 roofline={"bound": "tensor", "achieved": flops / t_vjp / 1e9, "peak": tf32_peak, "unit": "TFLOP/s",
                           "frac": flops / t_vjp / 1e9 / tf32_peak,
                           "peak_source": "measured bf16 x 1.1/2.25 (tf32/bf16 nominal)",
                           "hbm_gbs": N * d * 4 / t_vjp / 1e6, "hbm_frac": N * d * 4 / t_vjp / 1e6 / hbm},
                 cpu_baseline={"value": orate, "unit": "points/s", "cores": 1, "kind": "oracle",
                               "sample": "2048 points, k = 256, d = 32"})


def _batch_segments(nseg, seed):
    import torch
    from paper_2202_10297_gb300 import synth
    lens, dts, zs = synth.batch_plan(nseg, seed=seed)
    g = synth.rng(seed + 1)
    segs = []
    for i, (L, dt, z) in enumerate(zip(lens, dts, zs)):
        tdt = torch.float64 if dt else torch.float32
        x = (torch.rand(int(L), dtype=tdt, device="cuda") + 0.5)
        if z:
            x[torch.from_numpy(g.choice(int(L), size=int(z), replace=False)).cuda()] = 0
        a = torch.rand(int(L), dtype=tdt, device="cuda") * 0.1 + 0.9
        segs.append(dict(x=x, a=a, b=torch.randn_like(a), ybar_a=torch.randn_like(a), ybar_b=torch.randn_like(a),
                         ybar_prod=1.0))
    return segs


def row_batch(args):
    """4096 uneven segments: one graph-replayed persistent launch vs 4096 plain calls."""
    import torch
    from paper_2202_10297_gb300 import adpar as A
    from paper_2202_10297_gb300 import batch as B
    from paper_2202_10297_gb300 import synth
    segs = _batch_segments(4096, synth.SEED_BASE + 3)
    total = sum(s["x"].numel() for s in segs)
    bytes_alg = sum(s["x"].numel() * (44 if s["x"].dtype == torch.float32 else 88) for s in segs)
    bt = B.Batch(segs)
    best, best_ms, results = B.tune(bt, reps=3)
    g = bt.graph()
    t_graph = _cuda_ms(g.replay, 10, 2)
    t_launch = _cuda_ms(bt.run, 10, 2)
    works = {}

    def plain():
        for s in segs:
            dt = A._dtype_code(s["x"])
            n = s["x"].numel()
            key = (dt, n)
            if key not in works:
                works[key] = (A.workspace(A.adpar_workspace_size(A.RULE_REDUCE, A.OP_MUL, dt, n), "cuda"),
                              A.workspace(A.adpar_workspace_size(A.RULE_SCAN, A.OP_LINREC, dt, n), "cuda"))
            w1, w2 = works[key]
            A.adpar_vjp_reduce("mul", s["x"], s["ybar_prod"], abar=s["xbar"], work=w1)
            A.adpar_vjp_scan("linrec", s["a"], s["ybar_a"], b=s["b"], ybar_b=s["ybar_b"], abar=s["abar"],
                             bbar=s["bbar"], work=w2)
    t_plain = _cuda_ms(plain, 3, 1)
    hbm, _ = measured_peaks()
    return _line("batch", metric="batched VJP elements/s", segments=len(segs), elements=total,
                 tuned_config={"variant": best[0], "ctas_per_sm": best[1], "order": best[2]},
                 graph_ms=t_graph, launch_ms=t_launch, plain_calls_ms=t_plain,
                 speedup_vs_plain=t_plain / t_graph, elements_per_s=total / t_graph * 1e3,
                 hbm_frac_of_measured=bytes_alg / t_graph / 1e6 / hbm,
                 tuner=[{"config": r[1], "ms": r[0]} for r in results])


def row_serve(args):
    """Poisson arrivals at 50/80/95% of the measured capacity vs one call at a time:
    mixed operators, FP32 and FP64, sizes 2^U[10,24], each request on its own
    inputs, outputs and workspace allocated from a 32 GiB device arena."""
    from paper_2202_10297_gb300 import adpar as A
    from paper_2202_10297_gb300 import serve as S
    A.lib()
    srv = S.Server(budget_bytes=32 << 30, slots=8, max_n=1 << 24)
    srv.serve(S.make_requests(200, rate=None, seed=1))  # warm-up
    cap = srv.serve(S.make_requests(2000, rate=None, seed=2))
    cap_plain = S.serve_plain(S.make_requests(2000, rate=None, seed=2), srv.pool, srv.arena)
    out = {"capacity": cap, "capacity_plain": cap_plain, "sweep": {}}
    for frac in (0.5, 0.8, 0.95):
        rate = frac * cap["throughput_rps"]
        res = srv.serve(S.make_requests(3000, rate=rate, seed=3))
        res_plain = S.serve_plain(S.make_requests(3000, rate=rate, seed=3), srv.pool, srv.arena)
        out["sweep"]["%d%%" % int(frac * 100)] = {"rate_rps": rate, "served": res, "plain": res_plain}
    out["peak_arena_bytes"] = srv.peak_resident
    return _line("serve", metric="served p50/p99 latency and throughput", budget_gib=32, slots=8, **out)


def _sig(x, k=4):
    """Floats rounded to k significant digits (keeps the JSON line short)."""
    if isinstance(x, float):
        return float("%.*g" % (k, x))
    if isinstance(x, dict):
        return {a: _sig(b, k) for a, b in x.items()}
    if isinstance(x, (list, tuple)):
        return [_sig(v, k) for v in x]
    return x


def default_rows(args):
    """The other configurations of the hot path, each measured once on this
    GPU with CUDA events and summarised (the full per-case lines come from
    ``--workload NAME``): the product reduce at 65536 FP64 with 0/1/2 zeros,
    reduce_by_index at 2^27 and scatter at 2^26 -> 2^28, the 4096-segment
    batch, the k-means loss and gradient, and the served form."""
    t0 = time.perf_counter()
    hin = hist_inputs()
    sin = scatter_inputs()
    t_gen = time.perf_counter() - t0
    prod = row_prod(args)
    hist = row_hist(args, hin)
    del hin
    sc = row_scatter(args, sin, map_acc=False)
    del sin
    batch = row_batch(args)
    km = row_kmeans(args)
    srv = row_serve(args)
    rows = {}
    c1 = {k: {kk: v[kk] for kk in ("vjp_value_us", "vjp_logdomain_us", "primal_us", "vjp_primal_ratio",
                                   "launches_per_call", "oracle_elements_per_s")}
          for k, v in prod["cases"].items() if k.startswith("n65536")}
    big = prod["cases"]["n2^28_f64_value"]
    c1["n2^28_f64"] = {"ms": big["ms"], "hbm_frac_of_measured": big["hbm_frac_of_measured"],
                       "vjp_primal_ratio": big["vjp_primal_ratio"], "bytes_per_element": 16}
    rows["config1_prod_reduce"] = c1
    rows["config3_hist"] = {
        "n": hist["n"], "bytes_per_element": hist["algorithmic_bytes_per_element"],
        "fields": ["ms", "hbm_frac_of_measured", "vjp_primal_ratio"],
        "cases": {k: [v["ms"], v["hbm_frac_of_measured"], v["vjp_primal_ratio"]] for k, v in hist["cases"].items()},
        "oracle": hist["cpu_baseline"]}
    rows["config3_scatter"] = {
        "n": 1 << 28, "m": 1 << 26, "bytes_per_element": 16,
        "cases": {k: {kk: v[kk] for kk in ("ms", "hbm_frac_of_measured", "sector_frac_of_measured")}
                  for k, v in sc["cases"].items()},
        "oracle": sc["cpu_baseline"]}
    rows["config4_batch"] = {k: batch[k] for k in ("segments", "elements", "graph_ms", "plain_calls_ms",
                                                   "speedup_vs_plain", "elements_per_s", "hbm_frac_of_measured",
                                                   "tuned_config")}
    rows["config5_kmeans"] = {"N": km["N"], "d": km["d"], "k": km["k"], "vjp_ms": km["vjp_ms"],
                              "forward_ms": km["forward_ms"], "grad_and_hessdiag_ms": km["grad_and_hessdiag_ms"],
                              "vjp_primal_ratio": km["vjp_primal_ratio"],
                              "tensor_frac_of_tf32_peak": km["roofline"]["frac"],
                              "hbm_frac_of_measured": km["roofline"]["hbm_frac"], "oracle": km["cpu_baseline"]}
    sv = {"capacity_rps": srv["capacity"]["throughput_rps"],
          "capacity_plain_rps": srv["capacity_plain"]["throughput_rps"],
          "peak_arena_bytes": srv["peak_arena_bytes"], "budget_gib": srv["budget_gib"], "slots": srv["slots"]}
    for load, r in srv["sweep"].items():
        sv[load] = {"rate_rps": r["rate_rps"], "p50_ms": r["served"]["p50_ms"], "p99_ms": r["served"]["p99_ms"],
                    "plain_p50_ms": r["plain"]["p50_ms"], "plain_p99_ms": r["plain"]["p99_ms"]}
    rows["config5_serve"] = sv
    rows["input_generation_s"] = t_gen
    rows["wall_s"] = time.perf_counter() - t0
    return _sig(rows)


def _one_call(name, log2n):
    """A closure running one entry point on seeded synthetic inputs of 2^log2n elements."""
    import torch
    from paper_2202_10297_gb300 import adpar as A
    from paper_2202_10297_gb300 import synth
    n = 1 << log2n
    if name.startswith("scan-"):
        _, op, dt = name.split("-")
        npdt = np.float64 if dt == "f64" else np.float32
        if op == "linrec":
            a, b, ya, yb = (_dev(v) for v in synth.linrec(n, npdt, seed=synth.SEED_BASE + 1))
            return lambda: A.adpar_vjp_scan("linrec", a, ya, b=b, ybar_b=yb)
        x = _dev(synth.normal(n, npdt, seed=synth.SEED_BASE + 1))
        y = _dev(synth.normal(n, npdt, seed=synth.SEED_BASE + 11))
        return lambda: A.adpar_vjp_scan(op, x, y)
    if name == "kmeans":
        X, Cm = synth.kmeans(n, 32, 256)
        Xt, Ct = _dev(X), _dev(Cm)
        return lambda: A.adpar_kmeans_vjp(Xt, Ct, ybar=1.0)
    if name.startswith("hist-"):
        op = name.split("-")[1]
        vals, inds, hsbar = synth.hist(n, 256, "zipf", seed=synth.SEED_BASE + 2)
        v, ix, hb = _dev(vals), _dev(inds), _dev(hsbar)
        return lambda: A.adpar_vjp_hist(op, ix, 256, hb, vals=v)
    if name == "hist_general-linrec":
        vals, inds, hsbar = synth.hist(n, 1 << 16, "zipf", seed=synth.SEED_BASE + 2)
        v, ix, hb = _dev(vals), _dev(inds), _dev(hsbar)
        b, hbb = torch.randn_like(v), torch.randn_like(hb)
        return lambda: A.adpar_vjp_hist_general("linrec", v, ix, 1 << 16, hb, b=b, hsbar_b=hbb)
    if name == "prod-f64":
        a = _dev(synth.prod_reduce(n, 0)[0])
        return lambda: A.adpar_vjp_reduce("mul", a, 1.0)
    if name == "scatter":
        is_, ysbar, _ = synth.scatter(4 * n, n, seed=synth.SEED_BASE + 2)
        it, yt = _dev(is_), _dev(ysbar)
        return lambda: A.adpar_vjp_scatter(it, yt)
    raise ValueError(name)


CALLS_ONE = ("scan-linrec-f64", "scan-linrec-f32", "scan-add-f32", "scan-max-f32", "kmeans", "hist-mul",
             "hist-max", "hist-add", "prod-f64", "scatter", "hist_general-linrec")


def row_call(args):
    """Runs one entry point --reps times on a small case (the ncu driver)."""
    import torch
    f = _one_call(args.call, args.log2n)
    for _ in range(args.reps):
        f()
    torch.cuda.synchronize()
    return _line("call", call=args.call, log2n=args.log2n, reps=args.reps)


ROWS = {"prod": row_prod, "hist": row_hist, "hist_general": row_hist_general, "scatter": row_scatter,
        "scan_wide": row_scan_wide, "kmeans": row_kmeans, "batch": row_batch, "serve": row_serve, "call": row_call, "reduce_general": row_reduce_general, "jvp": row_jvp,
        "scan_vec": row_scan_vec}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)  # a timed region of about 1.2 s
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="adpar", choices=["adpar", "reference"])
    ap.add_argument("--workload", default="scan",
                    choices=["scan", "prod", "hist", "hist_general", "scan_wide", "scatter", "kmeans", "batch", "serve", "call",
                             "reduce_general", "jvp", "scan_vec"])
    ap.add_argument("--call", default="scan-linrec-f64", choices=sorted(CALLS_ONE))
    ap.add_argument("--log2n", type=int, default=24)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--no-rows", action="store_true",
                    help="print the headline line without the other configurations' rows")
    args = ap.parse_args()
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, ws, rank)
    if args.workload != "scan":
        print(json.dumps(ROWS[args.workload](args)), flush=True)
        return 0
    return run_adpar(args, ws, rank, local)


if __name__ == "__main__":
    sys.exit(main())
