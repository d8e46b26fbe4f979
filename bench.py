"""Benchmark of the adpar VJP hot path on GB300.

One step = one pass of every VJP of the scan workload over its batch of
synthetic inputs, at the sizes the metric is quoted on:
  * linear-recurrence scan VJP, n = 2^26 pairs, FP32
  * linear-recurrence scan VJP, n = 2^26 pairs, FP64
  * + scan VJP, n = 2^28 FP32
  * max scan VJP, n = 2^28 FP32
Inputs are resident in HBM when the timed region starts and every array is
larger than L2 (no flush needed).  ``value`` is VJP elements/s over the
whole job; the JSON line also carries the roofline of the dominant call,
the VJP/primal time ratio per operator, the oracle CPU baseline, clocks
sampled during the timed region, and an end-to-end figure through host
buffers.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl adpar|reference]
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
# kernel launches of one call: init + (primal pass) + adjoint pass
LAUNCHES = {"linrec": 3, "max": 3, "add": 2, "mul": 3, "min": 3}

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
    ms = t0.elapsed_time(t1)
    if ws > 1:
        tt = torch.tensor([ms], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
    el_step = sum(1 << c[3] for c in CALLS)
    value = el_step * ws * args.steps / (ms / 1000.0)

    # per-call averages and the roofline of the dominant call
    hbm, peak_kind = measured_peaks()
    per_call = {}
    for name, op, dt, lg, vb, pb in CALLS:
        t = np.mean([s.elapsed_time(e) for s, e in ev[name]])
        n = 1 << lg
        per_call[name] = {"ms": float(t), "elements_per_s": n / (t / 1000.0),
                          "hbm_frac_of_measured": (vb * n / (t / 1000.0)) / (hbm * 1e9)}
    dom = max(per_call, key=lambda k: per_call[k]["ms"])
    dcall = [c for c in CALLS if c[0] == dom][0]
    ach = dcall[4] * (1 << dcall[3]) / (per_call[dom]["ms"] / 1000.0) / 1e9
    roofline = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                "traffic": None, "kernel": "adpar_vjp_scan(%s): init + primal pass + adjoint pass" % dom,
                "peak_source": peak_kind}

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

    def e2e_step():
        for k, d in pinned.items():
            for kk, v in d.items():
                devin[k][kk].copy_(v, non_blocking=True)
        step(False)
        for name in outs:
            for o, h in zip(outs[name], hout[name]):
                if o is not None:
                    h.copy_(o, non_blocking=True)

    e2e_steps = max(1, min(args.steps, 5))
    e2e_step()
    barrier()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record(stream)
    for _ in range(e2e_steps):
        e2e_step()
    e.record(stream)
    barrier()
    ems = s.elapsed_time(e)
    if ws > 1:
        tt = torch.tensor([ems], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ems = float(tt.item())
    e2e = {"value": el_step * ws * e2e_steps / (ems / 1000.0), "unit": "elements/s",
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": e2e_steps}

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
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="adpar", choices=["adpar", "reference"])
    args = ap.parse_args()
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, ws, rank)
    return run_adpar(args, ws, rank, local)


if __name__ == "__main__":
    sys.exit(main())
