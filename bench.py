#!/usr/bin/env python3
"""Benchmark of the escape-time renderer on one GB300 (or N replicas).

One step = one pass of the render path over the 8192 x 8192 view
re[-2, 1] x im[-1.5, 1.5] at iterMax 10000 (R^2 = 4): pixel map, then the
scheduled escape-time kernel, counts written to HBM.  Throughput is
Giter/s = (sum of counts, i.e. z-updates) / time; the roofline is the FP64
pipe, measured in this run by the library's own microbenchmark.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank renders its own replica (weak scaling); the
timed region is bracketed by a barrier and synchronize on every rank and the
maximum over ranks is reported by rank 0.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

ALG_OPS_PER_ITER = 8  # 3 mul + 1 doubling + 4 add/sub per escape step (binary64)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--sched", default="fcfs_tiles")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-peak", action="store_true", help="skip the FP64 microbenchmark (profiling runs)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-compare", action="store_true", help="skip the per-scheduler makespan comparison")
    p.add_argument("--size", type=int, default=0, help="override m = n (profiling runs)")
    p.add_argument("--iter-max", type=int, default=0, help="override iterMax (profiling runs)")
    p.add_argument("--cpu-rows-stride", type=int, default=4)
    return p.parse_args()


def bench_view(args):
    from paper_2007_00745_gb300 import workloads as wl
    v = wl.FULL_VIEW_2
    if args.size or args.iter_max:
        v = wl.scaled(v, args.size or v.m, args.size or v.n, args.iter_max or v.iter_max)
    return v


def trace_stats(tr, sms):
    """Makespan and idle tail from per-CTA (start, end, smid) records: idle tail =
    sum over SMs of (makespan - that SM's last end) / (#SMs * makespan)."""
    import numpy as np
    start = tr[:, 0].astype(np.int64)
    end = tr[:, 1].astype(np.int64)
    smid = (tr[:, 2] & 0xFFFFFFFF).astype(np.int64)
    t0, t1 = int(start.min()), int(end.max())
    span = max(t1 - t0, 1)
    last = np.full(sms, t0, np.int64)
    for s_, e_ in zip(smid, end):
        if 0 <= s_ < sms:
            last[s_] = max(last[s_], e_)
    idle = float((t1 - last).sum()) / (sms * span)
    return {"makespan_ms": span / 1e6, "idle_tail": idle,
            "cta_end_spread_ms": float(end.max() - end.min()) / 1e6}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---- clocks ------------------------------------------------------------------

QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    def __init__(self, device_index):
        self.path = tempfile.mktemp(prefix="mb_clocks_", suffix=".csv")
        self.proc = None
        self.dev = device_index

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + QUERY, "--format=csv,noheader,nounits",
                                          "-i", str(self.dev), "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx = max(mx, float(parts[2]))
                except ValueError:
                    continue
                for nm, val in zip(names, parts[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(nm)
            os.unlink(self.path)
        except OSError:
            pass
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": mx or None, "reasons": sorted(reasons), "samples": len(sm)}


# ---- reference arm: the CPU oracle ------------------------------------------

def cpu_sample_parallel(view, stride):
    """Every `stride`-th row, all rows in one oracle call (rows shared FCFS across cores)."""
    import numpy as np
    import oracle
    oracle.lib()
    rows = np.arange(0, view.m, stride, dtype=np.uint64)
    idx = (rows[:, None] * np.uint64(view.n) + np.arange(view.n, dtype=np.uint64)[None, :]).reshape(-1)
    t0 = time.perf_counter()
    counts = oracle.render_pixels(view.window, view.m, view.n, view.iter_max, view.r2, idx)
    dt = time.perf_counter() - t0
    return int(counts.astype(np.uint64).sum()), dt, len(rows), oracle.max_threads()


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from paper_2007_00745_gb300 import workloads as wl
    v = bench_view(args)
    times, iters = [], 0
    stride = max(args.cpu_rows_stride, 1)
    for k in range(args.warmup + args.steps):
        it, dt, nrows, cores = cpu_sample_parallel(v, stride)
        if k >= args.warmup:
            times.append(dt)
            iters = it
    t = sum(times) / len(times)
    val = iters / t / 1e9
    line = {
        "impl": "reference", "metric": "Giter/s", "value": val, "unit": "Giter/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "8192x8192 re[-2,1] im[-1.5,1.5] iterMax 10000 R2 4 (every %d-th row)" % stride},
        "cpu_baseline": {"value": val, "unit": "Giter/s", "cores": cores, "kind": "oracle",
                         "sample": "%d of %d rows (every %d-th), %d iterations" % (nrows, v.m, stride, iters)},
        "e2e": {"value": val, "unit": "Giter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---- our arm -------------------------------------------------------------------

def run_ours(args):
    import numpy as np
    import torch

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        torch.distributed.init_process_group("nccl")
    try:
        import paper_2007_00745_gb300 as mb
        mb.mb_version()
    except ImportError:
        import __graft_entry__
        __graft_entry__.build()
        import paper_2007_00745_gb300 as mb
    from paper_2007_00745_gb300 import workloads as wl

    v = bench_view(args)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    out = torch.empty(v.m * v.n, dtype=torch.int32, device=dev)
    host = torch.empty(v.m * v.n, dtype=torch.int32, pin_memory=True)
    total = torch.zeros(1, dtype=torch.int64, device=dev)

    def step():
        mb.mb_render(v.window, v.m, v.n, v.iter_max, v.r2, out, sched=args.sched, stream=stream)

    # FP64 pipe peak (the roofline denominator), measured now on this GPU.
    if args.no_peak:
        peak = float("nan")
    else:
        peak_add, _ = mb.mb_fp64_peak(0)
        peak_mul, _ = mb.mb_fp64_peak(1)
        peak = max(peak_add, peak_mul)

    step()
    mb.mb_sum_counts(out, total, stream=stream)
    torch.cuda.synchronize()
    iters = int(total.item())

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for k in range(args.steps):
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
        t1.record(stream)
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
    ms_total = t0.elapsed_time(t1)
    kernel_ms = [a.elapsed_time(b) for a, b in ev]
    clocks = clk.summary()

    # end to end through the public call with host buffers: render + D2H of the counts
    e2e_ms = []
    for k in range(0 if args.no_e2e else max(2, min(args.steps, 3))):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        step()
        host.copy_(out, non_blocking=True)
        b.record(stream)
        b.synchronize()
        e2e_ms.append(a.elapsed_time(b))

    if ws > 1:
        t = torch.tensor([ms_total], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms_total = float(t.item())
    ms_step = ms_total / args.steps
    value = ws * iters / (ms_step * 1e-3) / 1e9
    k_ms = sum(kernel_ms) / len(kernel_ms)
    achieved = iters * ALG_OPS_PER_ITER / (k_ms * 1e-3) / 1e12
    e2e_val = ws * iters / (sum(e2e_ms) / len(e2e_ms) * 1e-3) / 1e9 if e2e_ms else None

    # Makespan of each scheduler on the same view (outside the timed region).
    compare = {}
    if not args.no_compare:
        sms, _ = mb.mb_device_info(256)
        for sched in ("naive", "alternating", "fcfs_rows", "fcfs_tiles"):
            g = sms * mb.mb_device_info(256)[1]
            tr = torch.zeros(g * 3, dtype=torch.int64, device=dev)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            mb.mb_render(v.window, v.m, v.n, v.iter_max, v.r2, out, sched=sched, stream=stream, grid=g,
                         trace=tr)
            b.record(stream)
            torch.cuda.synchronize()
            st = trace_stats(tr.cpu().numpy().reshape(-1, 3), sms)
            st["ms"] = a.elapsed_time(b)
            st["giter_s"] = iters / (st["ms"] * 1e-3) / 1e9
            compare[sched] = st

    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return

    line = {
        "metric": "Giter/s", "value": value, "unit": "Giter/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "%dx%d re[-2,1] im[-1.5,1.5] iterMax %d R2 4, sched %s"
                               % (v.m, v.n, v.iter_max, args.sched),
                   "iterations_per_step": iters, "l2": "output 268 MB > 129 MB L2 per step",
                   "parallelism": "replicas" if ws > 1 else "1 GPU"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak / 1e12, "unit": "TFLOP/s",
                     "peak_source": "mb_fp64_peak: binary64 add/mul issue rate measured in this run",
                     "frac": achieved / (peak / 1e12), "traffic": None,
                     "note": "binary64 ops: 8 per escape step; peak = measured FP64 issue rate (mb_fp64_peak)"},
        "pct_fp64_peak": 100.0 * achieved / (peak / 1e12),
        "kernel_ms": k_ms,
        "clocks": clocks,
        "e2e": {"value": e2e_val, "unit": "Giter/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": v.m * v.n * 4},
        "gpu_launches": 2 * args.steps,
        "schedulers": compare,
    }
    if not args.no_cpu_baseline:
        stride = max(args.cpu_rows_stride, 1)
        it, dt, nrows, cores = cpu_sample_parallel(v, stride)
        line["cpu_baseline"] = {"value": it / dt / 1e9, "unit": "Giter/s", "cores": cores, "kind": "oracle",
                                "sample": "%d of %d rows (every %d-th), %d iterations, %.1f s"
                                          % (nrows, v.m, stride, it, dt)}
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
