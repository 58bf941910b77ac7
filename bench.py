#!/usr/bin/env python3
"""Benchmark of the GB300 escape-time renderer (one GPU, or one image over N GPUs).

Headline step: the learned first-come-first-served pipeline on the 8192 x 8192
view re[-2, 1] x im[-1.5, 1.5], iterMax 10000, |z|^2 > 4 -- pixel map, probe,
tile features, MLP cost prediction, longest-first order with splits, and the
FCFS render of the rest -- with every count bit-identical to the FP64 oracle.
Giter/s = (sum of counts, i.e. z-updates) / step time.  The roofline is the
FP64 pipe, measured in this run by the library's own microbenchmark
(mb_fp64_peak): a step's 8 nominal binary64 operations take 2.5 FP64-pipe
issues on average (the products, the doubling and every other subtraction
are formed exactly on the integer pipes), so the attainable rate is the
measured issue rate x 8/2.5.

Beside the headline (outside the timed region, rank 0 only): the paper's three
row schedulers and plain tile FCFS on the same view (makespan, idle tail) beside
the learned order and the exact longest-first order of the same tiles, the
end-to-end figure through host buffers, the paper's computation / total timing
with the PPM file, the 640 x 480 naive view, the binary32 and double-float
variants (their own rates and how many pixels differ from binary64), exact
cycle detection (time to the identical image), the CPU oracle on a row sample,
the 256-viewport batch as a replayed CUDA graph (default and learned queue
order), a short Poisson serving run (p50 / p99 latency), plain and with cycle
detection, the 16384^2 deep-zoom comparison (learned vs plain FCFS), and a
serving sweep over request rates that replays one fixed draw of requests.
--table2 adds the GPU analogue of the paper's Table II.  Under torchrun
(--gpus N > 1) the step is one image rendered over the N GPUs, first come
first served (see run_sharded).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

ALG_OPS_PER_ITER = 8  # binary64 operations per escape step: 3 mul, 1 doubling, 4 add/sub
# of which issued on the FP64 pipe, on average: the 3 additions of a step, less the subtraction that
# every other step does exactly on the integer pipes (products and doubling are always there)
FP64_PIPE_OPS_PER_ITER = 2.5

# From the ncu capture of the main render kernel summarised in
# profiles/render_kernel_list_8192x8192_it1000.md: DRAM traffic per pixel (dram
# read + write per launch / pixels; traffic does not depend on iterMax, so it
# scales by pixel count) and the busy fraction of each pipe the step is split
# across, so that the binding pipes are visible beside the FP64 roofline; used
# only while the kernel sources still hash to src_sha1 and the run uses the
# captured unroll, else null.
NCU_RENDER = {"src_sha1": "bc9673f8bce11ced2c8ad63c4f07ac1a3053585d", "unroll": 4, "dram_bytes_per_pixel": 3.876,
              "pipes": {"fp64": 0.802, "alu": 0.795, "fma": 0.280, "issue": 0.732},
              # sm__inst_executed_pipe_fp64.sum x 32 / escape steps of the same launch: the FP64
              # instructions actually issued per step, idle lanes and replays included (taken at
              # iterMax 1000, where lanes refill more often than at the benchmark's 10000)
              "fp64_issued_per_step": 2.56}
KERNEL_SOURCES = ("escape_core.cuh", "escape_lowp.cuh", "render_kernels.cuh")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--sched", default="learned",
                   help="learned (default) or a plain scheduler: naive, alternating, fcfs_rows, fcfs_tiles")
    p.add_argument("--tile", type=int, default=32)
    p.add_argument("--block", type=int, default=512)
    p.add_argument("--unroll", type=int, default=4)
    p.add_argument("--min-strips", type=int, default=1,
                   help="learned order: cut every tile into at least this many row strips (power of two)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-peak", action="store_true", help="skip the FP64 microbenchmark (profiling runs)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-compare", action="store_true", help="skip the per-scheduler comparison")
    p.add_argument("--no-batch", action="store_true")
    p.add_argument("--batch-count", type=int, default=256,
                   help="viewports in the batch (default 256; fewer for profiling runs)")
    p.add_argument("--no-serve", action="store_true")
    p.add_argument("--no-precision", action="store_true", help="skip the binary32 / double-float variants")
    p.add_argument("--no-cycle", action="store_true", help="skip the exact-cycle-detection timing")
    p.add_argument("--no-zoom", action="store_true", help="skip the 16384^2 deep-zoom comparison (about a minute)")
    p.add_argument("--table2", action="store_true",
                   help="add the GPU analogue of the paper's Table II: speed-up over one worker (CTA) of the "
                        "naive, alternating and FCFS row schemes on the paper's test shape (2000^2 sample)")
    p.add_argument("--serve-sweep", default="10,20,40,50,80,100,200,500,1000,2000",
                   help="comma-separated request rates (1/s) of the serving sweep ('' = none); one fixed draw of "
                        "--serve-sweep-count requests is replayed at every rate")
    p.add_argument("--serve-sweep-count", type=int, default=200)
    p.add_argument("--serve-count", type=int, default=100)
    p.add_argument("--ppm", default="", help="also write the headline image there (default: a temporary file)")
    p.add_argument("--size", type=int, default=0, help="override m = n (profiling runs)")
    p.add_argument("--iter-max", type=int, default=0, help="override iterMax (profiling runs)")
    p.add_argument("--window", default="", help="override the window: xmin,xmax,ymin,ymax (profiling runs)")
    p.add_argument("--cpu-rows-stride", type=int, default=4,
                   help="the CPU oracle legs (cpu_baseline and --impl reference) time every k-th row of the view")
    p.add_argument("--cpu-reps", type=int, default=3, help="repetitions of the cpu_baseline row sample")
    return p.parse_args()


def dist_env():
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def bench_view(args):
    from paper_2007_00745_gb300 import workloads as wl
    v = wl.FULL_VIEW_2
    if args.size or args.iter_max:
        v = wl.scaled(v, args.size or v.m, args.size or v.n, args.iter_max or v.iter_max)
    if args.window:
        w = tuple(float(x) for x in args.window.split(","))
        if len(w) != 4 or not (w[0] < w[1] and w[2] < w[3]):
            raise SystemExit("--window wants xmin,xmax,ymin,ymax with xmin < xmax and ymin < ymax")
        v = wl.View(w, v.m, v.n, v.iter_max, v.r2)
    return v


def bench_config(args, v, ws):
    """The workload of both arms (ours and --impl reference): the same dict in both JSON lines."""
    return {"workload": "%dx%d re[%g,%g] im[%g,%g] iterMax %d R2 %g, %s (tile %d%s, block %d, unroll %d)"
                        % (v.m, v.n, v.window[0], v.window[1], v.window[2], v.window[3], v.iter_max, v.r2,
                           "learned FCFS" if args.sched == "learned" else args.sched,
                           args.tile, ", %d strips per tile at least" % args.min_strips
                           if args.sched == "learned" else "", args.block, args.unroll),
            "l2": "counts %.0f MB per step %s 129 MB L2 (compute-bound)"
                  % (v.m * v.n * 4 / 1e6, ">" if v.m * v.n * 4 > 129e6 else "<="),
            "parallelism": ("one image sharded over %d GPUs: raster tile chunks dealt first come first served "
                            "from rank 0's store counter, packed gather to rank 0" % ws) if ws > 1 else "1 GPU",
            "bit_exact": "vs FP64 oracle (tests)"}


def kernel_sha1():
    h = hashlib.sha1()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2007_00745_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


# ---- clocks --------------------------------------------------------------------

QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    def __init__(self, device_index):
        fd, self.path = tempfile.mkstemp(prefix="mb_clocks_", suffix=".csv")
        os.close(fd)
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
        sm, mx, power, reasons = [], 0.0, 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx = max(mx, float(parts[2]))
                    power = max(power, float(parts[3]))
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
        return {"sm_mhz": med, "sm_max_mhz": mx or None, "power_w_max": power or None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---- CPU oracle (cpu_baseline and the reference arm) -----------------------------

def cpu_sample(view, stride):
    """The oracle on every `stride`-th row of the view (rows shared FCFS over all host cores)."""
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
    v = bench_view(args)
    stride = max(args.cpu_rows_stride, 1)   # the same row sample as our arm's cpu_baseline
    times, iters, nrows, cores = [], 0, 0, 0
    for k in range(args.warmup + args.steps):
        it, dt, nrows, cores = cpu_sample(v, stride)
        if k >= args.warmup:
            times.append(dt)
            iters = it
    t = sum(times) / len(times)
    val = iters / t / 1e9
    sample = "%d of %d rows (every %d-th), %d iterations per step" % (nrows, v.m, stride, iters)
    print(json.dumps({
        "impl": "reference", "metric": "Giter/s", "value": val, "unit": "Giter/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": bench_config(args, v, ws),
        "cpu_baseline": {"value": val, "unit": "Giter/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": "Giter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ---- helpers for our arm -------------------------------------------------------------

def trace_stats(tr, sms):
    """Makespan and idle tail from per-CTA (start, end, smid) records: idle tail =
    sum over SMs of (makespan - that SM's last end) / (#SMs * makespan)."""
    import numpy as np
    start = tr[:, 0].astype(np.int64)
    end = tr[:, 1].astype(np.int64)
    smid = (tr[:, 2] & 0xFFFFFFFF).astype(np.int64)
    ok = end > 0
    start, end, smid = start[ok], end[ok], smid[ok]
    t0, t1 = int(start.min()), int(end.max())
    span = max(t1 - t0, 1)
    last = np.full(sms, t0, np.int64)
    for s_, e_ in zip(smid, end):
        if 0 <= s_ < sms:
            last[s_] = max(last[s_], e_)
    return {"makespan_ms": span / 1e6, "idle_tail": float((t1 - last).sum()) / (sms * span)}


def pct(xs, q):
    xs = sorted(xs)
    if not xs:
        return None
    k = min(len(xs) - 1, max(0, int(round(q / 100.0 * (len(xs) - 1)))))
    return xs[k]


def run_serve(mb, wl, torch, rate, count, views=None, **sopts):
    """Open-loop Poisson stream of batch-distribution viewports into a server with a
    40 GB budget; latency percentiles (submit to done) and delivered Giter/s.
    `views` (default: a seeded draw of `count`) arrive at the times of one seeded
    unit-rate Poisson stream divided by `rate`, so that runs at different rates
    replay the same requests in the same pattern, only faster or slower."""
    if views is None:
        views = wl.batch_views(count=count, seed=wl.SEED + 500)
    count = len(views)
    arrivals = [t / rate for t in wl.poisson_arrivals(1.0, count)]
    srv = mb.Server(budget_bytes=40 << 30, queue_limit=4096, **sopts)
    ids, lat, iters, failed = [None] * count, [], 0, 0
    tot = torch.zeros(1, dtype=torch.int64, device="cuda")
    side = torch.cuda.Stream()
    max_queued = 0
    t0 = time.perf_counter()
    for k, (v, ta) in enumerate(zip(views, arrivals)):
        d = t0 + ta - time.perf_counter()
        if d > 0:
            time.sleep(d)
        try:
            ids[k] = srv.submit(v)
        except mb.MBError:
            failed += 1
        if k % 8 == 0:
            max_queued = max(max_queued, srv.counters()["queued"])
    t_first, t_last = None, 0
    for k, rid in enumerate(ids):
        if rid is None:
            continue
        rc, st = srv.wait(rid, 600000)
        if rc != 0:
            failed += 1
            continue
        lat.append((st["done_ns"] - st["submit_ns"]) / 1e6)
        t_first = st["submit_ns"] if t_first is None else min(t_first, st["submit_ns"])
        t_last = max(t_last, st["done_ns"])
        mb.mb_sum_counts_ptr(srv.result(rid), views[k].m * views[k].n, tot, stream=side)
        side.synchronize()
        iters += int(tot.item())
        srv.release(rid)
    c = srv.counters()
    srv.destroy()
    span = (t_last - t_first) / 1e9 if t_first is not None else 0.0
    offered = iters / arrivals[-1] / 1e9 if arrivals and arrivals[-1] > 0 else None
    return {"rate_per_s": rate, "requests": count, "submitted": c["submitted"], "admitted": c["admitted"],
            "completed": len(lat), "rejected_or_failed": failed, "max_queued": max_queued,
            "p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99), "giter_s": iters / span / 1e9 if span else None,
            "offered_giter_s": offered, "iterations": iters, "rounds": c["rounds"], "peak_gb": c["peak_bytes"] / 1e9,
            "budget_gb": 40 * 2 ** 30 / 1e9}


# FP32-pipe operations per escape step of the reduced-precision lanes: binary32 =
# 3 multiplies, 1 doubling, 4 adds; double-float = 3 double-word products
# (9 each), 4 double-word sums (20 each), 2 adds for the doubling.
LOWP_OPS_PER_STEP = {"fp32": 8, "dfloat": 109}
FP32_LANES_PER_SM = 128


def precision_variants(mb, v, ref, stream, clocks, args):
    """Binary32 and double-float renders of the headline view: each variant's
    own throughput (its own iteration count), the fraction of the FP32 pipe it
    keeps busy, and how many pixels differ from the binary64 image `ref`."""
    import torch
    E = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    sms, _ = mb.mb_device_info(args.block)
    mhz = clocks.get("sm_mhz") or 2070.0
    lo = torch.empty_like(ref)
    total = torch.zeros(1, dtype=torch.int64, device=ref.device)
    res = {}
    for prec in ("fp32", "dfloat"):
        runs = {}
        for sched, tile in (("fcfs_rows", 64), ("fcfs_tiles", 16)):
            for unroll in (8, 16):
                kw = dict(sched=sched, tile=tile, block=args.block, unroll=unroll, precision=prec, stream=stream)
                mb.mb_render(v.window, v.m, v.n, v.iter_max, v.r2, lo, **kw)
                a, b = E(), E()
                a.record(stream)
                mb.mb_render(v.window, v.m, v.n, v.iter_max, v.r2, lo, **kw)
                b.record(stream)
                b.synchronize()
                runs["%s_u%d" % (sched, unroll)] = a.elapsed_time(b)
        mb.mb_sum_counts(lo, total, stream=stream)
        torch.cuda.synchronize()
        iters = int(total.item())
        differ = int((lo != ref).sum().item())
        cls = int(((lo == v.iter_max) != (ref == v.iter_max)).sum().item())
        best = min(runs, key=runs.get)
        steps_s = iters / (runs[best] * 1e-3)
        res[prec] = {"best": best, "ms": runs[best], "giter_s": steps_s / 1e9, "iterations": iters,
                     "ms_by_launch": runs, "fp32_ops_per_step": LOWP_OPS_PER_STEP[prec],
                     "fp32_pipe_frac": steps_s * LOWP_OPS_PER_STEP[prec] / (sms * FP32_LANES_PER_SM * mhz * 1e6),
                     "pixels_differing_from_fp64": differ / ref.numel(),
                     "interior_exterior_disagree": cls / ref.numel()}
    res["note"] = ("not the paper's method: counts are exact for each variant's own operation sequence "
                   "(parity tests) and differ from binary64 on the fraction shown; fp32_pipe_frac uses "
                   "%d SMs x %d lanes at the sampled SM clock" % (sms, FP32_LANES_PER_SM))
    return res


def measured_hbm_gbs():
    """Copy bandwidth of this GPU model from MEASURED_PEAKS.json at the repository root, if present."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, ValueError, KeyError, TypeError):
        return None


def roofline_entry(steps, kernel_ms, peak, traffic, issued_per_step=None):
    """Roofline of the main render launch: `steps` escape steps in `kernel_ms`,
    against the FP64-pipe issue rate `peak` (binary64 ops/s) measured in this run.
    The FP64 pipe carries 2.5 of a step's 8 nominal binary64 ops on average (the
    three additions, less the subtraction of every other step, which runs exactly
    on the integer pipes), so the attainable rate of the 8 ops is peak x 8/2.5,
    as long as the integer pipes keep up (they are co-saturated: ncu shows FP64
    ~80 % and integer ALU ~80 % busy).  With `issued_per_step` (FP64 instructions that
    ncu counted per step, idle lanes and replays included) the entry also gives the
    FP64 pipe's fraction by issued instructions."""
    step_peak = peak * ALG_OPS_PER_ITER / FP64_PIPE_OPS_PER_ITER
    achieved = steps * ALG_OPS_PER_ITER / (kernel_ms * 1e-3)
    return {"bound": "alu", "achieved": achieved / 1e12, "peak": step_peak / 1e12, "unit": "TFLOP/s",
            "frac": achieved / step_peak, "traffic": traffic,
            "peak_source": ("derived from measured (of measured): the FP64-pipe issue rate measured now "
                            "by mb_fp64_peak (%.4f T binary64 ops/s) x 8/2.5 -- an escape step's 8 "
                            "nominal binary64 ops need 2.5 FP64-pipe issues on average (its three "
                            "additions, less the subtraction that every other step does on the integer "
                            "pipes); the products and the doubling run exactly on the integer pipes, "
                            "which are co-saturated with the FP64 pipe" % (peak / 1e12)),
            "fp64_pipe_frac": FP64_PIPE_OPS_PER_ITER * steps / (kernel_ms * 1e-3) / peak,
            "fp64_pipe_frac_issued": (issued_per_step * steps / (kernel_ms * 1e-3) / peak
                                      if issued_per_step else None),
            "nominal_frac": achieved / peak,
            "nominal_note": "8 nominal ops per step over the plain FP64-pipe peak (the metric's "
                            "'% of FP64 peak' form, above 1 because 5.5 of the 8 ops are not FP64-pipe "
                            "instructions)",
            "kernel": "render_kernel (main FCFS render, CUDA events around its launch)",
            "algorithmic": "8 binary64 ops per escape step x %d steps per launch" % steps,
            "dram_gbs": traffic / (kernel_ms * 1e-3) / 1e9 if traffic else None,
            "dram_frac_of_measured_hbm": (traffic / (kernel_ms * 1e-3) / 1e9 / measured_hbm_gbs()
                                          if traffic and measured_hbm_gbs() else None)}


def spearman(a, b):
    """Rank correlation of two 1-D arrays (ties broken by position)."""
    import numpy as np
    ra = np.empty(len(a)); ra[np.argsort(a, kind="stable")] = np.arange(len(a))
    rb = np.empty(len(b)); rb[np.argsort(b, kind="stable")] = np.arange(len(b))
    return float(np.corrcoef(ra, rb)[0, 1])


def model_quality(mb, v, params, tile, stream):
    """How well the trained network predicts the view's per-tile costs, next to
    the probe-sum estimate it corrects: rank correlation with the true tile
    totals (recorded by the renderer) and RMSE on the log2(1 + total) / 32
    scale the model is trained on."""
    import numpy as np
    import torch
    nt = ((v.m + tile - 1) // tile) * ((v.n + tile - 1) // tile)
    probe = torch.empty(nt * 64, dtype=torch.int32, device="cuda")
    mb.mb_probe(v.window, v.m, v.n, v.iter_max, v.r2, probe, tile=tile, stream=stream)
    feat = torch.empty((nt, 70), dtype=torch.float32, device="cuda")
    mb.mb_tile_features(probe, v.window, v.m, v.n, v.iter_max, tile, feat, stream=stream)
    y = torch.empty(nt, dtype=torch.float32, device="cuda")
    mb.mb_mlp_forward(params, feat, nt, y, stream=stream)
    tot = torch.zeros(nt, dtype=torch.int64, device="cuda")
    out = torch.empty(v.m * v.n, dtype=torch.int32, device="cuda")
    mb.mb_render(v.window, v.m, v.n, v.iter_max, v.r2, out, sched="fcfs_tiles", tile=tile, tile_totals=tot,
                 stream=stream)
    tgt = torch.empty(nt, dtype=torch.float32, device="cuda")
    mb.mb_tile_targets(tot, nt, tgt, stream=stream)
    torch.cuda.synchronize()
    t = tgt.cpu().numpy().astype(np.float64)
    net = y.cpu().numpy().astype(np.float64)
    ps = feat[:, 68].cpu().numpy().astype(np.float64)
    return {"tiles": nt, "tile": tile,
            "spearman": {"network": spearman(net, t), "probe_sum": spearman(ps, t)},
            "rmse_log2_cost_over_32": {"network": float(np.sqrt(np.mean((net - t) ** 2))),
                                       "probe_sum": float(np.sqrt(np.mean((ps - t) ** 2)))}}


def cycle_variant(mb, v, ref, stream, args):
    """Time to the same binary64 image with exact cycle detection (mb_opts.cycle_check)
    against the same launch without it.  Reported as time only: the detected
    pixels' remaining steps do not run, so a Giter/s figure would count steps
    that were never executed."""
    import torch
    E = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    got = torch.empty_like(ref)
    res = {}
    for name, kw in (("fcfs_rows", dict(sched="fcfs_rows", tile=64)), ("fcfs_tiles16", dict(sched="fcfs_tiles", tile=16))):
        t = {}
        for cyc in (0, 1):
            kws = dict(kw, block=args.block, unroll=args.unroll, stream=stream, cycle_check=cyc)
            mb.mb_render(v.window, v.m, v.n, v.iter_max, v.r2, got, **kws)
            a, b = E(), E()
            a.record(stream)
            mb.mb_render(v.window, v.m, v.n, v.iter_max, v.r2, got, **kws)
            b.record(stream)
            b.synchronize()
            t[cyc] = a.elapsed_time(b)
        res[name] = {"ms_full_iteration": t[0], "ms_cycle_check": t[1], "speedup": t[0] / t[1],
                     "same_image": bool(torch.equal(got, ref))}
    res["note"] = ("exact shortcut, not in the paper: a pixel whose binary64 state repeats bit for bit at a "
                   "block start is periodic and never escapes, so it gets iterMax at once; the image is "
                   "identical (same_image) and only time is reported")
    return res


def run_sharded(args, ws, rank, local):
    """N > 1: one image per step, rendered across the N GPUs.  The raster tile list is
    cut into chunks that a counter in the job's store (served by rank 0, the paper's
    master) hands out first come first served (Sec. III-B one level up); each GPU
    renders its chunks with the item scheduler and sends only their pixels to rank 0
    (packed gather).  Strong scaling: the work per step is one image whatever N is."""
    import torch
    import torch.distributed as dist

    from paper_2007_00745_gb300 import shard
    torch.cuda.set_device(local)
    store = shard.make_store(rank, ws)
    dist.init_process_group("nccl", store=store, rank=rank, world_size=ws)
    try:
        import paper_2007_00745_gb300 as mb
        mb.mb_version()
    except ImportError:
        import __graft_entry__
        __graft_entry__.build()
        import paper_2007_00745_gb300 as mb
    v = bench_view(args)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    total = torch.zeros(1, dtype=torch.int64, device=dev)
    opts = dict(block=args.block, unroll=args.unroll)

    def step(stats=None):
        return shard.render_sharded(v.window, v.m, v.n, v.iter_max, v.r2, tile=args.tile, store=store, stats=stats,
                                    **opts)

    img = step()
    if rank == 0:
        mb.mb_sum_counts(img, total, stream=stream)
    dist.broadcast(total, src=0)
    iters = int(total.item())
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    E = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    stats = [dict() for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        dist.barrier()
        torch.cuda.synchronize()
        t0, t1 = E(), E()
        t0.record(stream)
        for k in range(args.steps):
            img = step(stats[k])
        t1.record(stream)
        torch.cuda.synchronize()
        dist.barrier()
    tt = torch.tensor([t0.elapsed_time(t1)], dtype=torch.float64, device=dev)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    ms_step = float(tt.item()) / args.steps
    clocks = clk.summary()
    chunks = torch.tensor([sum(len(s_["chunks"]) for s_ in stats)], dtype=torch.int64, device=dev)
    per_rank = [torch.zeros_like(chunks) for _ in range(ws)]
    dist.all_gather(per_rank, chunks)
    # end to end: the same step with rank 0's assembled image read back into pinned host memory
    host = torch.empty(v.m * v.n, dtype=torch.int32, pin_memory=True) if rank == 0 else None
    dist.barrier()
    torch.cuda.synchronize()
    a, b = E(), E()
    a.record(stream)
    img = step()
    if rank == 0:
        host.copy_(img, non_blocking=True)
    b.record(stream)
    torch.cuda.synchronize()
    et = torch.tensor([a.elapsed_time(b)], dtype=torch.float64, device=dev)
    dist.all_reduce(et, op=dist.ReduceOp.MAX)
    if rank != 0:
        dist.destroy_process_group()
        return
    peak = max(mb.mb_fp64_peak(0)[0], mb.mb_fp64_peak(1)[0]) if not args.no_peak else float("nan")
    value = iters / (ms_step * 1e-3) / 1e9
    step_peak = ws * peak * ALG_OPS_PER_ITER / FP64_PIPE_OPS_PER_ITER
    achieved = iters * ALG_OPS_PER_ITER / (ms_step * 1e-3)
    cfg = bench_config(args, v, ws)
    line = {
        "metric": "Giter/s", "value": value, "unit": "Giter/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg, "iterations_per_step": iters,
        "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": step_peak / 1e12, "unit": "TFLOP/s",
                     "frac": achieved / step_peak, "traffic": None,
                     "kernel": "whole sharded step (all chunks' render launches plus the gather) over %d GPUs" % ws,
                     "peak_source": "derived from measured (of measured): %d x mb_fp64_peak x 8/2.5" % ws},
        "clocks": clocks,
        "chunks_per_rank": [int(x.item()) / args.steps for x in per_rank],
        "e2e": {"value": iters / (float(et.item()) * 1e-3) / 1e9, "unit": "Giter/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": v.m * v.n * 4,
                "note": "the same step with rank 0's assembled image copied to pinned host memory"},
        "gpu_launches": int(sum(x.item() for x in per_rank)) * 2 + (ws - 1) * 2 * args.steps,
    }
    if not args.no_cpu_baseline:
        dts = []
        for _ in range(max(args.cpu_reps, 1)):
            it, dt, nrows, cores = cpu_sample(v, max(args.cpu_rows_stride, 1))
            dts.append(dt)
        dt = sum(dts) / len(dts)
        line["cpu_baseline"] = {"value": it / dt / 1e9, "unit": "Giter/s", "cores": cores, "kind": "oracle",
                                "sample": "%d of %d rows (every %d-th), %d iterations, mean of %d runs of %.1f s"
                                          % (nrows, v.m, max(args.cpu_rows_stride, 1), it, len(dts), dt)}
    print(json.dumps(line), flush=True)
    dist.destroy_process_group()


def run_ours(args):
    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        return run_sharded(args, ws, rank, local)
    torch.cuda.set_device(local)
    try:
        import paper_2007_00745_gb300 as mb
        mb.mb_version()
    except ImportError:
        import __graft_entry__
        __graft_entry__.build()
        import paper_2007_00745_gb300 as mb
    from paper_2007_00745_gb300 import tilemodel, workloads as wl

    v = bench_view(args)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    out = torch.empty(v.m * v.n, dtype=torch.int32, device=dev)
    host = torch.empty(v.m * v.n, dtype=torch.int32, pin_memory=True)
    total = torch.zeros(1, dtype=torch.int64, device=dev)
    learned = args.sched == "learned"
    ropts = dict(tile=args.tile, block=args.block, unroll=args.unroll, stream=stream)
    lopts = dict(ropts, min_strips=args.min_strips)

    peak = float("nan")
    if not args.no_peak:
        peak = max(mb.mb_fp64_peak(0)[0], mb.mb_fp64_peak(1)[0])

    params, train_s = None, None
    if learned:
        t = time.perf_counter()
        params, _ = tilemodel.default_model(tile=args.tile, stream=stream)
        torch.cuda.synchronize()
        train_s = time.perf_counter() - t

    def step(events=None):
        if learned:
            mb.mb_render_learned(v.window, v.m, v.n, v.iter_max, v.r2, out, params, events=events, **lopts)
        else:
            mb.mb_render(v.window, v.m, v.n, v.iter_max, v.r2, out, sched=args.sched, events=events, **ropts)

    # iterations of the view (the same for every scheduler) and of the probe
    # (computed before, and skipped by, the main render kernel)
    step()
    mb.mb_sum_counts(out, total, stream=stream)
    torch.cuda.synchronize()
    iters = int(total.item())
    probe_iters = 0
    if learned:
        nt = tilemodel.tiles_of(v.m, v.n, args.tile)
        pr = torch.empty(nt * 64, dtype=torch.int32, device=dev)
        mb.mb_probe(v.window, v.m, v.n, v.iter_max, v.r2, pr, tile=args.tile, stream=stream)
        mb.mb_sum_counts(pr, total, stream=stream)
        torch.cuda.synchronize()
        probe_iters = int(total.item())

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    def E():
        return torch.cuda.Event(enable_timing=True)

    kev = [(E(), E()) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        t0, t1 = E(), E()
        t0.record(stream)
        for k in range(args.steps):
            step(events=kev[k])
        t1.record(stream)
        torch.cuda.synchronize()
    ms_total = t0.elapsed_time(t1)
    kernel_ms = sum(a.elapsed_time(b) for a, b in kev) / args.steps
    clocks = clk.summary()
    ms_step = ms_total / args.steps
    value = iters / (ms_step * 1e-3) / 1e9

    # roofline of the dominant kernel: the main render, timed by its own events
    render_iters = iters - probe_iters
    traffic = None
    pipes = None
    issued = None
    if NCU_RENDER["src_sha1"] == kernel_sha1() and NCU_RENDER["unroll"] == args.unroll:
        traffic = NCU_RENDER["dram_bytes_per_pixel"] * v.m * v.n
        pipes = NCU_RENDER["pipes"]
        issued = NCU_RENDER["fp64_issued_per_step"]
    line = {
        "metric": "Giter/s", "value": value, "unit": "Giter/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": bench_config(args, v, ws),
        "iterations_per_step": iters,
        "roofline": dict(roofline_entry(render_iters, kernel_ms, peak, traffic, issued),
                         ncu_pipe_busy=pipes,
                         ncu_pipe_note="busy fraction of each pipe in the ncu capture of this kernel (8192^2, "
                                       "iterMax 1000): the FP64 pipe's own ceiling is ~0.84 (the peak "
                                       "microbenchmark's), the integer ALU's issue limit 1.0"),
        "pct_fp64_peak": 100.0 * value * 1e9 * ALG_OPS_PER_ITER / peak,
        "kernel_ms": kernel_ms,
        "clocks": clocks,
        "gpu_launches": (6 if learned else 2) * args.steps,
    }
    if learned:
        line["model"] = {"train_s": train_s, "probe_iterations": probe_iters}
        if not args.no_compare:
            line["model"]["quality"] = model_quality(mb, v, params, args.tile, stream)

    if not args.no_e2e:
        e2e = []
        for _ in range(3):
            a, b = E(), E()
            torch.cuda.synchronize()
            a.record(stream)
            step()
            host.copy_(out, non_blocking=True)
            b.record(stream)
            b.synchronize()
            e2e.append(a.elapsed_time(b))
        ems = sum(e2e) / len(e2e)
        copy_e2e = {"value": iters / (ems * 1e-3) / 1e9, "unit": "Giter/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": v.m * v.n * 4, "ms_per_step": ems,
                    "note": "inputs are five scalars passed by value; counts rendered on the device, "
                            "then copied to pinned host memory"}
        # the same step with the counts written by the kernels straight into pinned host memory
        direct = []
        for _ in range(3):
            a, b = E(), E()
            torch.cuda.synchronize()
            a.record(stream)
            if learned:
                mb.mb_render_learned(v.window, v.m, v.n, v.iter_max, v.r2, host, params, **lopts)
            else:
                mb.mb_render(v.window, v.m, v.n, v.iter_max, v.r2, host, sched=args.sched, **ropts)
            b.record(stream)
            b.synchronize()
            direct.append(a.elapsed_time(b))
        dms = sum(direct) / len(direct)
        step()
        torch.cuda.synchronize()
        same = bool(torch.equal(out.cpu(), host))
        direct_e2e = {"value": iters / (dms * 1e-3) / 1e9, "unit": "Giter/s", "h2d_bytes_per_step": 0,
                      "d2h_bytes_per_step": v.m * v.n * 4, "ms_per_step": dms, "same_counts": same,
                      "note": "inputs are five scalars passed by value; the kernels store every count "
                              "straight into pinned host memory (NVLink-C2C on GB300), so no copy step"}
        line["e2e"] = direct_e2e if same and dms < ems else copy_e2e
        line["e2e_variants"] = {"direct_to_host": direct_e2e, "device_then_copy": copy_e2e}

    if not args.no_e2e:
        # The paper's two timings (Sec. IV listing): computation, and total including the image file.
        rgb = torch.empty(v.m * v.n * 3, dtype=torch.uint8, device=dev)
        rgb_host = torch.empty(v.m * v.n * 3, dtype=torch.uint8, pin_memory=True)
        path = args.ppm or os.path.join(tempfile.mkdtemp(prefix="mb_ppm_"), "Mandelbrot.ppm")
        torch.cuda.synchronize()
        t_a = time.perf_counter()
        step()
        torch.cuda.synchronize()
        t_b = time.perf_counter()
        mb.mb_colorize(out, v.iter_max, rgb, stream=stream)
        rgb_host.copy_(rgb, non_blocking=True)
        torch.cuda.synchronize()
        mb.mb_write_ppm(path, rgb_host, v.m, v.n)
        t_c = time.perf_counter()
        line["paper_timings"] = {"computational_s": t_b - t_a, "total_s": t_c - t_a, "ppm_bytes": os.path.getsize(path)}
        if not args.ppm:
            os.unlink(path)
            os.rmdir(os.path.dirname(path))

    if not args.no_compare:
        sms, per = mb.mb_device_info(args.block)
        g = sms * per
        cmp = {}
        variants = [("naive", dict(sched="naive", tile=64)), ("alternating", dict(sched="alternating", tile=64)),
                    ("fcfs_rows", dict(sched="fcfs_rows", tile=64)), ("fcfs_tiles64", dict(sched="fcfs_tiles", tile=64)),
                    ("fcfs_tiles32", dict(sched="fcfs_tiles", tile=32)), ("fcfs_tiles16", dict(sched="fcfs_tiles", tile=16)),
                    ("learned", None), ("probe_sum", "probe"),
                    ("learned64", "learned64"), ("lpt_exact16", ("lpt", 16)), ("lpt_exact32", ("lpt", 32))]
        params64 = tilemodel.default_model(tile=64, stream=stream)[0] if params is not None else None
        # the bound on any ordering: tiles longest-first by their true cost (per-tile totals of an
        # untimed render), which no prediction can beat
        lpt_items = {}
        for T in (16, 32):
            tt = torch.zeros((-(-v.m // T)) * (-(-v.n // T)), dtype=torch.int64, device=dev)
            mb.mb_render(v.window, v.m, v.n, v.iter_max, v.r2, out, sched="fcfs_tiles", tile=T, tile_totals=tt,
                         block=args.block, unroll=args.unroll, stream=stream)
            torch.cuda.synchronize()
            order = torch.argsort(tt, descending=True, stable=True)
            it = torch.empty((order.numel(), 2), dtype=torch.int32, device=dev)
            it[:, 0] = order.to(torch.int32)
            it[:, 1] = T << 16
            lpt_items[T] = it
        for name, kw in variants:
            if kw in (None, "learned64") and params is None:
                continue
            tr = torch.zeros(g * 3, dtype=torch.int64, device=dev)
            a, b = E(), E()
            a.record(stream)
            if kw is None or kw == "probe":   # learned order, or its ablation ordered by the probe sum
                mb.mb_render_learned(v.window, v.m, v.n, v.iter_max, v.r2, out, params if kw is None else None,
                                     tile=args.tile, block=args.block, unroll=args.unroll, grid=g, trace=tr,
                                     min_strips=args.min_strips, stream=stream)
            elif kw == "learned64":           # the learned pipeline on 64-pixel tiles (a 1/64 probe), 16 strips
                mb.mb_render_learned(v.window, v.m, v.n, v.iter_max, v.r2, out, params64, tile=64,
                                     block=args.block, unroll=args.unroll, grid=g, trace=tr, min_strips=16,
                                     stream=stream)
            elif isinstance(kw, tuple):        # exact longest-first order (the bound), no probe
                T = kw[1]
                mb.mb_render(v.window, v.m, v.n, v.iter_max, v.r2, out, sched="fcfs_items", items=lpt_items[T],
                             n_items=int(lpt_items[T].shape[0]), tile=T, block=args.block, unroll=args.unroll,
                             grid=g, trace=tr, stream=stream)
            else:
                mb.mb_render(v.window, v.m, v.n, v.iter_max, v.r2, out, block=args.block, unroll=args.unroll,
                             grid=g, trace=tr, stream=stream, **kw)
            b.record(stream)
            torch.cuda.synchronize()
            st = trace_stats(tr.cpu().numpy().reshape(-1, 3), sms)
            st["ms"] = a.elapsed_time(b)
            st["giter_s"] = iters / (st["ms"] * 1e-3) / 1e9
            cmp[name] = st
        line["schedulers"] = cmp
        line["schedulers_note"] = ("makespan = first CTA start to last CTA end of the render kernel; ms = the whole call "
                                   "(learned, probe_sum and learned64 include the probe and the ordering); "
                                   "lpt_exact16/32 = the same tiles queued longest-first by their true cost (from an "
                                   "untimed render's per-tile totals): the bound on any ordering of those tiles")
        if params64 is not None:
            # where the order matters: the same size and budget with the set's interior in the last
            # rows of the raster order; raster FCFS over 64-pixel tiles against the learned order of
            # the same tiles (probe included), and raster FCFS over 16-pixel tiles
            hv = wl.View(wl.HEAVY_LAST.window, v.m, v.n, v.iter_max, v.r2)
            hres = {}
            for name, kw in (("fcfs_tiles64", dict(sched="fcfs_tiles", tile=64)),
                             ("learned64", None), ("fcfs_tiles16", dict(sched="fcfs_tiles", tile=16))):
                a, b = E(), E()
                a.record(stream)
                if kw is None:
                    mb.mb_render_learned(hv.window, hv.m, hv.n, hv.iter_max, hv.r2, out, params64, tile=64,
                                         block=args.block, unroll=args.unroll, grid=g, min_strips=16, stream=stream)
                else:
                    mb.mb_render(hv.window, hv.m, hv.n, hv.iter_max, hv.r2, out, block=args.block,
                                 unroll=args.unroll, grid=g, stream=stream, **kw)
                b.record(stream)
                torch.cuda.synchronize()
                hres[name] = {"ms": a.elapsed_time(b)}
            line["order_heavy_last"] = dict(
                hres, window=list(hv.window),
                note="the set's interior in the last rows of the raster order: raster FCFS over 64-pixel tiles "
                     "ends on its heaviest tiles; the learned order (probe included) takes them first")
        # the small plain-method view (640 x 480, iterMax 1000, naive rows).  With the default grid
        # (G CTAs) the paper's remainder rule (Sec. III-A) gives floor(480 / G) rows to each CTA and the
        # m mod G remaining rows to the last one, so the launch is that CTA's serial tail; the paper's
        # own worker counts N = 2..32 are timed beside it.
        c1 = wl.FULL_VIEW_1
        c1o = torch.empty(c1.m * c1.n, dtype=torch.int32, device=dev)

        def c1_time(grid):
            mb.mb_render(c1.window, c1.m, c1.n, c1.iter_max, c1.r2, c1o, sched="naive", grid=grid, stream=stream)
            a, b = E(), E()
            a.record(stream)
            for _ in range(10):
                mb.mb_render(c1.window, c1.m, c1.n, c1.iter_max, c1.r2, c1o, sched="naive", grid=grid,
                             stream=stream)
            b.record(stream)
            b.synchronize()
            return a.elapsed_time(b) / 10

        c1ms = c1_time(0)
        mb.mb_sum_counts(c1o, total, stream=stream)
        torch.cuda.synchronize()
        c1it = int(total.item())
        per, last = c1.m // g, c1.m // g + c1.m % g
        workers = {}
        for nw in (2, 4, 8, 16, 32):
            ms = c1_time(nw)
            workers[str(nw)] = {"ms": ms, "giter_s": c1it / (ms * 1e-3) / 1e9,
                                "rows_per_cta": c1.m // nw, "last_cta_rows": c1.m // nw + c1.m % nw}
        line["config1_640x480"] = {"sched": "naive", "grid": g, "rows_per_cta": per, "last_cta_rows": last,
                                   "last_cta_row_share": last / c1.m, "ms": c1ms, "iterations": c1it,
                                   "giter_s": c1it / (c1ms * 1e-3) / 1e9, "paper_worker_counts": workers,
                                   "note": "naive rows under the paper's remainder rule: with %d CTAs the last "
                                           "CTA owns %d of the %d rows, so the launch is its serial tail"
                                           % (g, last, c1.m)}
        if "naive" in cmp and "learned" in cmp:
            line["learned_vs_naive"] = {"speedup": cmp["naive"]["ms"] / cmp["learned"]["ms"],
                                        "makespan_ratio": cmp["learned"]["makespan_ms"] / cmp["naive"]["makespan_ms"]}

    if not args.no_precision:
        line["precision_variants"] = precision_variants(mb, v, out, stream, clocks, args)
    if not args.no_cycle:
        line["cycle_check"] = cycle_variant(mb, v, out, stream, args)

    if not args.no_batch:
        views = wl.batch_views(args.batch_count)
        outs = [torch.empty(q.m * q.n, dtype=torch.int32, device=dev) for q in views]
        cache = os.path.join(ROOT, "paper_2007_00745_gb300", "_build", "autotune_cache.txt")
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        best, tune_ms = mb.mb_batch_autotune(views, outs, sample_stride=8, cache_path=cache)
        sms, per = mb.mb_device_info(best["block"])
        g = sms * per
        btr = torch.zeros(g * 3, dtype=torch.int64, device=dev)

        def time_plan(plan, reps=2):
            plan.launch()
            torch.cuda.synchronize()
            ms = []
            for _ in range(reps):
                a, b = E(), E()
                a.record()
                plan.launch()
                b.record()
                b.synchronize()
                ms.append(a.elapsed_time(b))
            st = trace_stats(btr.cpu().numpy().reshape(-1, 3), sms)
            return min(ms), st

        plan = mb.BatchPlan(views, outs, trace=btr, **best)
        bm, bst = time_plan(plan)
        bi = 0
        for o in outs:
            mb.mb_sum_counts(o, total)
            torch.cuda.synchronize()
            bi += int(total.item())
        info = plan.info()
        plan.destroy()
        line["batch"] = {"workload": "%d viewports, sides U(256..4096), widths log-U(1e-9..1e-1), " % len(views) +
                                     "iterMax log-U(256..65536), one persistent launch, CUDA graph replay",
                         "giter_s": bi / (bm * 1e-3) / 1e9, "ms": bm, "iterations": bi, "items": info["items"],
                         "pixels": info["pixels"], "autotuned": best, "autotune_sample_ms": tune_ms,
                         "queue": "views by decreasing iterMax, tiles in raster order",
                         "makespan_ms": bst["makespan_ms"], "idle_tail": bst["idle_tail"]}
        # the same batch with the learned queue: every view probed once when the plan is built,
        # (view, tile) items of all views longest-first by the tile-cost network, heavy tiles split
        if best["tile"] >= 16:
            bparams = tilemodel.default_model(tile=best["tile"], stream=stream)[0]
            louts = [torch.empty_like(o) for o in outs]
            t = time.perf_counter()
            lplan = mb.BatchPlan(views, louts, trace=btr, learned_order=1, model=bparams, **best)
            torch.cuda.synchronize()
            build_s = time.perf_counter() - t
            lm, lst = time_plan(lplan)
            linfo = lplan.info()
            lplan.destroy()
            same = all(bool(torch.equal(x, y)) for x, y in zip(outs, louts))
            line["batch"]["learned"] = {"giter_s": bi / (lm * 1e-3) / 1e9, "ms": lm, "items": linfo["items"],
                                        "makespan_ms": lst["makespan_ms"], "idle_tail": lst["idle_tail"],
                                        "plan_build_s": build_s, "same_counts": same,
                                        "speedup_vs_default_queue": bm / lm}
            del louts
        if not args.no_cycle:   # the same batch with exact cycle detection: time and identical counts only
            couts = [torch.empty_like(o) for o in outs]
            cplan = mb.BatchPlan(views, couts, cycle_check=1, **best)
            cplan.launch()
            a, b = E(), E()
            a.record()
            cplan.launch()
            b.record()
            b.synchronize()
            cplan.destroy()
            same = all(bool(torch.equal(x, y)) for x, y in zip(outs, couts))
            line["batch"]["cycle_check"] = {"ms": a.elapsed_time(b), "speedup": bm / a.elapsed_time(b),
                                            "same_counts": same}
            del couts
        del outs

    if not args.no_serve:
        line["serve"] = run_serve(mb, wl, torch, 50.0, args.serve_count)
        if not args.no_cycle:   # the same request stream with exact cycle detection: latency only
            sc = run_serve(mb, wl, torch, 50.0, args.serve_count, cycle_check=1)
            sc["giter_s"] = None
            sc["note"] = ("cycle_check=1: identical counts; detected pixels skip their remaining steps, so "
                          "only latency and completions are reported")
            line["serve_cycle_check"] = sc
    if args.serve_sweep and not args.no_serve:
        # one fixed draw of requests, replayed at every rate (only the arrival times scale)
        sweep_views = wl.batch_views(count=args.serve_sweep_count, seed=wl.SEED + 600)
        runs = [run_serve(mb, wl, torch, float(r), args.serve_sweep_count, views=sweep_views)
                for r in args.serve_sweep.split(",")]
        line["serve_sweep"] = {"requests_per_rate": args.serve_sweep_count, "draw": "batch_views(seed=SEED+600)",
                               "note": "offered_giter_s = rate x mean iterations per request; below the render "
                                       "rate the arrivals bound the delivered Giter/s, above it queueing sets p99",
                               "rates": runs}
        # the same draw with the learned tile order in every request (probe, network, guard, rank),
        # at the sweep's two lowest rates and its highest
        if params is not None:
            rates = sorted(float(r) for r in args.serve_sweep.split(","))
            pick = sorted(set(rates[:2] + rates[-1:]))
            line["serve_sweep"]["learned_order"] = [
                run_serve(mb, wl, torch, r, args.serve_sweep_count, views=sweep_views, learned_order=1, model=params,
                          tile=args.tile) for r in pick]

    if not args.no_zoom:
        z = wl.ZOOM_3
        zo = torch.empty(z.m * z.n, dtype=torch.int32, device=dev)
        zparams = tilemodel.default_model(tile=64)[0] if params is not None else None
        runs = [("learned64", lambda: mb.mb_render_learned(z.window, z.m, z.n, z.iter_max, z.r2, zo, zparams, tile=64,
                                                          block=args.block, unroll=args.unroll)),
                ("probe_sum64", lambda: mb.mb_render_learned(z.window, z.m, z.n, z.iter_max, z.r2, zo, None, tile=64,
                                                            block=args.block, unroll=args.unroll)),
                ("fcfs_tiles64", lambda: mb.mb_render(z.window, z.m, z.n, z.iter_max, z.r2, zo, sched="fcfs_tiles",
                                                     tile=64, block=args.block)),
                ("fcfs_tiles16", lambda: mb.mb_render(z.window, z.m, z.n, z.iter_max, z.r2, zo, sched="fcfs_tiles",
                                                     tile=16, block=args.block)),
                ("naive", lambda: mb.mb_render(z.window, z.m, z.n, z.iter_max, z.r2, zo, sched="naive",
                                              block=args.block))]
        zc = {}
        for name, fn in runs:
            if name == "learned64" and params is None:
                continue
            a, b = E(), E()
            a.record()
            fn()
            b.record()
            b.synchronize()
            zc[name] = {"ms": a.elapsed_time(b)}
        mb.mb_sum_counts(zo, total)
        torch.cuda.synchronize()
        zi = int(total.item())
        for k in zc:
            zc[k]["giter_s"] = zi / (zc[k]["ms"] * 1e-3) / 1e9
        line["zoom16384"] = {"iterations": zi, "variants": zc}
        if zparams is not None:
            line["zoom16384"]["model_quality"] = model_quality(mb, z, zparams, 64, None)
        if not args.no_precision:   # the reduced-precision variants on the deep zoom (pixel spacing 6e-10)
            zl = torch.empty_like(zo)
            lowp = {}
            for prec in ("dfloat", "fp32"):
                a, b = E(), E()
                a.record()
                mb.mb_render(z.window, z.m, z.n, z.iter_max, z.r2, zl, sched="fcfs_tiles", tile=16,
                             block=args.block, unroll=16, precision=prec)
                b.record()
                b.synchronize()
                mb.mb_sum_counts(zl, total)
                torch.cuda.synchronize()
                ms = a.elapsed_time(b)
                lowp[prec] = {"ms": ms, "giter_s": int(total.item()) / (ms * 1e-3) / 1e9,
                              "iterations": int(total.item()),
                              "pixels_differing_from_fp64": float((zl != zo).float().mean().item())}
            line["zoom16384"]["precision_variants"] = lowp
        if not args.no_cycle:   # exact cycle detection on the deep zoom: time and identical counts only
            zc2 = torch.empty_like(zo)
            a, b = E(), E()
            a.record()
            mb.mb_render(z.window, z.m, z.n, z.iter_max, z.r2, zc2, sched="fcfs_tiles", tile=16, block=args.block,
                         cycle_check=1)
            b.record()
            b.synchronize()
            line["zoom16384"]["cycle_check"] = {"ms": a.elapsed_time(b),
                                                "speedup_vs_fcfs_tiles16": zc["fcfs_tiles16"]["ms"] / a.elapsed_time(b),
                                                "same_counts": bool(torch.equal(zc2, zo))}
            del zc2

    if args.table2:
        from paper_2007_00745_gb300 import report
        p = wl.PAPER_SHAPE
        pv = wl.scaled(p, 2000, 2000)   # same window, budget and R^2 as Sec. IV's test, 1/16 of the pixels
        po = torch.empty(pv.m * pv.n, dtype=torch.int32, device=dev)
        workers = [1, 2, 4, 8, 16, 32, 64, 152, 304]
        times = {}
        for sched in ("naive", "alternating", "fcfs_rows"):
            times[sched] = {}
            for g in workers:
                a, b = E(), E()
                a.record()
                mb.mb_render(pv.window, pv.m, pv.n, pv.iter_max, pv.r2, po, sched=sched, grid=g, block=args.block,
                             unroll=args.unroll)
                b.record()
                b.synchronize()
                times[sched][g] = a.elapsed_time(b) * 1e-3
        mb.mb_sum_counts(po, total)
        torch.cuda.synchronize()
        tab = report.scaling_table(times)
        line["table2"] = {"workload": "2000x2000 re[-2,1] im[-1.5,1.5] iterMax 2000 R2 160000 (paper Sec. IV shape, "
                                      "1/16 of its pixels); workers = CTAs of %d threads" % args.block,
                          "iterations": int(total.item()),
                          "seconds": {s_: {str(g): t for g, t in r.items()} for s_, r in times.items()},
                          "speedup": {s_: {str(g): round(x[0], 3) for g, x in r.items()} for s_, r in tab.items()},
                          "pct_diff_vs_linear": {s_: {str(g): round(x[1], 2) for g, x in r.items()}
                                                 for s_, r in tab.items()}}

    if not args.no_cpu_baseline:
        # the same row sample that `--impl reference` times each step, repeated cpu_reps times
        dts = []
        for _ in range(max(args.cpu_reps, 1)):
            it, dt, nrows, cores = cpu_sample(v, max(args.cpu_rows_stride, 1))
            dts.append(dt)
        dt = sum(dts) / len(dts)
        line["cpu_baseline"] = {"value": it / dt / 1e9, "unit": "Giter/s", "cores": cores, "kind": "oracle",
                                "sample": "%d of %d rows (every %d-th), %d iterations, mean of %d runs of %.1f s"
                                          % (nrows, v.m, max(args.cpu_rows_stride, 1), it, len(dts), dt)}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
