"""Benchmark of one DBaS-Log-MPPI step (arXiv 2504.06437) on GB300.

Metric: sample-timesteps per second of one MPPI iteration (K samples x T
steps / step time), with p50/p99 step latency, batched vs plain.  The
default line is the large single-controller workload (kinematic unicycle,
K=65536, T=100, 200 obstacles in a 50 x 50 m field), and it carries, under
"batched", the batched-vs-plain comparison on the 512-controller mix (one
persistent launch against one launch per controller).

* value: device-resident inputs, one step = one kernel launch
  (mppi_step_device); each step timed with CUDA events on the launching
  stream; L2 flushed (256 MB write) between steps, outside the timed events.
* e2e: the public host API (mppi_step with host x0/xref + mppi_get_control),
  host<->device copies inside the timed region, wall clock per step.
* roofline: the step kernel against the FP32 issue rate of the GPU.
* cpu_baseline: the CPU FP64 oracle on a bounded sample of the same workload.

``--impl reference`` times the CPU oracle alone on the same workload.
Multi-GPU (torchrun): every rank runs its own controller (replicas only,
weak scaling); value = all ranks' sample-steps / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "sample-timesteps/sec per MPPI step"
UNIT = "sample-steps/s"
# FP32-pipe operations per obstacle-point pair: 2 subtractions and 2 fmas for
# h, the reciprocal, the add into the sum and the min of the collision test
# (7); the h_eps floor's max, an eighth, is reported beside it
OPS_PER_PAIR = 7
OPS_PER_PAIR_WITH_FLOOR = 8
OPS_PER_SAMPLE_STEP = 135  # Philox (~80), NLN map (~20), dynamics + costs (~35)
L2_FLUSH_BYTES = 256 << 20


# grid-map lookup per shape point: grid coordinates (2 subtractions, 2
# products), 4 clamps, 2 conversions and 2 integer minima, 2 fractions, 3
# lerps (2 subtractions, 3 fmas), then max, reciprocal, add and min
OPS_PER_GRID_POINT = 24


def algorithmic_ops(K, T, P, J, grid=False, per_pair=OPS_PER_PAIR):
    return K * T * (per_pair * P * J + (OPS_PER_GRID_POINT * P if grid else 0)
                    + OPS_PER_SAMPLE_STEP)


def io_bytes_per_launch(K, T, n, J):
    """Bytes one step must move at least: x0, the reference, U and the
    obstacles in; the shifted U, U*, the per-sample costs (FP64) and
    collided flags out."""
    return 8 * (n + (T + 1) * n) + 8 * 2 * T + 24 * J + 2 * 8 * 2 * T + 9 * K


def kernel_src_sha():
    """Hash of the device code of the step and batch kernels (the kernel
    translation units k_*.cu and the device headers), not of the host
    runtime: the key of the committed traffic counters."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2504_06437_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        if f.endswith(".cuh") or (f.startswith("k_") and f.endswith(".cu")):
            h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the
    architecture) and its logical CPU count."""
    name = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=5).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                name = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not name:
        try:
            for ln in open("/proc/cpuinfo"):
                if ln.lower().startswith("model name"):
                    name = ln.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    return {"model": name or platform.machine(), "logical_cpus": os.cpu_count()}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def traffic_per_launch(workload):
    """dram bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source; else None."""
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "step_kernel_traffic.json")))
    except Exception:
        return None
    r = rec.get(workload)
    if not r or r.get("kernel_src_sha") != kernel_src_sha():
        return None
    return r.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None):
        self.proc = None
        self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "50"]
        if uuid:
            cmd += ["-i", uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=self.tmp, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.tmp.flush()
        rows = []
        for line in open(self.tmp.name):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.tmp.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def oracle_rate(world, n_samples, min_seconds, max_steps=None, threads=None):
    """Time the CPU oracle's full step on the first n_samples samples of the
    workload; returns (sample-steps/s, steps, seconds, threads)."""
    import oracle
    oracle.build()
    if threads:
        oracle.set_threads(threads)
    p = dict(world.params)
    p["K"] = n_samples
    ctl = oracle.new_controller(p)
    x = world.x_start
    xref = world.reference(x)
    oracle.step(p, world.obstacles, x, xref, ctl, want_sens=False)  # warm
    steps, t0 = 0, time.perf_counter()
    while True:
        oracle.step(p, world.obstacles, x, xref, ctl, want_sens=False)
        steps += 1
        el = time.perf_counter() - t0
        if (max_steps and steps >= max_steps) or (not max_steps and el >= min_seconds and steps >= 3):
            break
    return n_samples * p["T"] * steps / el, steps, el, oracle.get_threads()


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if os.environ.get("BENCH_BACKEND") != "gloo" else "gloo")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(ws, v):
    """Maximum of v over the ranks (the slowest rank's time)."""
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cpu" if dist.get_backend() == "gloo" else "cuda"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(ws, units_per_rank, ms_max):
    """Units per second of the whole job: every rank processes units_per_rank
    units per step and the step lasts as long as the slowest rank (ms_max)."""
    return ws * units_per_rank / (ms_max / 1e3)


def world_for(workload, seed, sgf=""):
    """The named workload; sgf "W,P" turns on Savitzky-Golay smoothing of the
    update (window W, order P) in its parameters."""
    import dataclasses
    from paper_2504_06437_gb300 import workloads as W
    world = W.PRESETS[workload](seed)
    if sgf:
        w_, p_ = (int(v) for v in sgf.split(","))
        world = dataclasses.replace(world, params=dict(world.params, sgf_window=w_, sgf_order=p_))
    return world


def describe(world):
    p = world.params
    P = int(np.asarray(p["shape"]).reshape(-1, 2).shape[0])
    return {"workload": world.name, "K": int(p["K"]), "T": int(p["T"]),
            "obstacles": int(world.obstacles.shape[0]), "shape_points": P,
            "model": {0: "unicycle", 1: "planar quadrotor (6 states)", 2: "Ackermann vehicle",
                      3: "planar quadrotor (5 states, the paper's)"}[int(p["model"])],
            "l2": "flushed between timed steps (256 MB write)",
            **({"sgf": {"window": int(p["sgf_window"]), "order": int(p["sgf_order"])}}
               if int(p.get("sgf_window", 0)) > 0 else {}),
            **({"grid_map": {"nx": int(p["grid"].shape[1]), "ny": int(p["grid"].shape[0]),
                             "res_m": float(p["grid_res"])}}
               if p.get("grid") is not None else {})}


def run_reference_mix(args):
    """The oracle on the batched or served mix: one reference step is one
    oracle step of each of the first controllers of the mix, each on a
    bounded sample of its K samples (the mix is far too large for a CPU
    step of every controller)."""
    from paper_2504_06437_gb300 import workloads as W
    import oracle
    serving = args.workload == "serving"
    worlds = (W.serving_mix(args.robots, seed=0) if serving else W.batch_mix(args.batch_n, seed=0))
    worlds = worlds[:8]
    oracle.build()
    oracle.set_threads(os.cpu_count() or 1)
    jobs = []
    for w in worlds:
        pp = dict(w.params)
        pp["K"] = min(int(pp["K"]), args.ref_samples)
        jobs.append((w, pp, oracle.new_controller(pp), w.reference(w.x_start)))
    def one():
        for w, pp, ctl, xr in jobs:
            oracle.step(pp, w.obstacles, w.x_start, xr, ctl, want_sens=False)
    for _ in range(max(args.warmup, 3)):
        one()
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        one()
        times.append(time.perf_counter() - t0)
    ms = 1e3 * float(np.mean(times))
    work = sum(int(pp["K"]) * int(pp["T"]) for _, pp, _, _ in jobs)
    value = work / (ms / 1e3)
    sample = (f"oracle step of the first {len(jobs)} controllers of the mix, "
              f"{args.ref_samples} samples each at most, {args.steps} steps")
    line = {"impl": "reference",
            "metric": METRIC + (" and p50/p99 step latency (serving)" if serving else " (batched)"),
            "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": ("serving_mix" if serving else "batch_mix")
                       + f": the first {len(jobs)} controllers"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.get_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_reference(args, ws, rank):
    if rank != 0:
        return
    if args.workload in ("batch_mix", "serving"):
        run_reference_mix(args)
        return
    world = world_for(args.workload, 0, args.sgf)
    p = world.params
    n_samples = min(int(p["K"]), args.ref_samples)
    threads = os.cpu_count() or 1
    import oracle
    oracle.build()
    oracle.set_threads(threads)
    pp = dict(p)
    pp["K"] = n_samples
    ctl = oracle.new_controller(pp)
    x = world.x_start
    xref = world.reference(x)
    # at least 10 untimed steps: the oracle's first steps run well below its
    # steady rate (thread start-up, first touch of its buffers)
    for _ in range(max(args.warmup, 10)):
        oracle.step(pp, world.obstacles, x, xref, ctl, want_sens=False)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.step(pp, world.obstacles, x, xref, ctl, want_sens=False)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * float(np.mean(times))
    value = n_samples * pp["T"] / (ms / 1e3)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": describe(world),
            "latency_ms": {"p50": 1e3 * float(np.percentile(times, 50)),
                           "p99": 1e3 * float(np.percentile(times, 99))},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.get_threads(),
                             "kind": "oracle",
                             "sample": f"full oracle step on {n_samples} of {p['K']} samples, "
                                       f"{args.steps} steps"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def measure_batch(args, ws, rank, local):
    """Batched workload: many controllers of mixed model, K, T and obstacle
    count stepped by one persistent launch (CUDA graph replay), against the
    same controllers stepped one launch each, back to back on one stream,
    and against the host loop that steps each and reads its control back.
    Returns the measurements (every rank), or None on ranks other than 0."""
    import torch
    from paper_2504_06437_gb300 import binding, workloads as W

    torch.cuda.set_device(local)
    binding.load()
    worlds = W.batch_mix(args.batch_n, seed=rank)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    policy, tune_ms = None, None
    if not args.no_autotune:
        policy, tune_ms = binding.batch_autotune([w.params for w in worlds],
                                                 [w.obstacles for w in worlds], iters=3,
                                                 pool_bytes=6 << 30)
    b = binding.Batch(len(worlds), 6 << 30)
    if policy:
        b.set_policy(policy)
    used_policy = b.get_policy()
    slots = [b.add(w.params, w.obstacles) for w in worlds]
    x0s = [w.x_start for w in worlds]
    xrefs = [w.reference(w.x_start) for w in worlds]
    work = sum(int(w.params["K"]) * int(w.params["T"]) for w in worlds)
    for _ in range(args.warmup):
        b.step(slots, x0s, xrefs, stream)
        b.controls()
    steps = args.batch_steps
    sampler = ClockSampler()
    e0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    e1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    wall = []
    barrier(ws)
    torch.cuda.synchronize()
    for i in range(steps):
        flush.fill_(float(i & 7))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e0[i].record(stream)
        b.step(slots, x0s, xrefs, stream)
        e1[i].record(stream)
        b.controls()
        wall.append(time.perf_counter() - t0)
    torch.cuda.synchronize()
    barrier(ws)
    clocks = sampler.stop()
    dev_ms = np.array([a.elapsed_time(c) for a, c in zip(e0, e1)])
    ms = allmax(ws, float(dev_ms.mean()))
    e2e_ms = allmax(ws, 1e3 * float(np.mean(wall)))
    # the same controllers, one launch each, back to back
    plain = []
    for w, sl in zip(worlds, slots):
        info = b.slot_info(sl)
        g = binding.Controller(w.params, tiling=dict(samples_per_cta=info["samples_per_cta"],
                                                     threads=256,
                                                     positions_per_thread=info["positions_per_thread"]))
        g.set_obstacles(w.obstacles)
        xr = w.reference(w.x_start)
        d_in = torch.tensor(np.concatenate([w.x_start, xr.ravel()]), dtype=torch.float64, device="cuda")
        plain.append((g, d_in, w.n))
    for g, d_in, n in plain:
        g.step_device(d_in.data_ptr(), d_in.data_ptr() + 8 * n, stream)
    torch.cuda.synchronize()
    p_ms = []
    psampler = ClockSampler()
    for i in range(max(3, steps // 10)):
        flush.fill_(1.0)
        a = torch.cuda.Event(enable_timing=True)
        c = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for g, d_in, n in plain:
            g.step_device(d_in.data_ptr(), d_in.data_ptr() + 8 * n, stream)
        c.record(stream)
        torch.cuda.synchronize()
        p_ms.append(a.elapsed_time(c))
    pclocks = psampler.stop()
    plain_ms = allmax(ws, float(np.mean(p_ms)))
    # and the naive host loop: each controller stepped from host data and its
    # control read back before the next (mppi_step + mppi_get_control)
    xr_host = [w.reference(w.x_start) for w in worlds]
    flush.fill_(1.0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for (g, _, _), w, xr in zip(plain, worlds, xr_host):
        g.step(w.x_start, xr, stream)
        g.get_control()
    synced_ms = allmax(ws, 1e3 * (time.perf_counter() - t0))
    for g, _, _ in plain:
        g.close()
    b.close()
    if rank != 0:
        return None
    # the same FP32 issue roofline as the one-controller step, over the sum
    # of the controllers' algorithmic work (the batch kernel is the only
    # kernel in the timed region)
    def ops(per_pair):
        return sum(algorithmic_ops(int(w.params["K"]), int(w.params["T"]),
                                   int(np.asarray(w.params["shape"]).reshape(-1, 2).shape[0]),
                                   int(w.obstacles.shape[0]), per_pair=per_pair) for w in worlds)
    peaks = measured_peaks()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    f_max = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    peak_tops = sms * 128 * f_max / 1e12
    achieved_tops = ops(OPS_PER_PAIR) / (ms / 1e3) / 1e12
    roofline = {"bound": "alu", "achieved": achieved_tops, "peak": peak_tops, "unit": "TOP/s",
                "frac": achieved_tops / peak_tops, "traffic": traffic_per_launch("batch_mix"),
                "kernel": "batch_kernel",
                "peak_basis": f"{sms} SMs x 128 FP32 lanes x {f_max/1e6:.0f} MHz (of measured max clock)",
                "ops_per_launch": ops(OPS_PER_PAIR),
                "ops_count": f"{OPS_PER_PAIR} per obstacle-point pair + {OPS_PER_SAMPLE_STEP} per sample-step",
                "frac_with_floor_op": ops(OPS_PER_PAIR_WITH_FLOOR) / (ms / 1e3) / 1e12 / peak_tops}
    return {"value": whole_job_value(ws, work, ms), "unit": UNIT, "ms_per_step": ms,
            "steps": steps, "warmup": args.warmup,
            "workload": f"batch_mix: {len(worlds)} controllers, half unicycle half planar "
                        "quadrotor, K log-uniform 1024..16384, T 20..80, 5..300 obstacles",
            "sample_steps_per_step": work, "l2": "flushed between timed steps (256 MB write)",
            "graph": "CUDA graph replay of copy-in, persistent kernel, copy-out",
            "tiling_policy": used_policy,
            "tiling_source": "autotuned (mppi_batch_autotune)" if policy else "default",
            "latency_ms": {"p50": float(np.percentile(dev_ms, 50)),
                           "p99": float(np.percentile(dev_ms, 99))},
            "plain": {"value": whole_job_value(ws, work, plain_ms), "unit": UNIT,
                      "ms_per_step": plain_ms, "steps": len(p_ms),
                      "form": "one launch per controller, back to back on one stream",
                      "clocks": pclocks},
            "plain_synced": {"value": whole_job_value(ws, work, synced_ms), "unit": UNIT,
                             "ms_per_step": synced_ms,
                             "form": "host loop: mppi_step + mppi_get_control per controller"},
            "batched_over_plain": plain_ms / ms,
            "batched_over_plain_synced": synced_ms / ms,
            "e2e": {"value": whole_job_value(ws, work, e2e_ms), "unit": UNIT, "ms_per_step": e2e_ms,
                    "h2d_bytes_per_step": int(sum(8 * w.n * (w.params["T"] + 2) for w in worlds)),
                    "d2h_bytes_per_step": 16 * len(worlds),
                    "latency_ms": {"p50": 1e3 * float(np.percentile(wall, 50)),
                                   "p99": 1e3 * float(np.percentile(wall, 99))}},
            "roofline": roofline, "gpu_launches": steps, "clocks": clocks}


def run_batch(args, ws, rank, local):
    """The batched workload as its own line (--workload batch_mix)."""
    m = measure_batch(args, ws, rank, local)
    if m is None:
        return
    line = {"metric": METRIC + " (batched)", "value": m["value"], "unit": UNIT,
            "n_gpus": ws, "steps": m["steps"], "warmup": args.warmup, "ms_per_step": m["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {k: m[k] for k in ("workload", "sample_steps_per_step", "l2", "graph",
                                         "tiling_policy", "tiling_source")},
            **{k: m[k] for k in ("latency_ms", "plain", "plain_synced", "batched_over_plain",
                                 "batched_over_plain_synced", "e2e", "roofline", "gpu_launches",
                                 "clocks")}}
    print(json.dumps(line), flush=True)


def _serving_buckets(rows, pct):
    """p50/p99 of latency, queueing and device time per request-size bucket
    (decades of K T (7 P J + 135) FP32 operations) and per size class."""
    edges = [0.0, 1e8, 1e9, 1e10, 1e11, float("inf")]
    names = ["<1e8", "1e8..1e9", "1e9..1e10", "1e10..1e11", ">=1e11"]
    out = {}
    def summ(sel):
        lat = np.array([r["latency"] for r in sel])
        q = np.array([r["queue"] for r in sel])
        d = np.array([r["device"] for r in sel])
        return {"requests": len(sel), "latency_ms": {"p50": pct(lat, 50), "p99": pct(lat, 99)},
                "queue_ms": {"p50": pct(q, 50), "p99": pct(q, 99)},
                "device_ms": {"p50": pct(d, 50), "p99": pct(d, 99)},
                "p99_within_2ms": bool(pct(lat, 99) <= 2.0)}
    for lo, hi, nm in zip(edges[:-1], edges[1:], names):
        sel = [r for r in rows if lo <= r["ops"] < hi]
        if sel:
            out[nm] = summ(sel)
    by_cls = {}
    for c, nm in ((0, "small"), (1, "large")):
        sel = [r for r in rows if r["size_class"] == c]
        if sel:
            by_cls[nm] = summ(sel)
    return out, by_cls


def run_serving(args, ws, rank, local):
    """Serving workload: robots of mixed model, K, T and obstacle count send
    closed-loop control-step requests to the continuous-batching runtime
    (by default its device queue: one resident kernel that takes requests
    as they arrive, small ones first).
    First the capacity is measured with every robot resubmitting at once
    (saturation), then requests arrive with exponential think times sized to
    a fraction of that capacity; latency is submission to completion, split
    into time queued and the device time of the request's batch, and
    reported per request-size bucket.  The plain form serves the same
    requests one at a time through the context API (mppi_step +
    mppi_get_control)."""
    import heapq

    import torch
    from paper_2504_06437_gb300 import binding, workloads as W

    torch.cuda.set_device(local)
    binding.load()
    worlds = W.serving_mix(args.robots, seed=rank)
    g = np.random.default_rng(rank)
    srv = binding.Server(len(worlds), args.pool_mb << 20, lanes=args.lanes)
    if args.batch_ops_small is None:
        args.batch_ops_small = 0.0 if args.device_queue else 4e9
    if args.small_ops > 0 or args.device_queue:
        srv.set_policy(small_ops_max=args.small_ops, small_lanes=args.small_lanes,
                       large_share=args.large_share, batch_ops_small=args.batch_ops_small,
                       batch_ops_large=args.batch_ops_large, shortest_first=args.shortest_first,
                       max_wait_s=args.max_wait_ms * 1e-3, device_queue=bool(args.device_queue))
    policy = srv.get_policy()

    def ops_of(w):
        p = w.params
        P = int(np.asarray(p["shape"]).reshape(-1, 2).shape[0])
        return float(p["K"]) * p["T"] * (7.0 * P * w.obstacles.shape[0] + 135.0)

    def run(n_req_per_robot, think_mean):
        waiting = list(range(len(worlds)))   # admission queue (memory)
        active, x, done, rows = {}, {}, {}, []
        timers = []
        t_start = time.perf_counter()
        completed = 0
        total_work = 0
        while waiting or active:
            while waiting:
                i = waiting[0]
                r = srv.join(worlds[i].params, worlds[i].obstacles)
                if r is None:
                    break
                waiting.pop(0)
                active[r] = i
                x[r] = worlds[i].x_start.copy()
                done[r] = 0
                heapq.heappush(timers, (time.perf_counter() + g.exponential(think_mean) if think_mean else 0.0, r))
            now = time.perf_counter()
            while timers and timers[0][0] <= now:
                _, r = heapq.heappop(timers)
                w = worlds[active[r]]
                srv.submit(r, x[r], w.reference(x[r]))
            for d in srv.poll_timed():
                r = d["robot"]
                w = worlds[active[r]]
                rows.append(dict(latency=d["latency"], queue=d["queue"], device=d["device"],
                                 size_class=d["size_class"], ops=ops_of(w)))
                completed += 1
                total_work += int(w.params["K"]) * int(w.params["T"])
                done[r] += 1
                x[r] = d["x1"][: w.n].copy()
                if done[r] >= n_req_per_robot:
                    srv.leave(r)
                    del active[r]
                else:
                    heapq.heappush(timers, (time.perf_counter() + (g.exponential(think_mean) if think_mean else 0.0), r))
        el = time.perf_counter() - t_start
        return dict(seconds=el, requests=completed, work=total_work, rows=rows,
                    lat=np.array([r["latency"] for r in rows]))

    run(1, 0.0)  # warm-up
    st0 = srv.stats()
    cap = run(args.serve_steps, 0.0)
    st1 = srv.stats()
    cap_rps = cap["requests"] / cap["seconds"]
    think = len(worlds) / (args.load * cap_rps)
    sampler = ClockSampler()
    loaded = run(args.serve_steps, think)
    clocks = sampler.stop()
    st2 = srv.stats()
    srv.close()
    # plain: the same kind of requests served one at a time
    plain_lat, plain_work = [], 0
    n_plain = min(len(worlds), args.plain_robots)
    for w in worlds[:n_plain]:
        with binding.Controller(w.params) as c:
            c.set_obstacles(w.obstacles)
            xx = w.x_start
            for _ in range(args.plain_steps):
                a = time.perf_counter()
                c.step(xx, w.reference(xx))
                c.get_control()
                plain_lat.append(time.perf_counter() - a)
                plain_work += int(w.params["K"]) * int(w.params["T"])
    plain_s = float(np.sum(plain_lat))
    if rank != 0:
        return
    pct = lambda a, q: 1e3 * float(np.percentile(a, q)) if len(a) else None
    buckets, classes = _serving_buckets(loaded["rows"], pct)
    line = {"metric": METRIC + " and p50/p99 step latency (serving)",
            "value": loaded["work"] / loaded["seconds"], "unit": UNIT, "n_gpus": ws,
            "steps": loaded["requests"], "warmup": len(worlds),
            "ms_per_step": 1e3 * loaded["seconds"] / max(1, loaded["requests"]),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"serving_mix: {len(worlds)} robots, half unicycle half planar quadrotor, "
                                   "K log-uniform 512..32768, T 20..100, 5..500 obstacles",
                       "requests_per_robot": args.serve_steps, "lanes": args.lanes,
                       "policy": policy,
                       "pool_mb": args.pool_mb, "offered_load": f"{args.load:.2f} of measured capacity",
                       "arrivals": "closed loop, exponential think time after each reply"},
            "latency_ms": {"p50": pct(loaded["lat"], 50), "p99": pct(loaded["lat"], 99)},
            "latency_by_request_ops": buckets,
            "latency_by_size_class": classes,
            "capacity": {"value": cap["work"] / cap["seconds"], "unit": UNIT,
                         "requests_per_s": cap_rps,
                         "latency_ms": {"p50": pct(cap["lat"], 50), "p99": pct(cap["lat"], 99)},
                         "mean_batch": (st1["requests"] - st0["requests"]) / max(1, st1["batches"] - st0["batches"])},
            "loaded": {"requests_per_s": loaded["requests"] / loaded["seconds"],
                       "mean_batch": (st2["requests"] - st1["requests"]) / max(1, st2["batches"] - st1["batches"])},
            "plain": {"value": plain_work / plain_s, "unit": UNIT,
                      "form": "one request at a time: mppi_step + mppi_get_control",
                      "requests": len(plain_lat),
                      "latency_ms": {"p50": pct(plain_lat, 50), "p99": pct(plain_lat, 99)}},
            "serving_over_plain": (cap["work"] / cap["seconds"]) / (plain_work / plain_s),
            "gpu_launches": int(st2["batches"] - st1["batches"]),
            "clocks": clocks}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="unicycle_stress")
    ap.add_argument("--batch-steps", type=int, default=20,
                    help="timed steps of the batched comparison")
    ap.add_argument("--no-batch", action="store_true",
                    help="leave the batched-vs-plain comparison out of the default line")
    ap.add_argument("--e2e-steps", type=int, default=500)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--ref-samples", type=int, default=256)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch-n", type=int, default=512)
    ap.add_argument("--robots", type=int, default=1000)
    ap.add_argument("--serve-steps", type=int, default=10)
    ap.add_argument("--lanes", type=int, default=4)
    ap.add_argument("--small-ops", type=float, default=2e9,
                    help="serving: requests of at most this many FP32 operations are small (0: one class)")
    ap.add_argument("--small-lanes", type=int, default=3)
    ap.add_argument("--large-share", type=float, default=0.75)
    ap.add_argument("--batch-ops-small", type=float, default=None,
                    help="lanes: work cap of a small batch (default 4e9); device queue: cap on "
                         "published small work (default 0, none)")
    ap.add_argument("--batch-ops-large", type=float, default=5e10)
    ap.add_argument("--shortest-first", type=int, default=1)
    ap.add_argument("--max-wait-ms", type=float, default=50.0)
    ap.add_argument("--device-queue", type=int, default=1,
                    help="serving: one resident kernel takes requests as they arrive (1) or lanes of batches (0)")
    ap.add_argument("--pool-mb", type=int, default=2048)
    ap.add_argument("--load", type=float, default=0.5)
    ap.add_argument("--plain-robots", type=int, default=100)
    ap.add_argument("--plain-steps", type=int, default=3)
    ap.add_argument("--sgf", default="",
                    help="W,P: Savitzky-Golay smoothing of the update, window W, order P")
    ap.add_argument("--tiling", default="",
                    help="explicit launch shape S,threads,points (skips the autotuner)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="use the library's default launch shape instead of the autotuned one")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.workload == "batch_mix":
        args.batch_steps = args.steps
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    if args.workload == "batch_mix":
        run_batch(args, ws, rank, local)
        return
    if args.workload == "serving":
        run_serving(args, ws, rank, local)
        return

    import torch
    from paper_2504_06437_gb300 import binding

    torch.cuda.set_device(local)
    binding.load()
    world = world_for(args.workload, rank, args.sgf)
    p = world.params
    K, T, n = int(p["K"]), int(p["T"]), world.n
    P = int(np.asarray(p["shape"]).reshape(-1, 2).shape[0])
    J = int(world.obstacles.shape[0])
    tiling, tune_us = None, None
    if args.tiling:
        S_, NT_, NP_ = (int(v) for v in args.tiling.split(","))
        tiling = dict(samples_per_cta=S_, threads=NT_, positions_per_thread=NP_)
    elif not args.no_autotune:
        # tuned the way it is timed below: each step alone after the L2 flush
        tiling, tune_us = binding.autotune(p, world.obstacles, iters=10, flush_bytes=L2_FLUSH_BYTES)
    ctl = binding.Controller(p, tiling=tiling)
    ctl.set_obstacles(world.obstacles)
    has_grid = p.get("grid") is not None
    if has_grid:
        ctl.set_grid(p["grid"], p["grid_ox"], p["grid_oy"], p["grid_res"])
    x0 = world.x_start
    xref = world.reference(x0)
    d_in = torch.tensor(np.concatenate([x0, xref.ravel()]), dtype=torch.float64, device="cuda")
    d_x0 = d_in.data_ptr()
    d_xref = d_x0 + 8 * n
    # a dedicated stream: the library launches on it, the events and the L2
    # flush are recorded on it (torch's default stream would be handle 0,
    # which the C ABI reads as "the context's own stream")
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    for _ in range(args.warmup):
        flush.fill_(1.0)
        ctl.step_device(d_x0, d_xref, stream)
    torch.cuda.synchronize()
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        uuid = None
    sampler = ClockSampler(uuid)
    time.sleep(0.2)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier(ws)
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.fill_(float(i & 7))
        starts[i].record(stream)
        ctl.step_device(d_x0, d_xref, stream)
        ends[i].record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    clocks = sampler.stop()
    times_ms = np.array([s.elapsed_time(e) for s, e in zip(starts, ends)])
    ms_local = float(times_ms.mean())
    ms = allmax(ws, ms_local)
    value = whole_job_value(ws, K * T, ms)

    # end to end through the host API (pinned staging inside the library)
    u0 = ctl.get_control()
    for _ in range(max(3, args.warmup)):  # untimed: the host path's own warm-up
        ctl.step(x0, xref, stream)
        u0 = ctl.get_control()
    e2e_t = []
    for i in range(args.e2e_steps):
        flush.fill_(float(i & 7))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctl.step(x0, xref, stream)
        u0 = ctl.get_control()
        e2e_t.append(time.perf_counter() - t0)
    e2e_ms = allmax(ws, 1e3 * float(np.mean(e2e_t)))
    h2d, d2h = ctl.io_bytes()
    tiling = ctl.tiling()

    peaks = measured_peaks()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    f_max = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    peak_tops = sms * 128 * f_max / 1e12
    ops_launch = algorithmic_ops(K, T, P, J, has_grid)
    achieved_tops = ops_launch / (ms_local / 1e3) / 1e12
    roofline = {"bound": "alu", "achieved": achieved_tops, "peak": peak_tops, "unit": "TOP/s",
                "frac": achieved_tops / peak_tops, "traffic": traffic_per_launch(world.name),
                "kernel": "step_kernel",
                "peak_basis": f"{sms} SMs x 128 FP32 lanes x {f_max/1e6:.0f} MHz (of measured max clock)",
                "ops_per_launch": ops_launch,
                "ops_count": f"{OPS_PER_PAIR} per obstacle-point pair + {OPS_PER_SAMPLE_STEP} per sample-step",
                "frac_with_floor_op": algorithmic_ops(K, T, P, J, has_grid, OPS_PER_PAIR_WITH_FLOOR)
                / (ms_local / 1e3) / 1e12 / peak_tops,
                "algorithmic_bytes_per_launch": io_bytes_per_launch(K, T, n, J)}
    if clocks.get("sm_mhz"):
        roofline["frac_at_median_clock"] = achieved_tops / (sms * 128 * clocks["sm_mhz"] * 1e6 / 1e12)
    batched = None
    if args.workload == "unicycle_stress" and not args.no_batch:
        # the other half of the metric, batched vs plain, in the same line
        # (every rank takes part: the measurement has barriers)
        ctl.close()
        del d_in, flush
        torch.cuda.empty_cache()
        batched = measure_batch(args, ws, rank, local)

    if rank != 0:
        return
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(describe(world), parallelism=f"replicas x{ws}", tiling=tiling,
                           tiling_source="autotuned" if tune_us else ("explicit" if args.tiling else "default")),
            "latency_ms": {"p50": float(np.percentile(times_ms, 50)),
                           "p99": float(np.percentile(times_ms, 99))},
            "e2e": {"value": whole_job_value(ws, K * T, e2e_ms), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
                    "latency_ms": {"p50": 1e3 * float(np.percentile(e2e_t, 50)),
                                   "p99": 1e3 * float(np.percentile(e2e_t, 99))}},
            "gpu_launches": args.steps, "clocks": clocks, "roofline": roofline}
    if batched is not None:
        line["batched"] = batched
    if not args.no_cpu_baseline and ws == 1:
        threads = os.cpu_count() or 1
        rate, steps, el, used = oracle_rate(world, min(K, args.ref_samples), args.cpu_seconds,
                                            threads=threads)
        rate1, steps1, el1, _ = oracle_rate(world, min(K, args.ref_samples), args.cpu_seconds / 3,
                                            threads=1)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": used, "kind": "oracle",
                                "sample": f"full oracle step on {min(K, args.ref_samples)} of {K} "
                                          f"samples (T={T}, J={J}, P={P}), {steps} steps in {el:.1f} s",
                                "single_thread": {"value": rate1, "unit": UNIT,
                                                  "sample": f"{steps1} steps in {el1:.1f} s"},
                                "cpu": cpu_model()}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
