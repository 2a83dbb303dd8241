"""Benchmark of the correlator X-engine on one GB300 (or N replicas).

One step = one whole integration through the public C ABI: xeng_push of the
block [T][F][N] (decode + tensor-core correlation + packed triangle) and
xeng_dump of the int32 triangle to a caller buffer.  Inputs are synthetic,
generated on the device from a seed (shape and statistics of the workload
named by --workload) and larger than L2, so no flush is needed between steps.

Prints one JSON line (rank 0).  Metric: useful correlation TOPS, 8 real
operations per complex multiply-accumulate, N(N+1)/2 baselines per channel.
`--impl reference` times the CPU oracle on a bounded sample instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (recipe attribute in synth, description)
    "chime_full": ("CHIME_FULL", "full-CHIME-shaped: N=2048 inputs, 1024 channels, T=8192, sky+noise (rho 0.1, sigma 2.5)"),
    "pathfinder_full": ("PATHFINDER_FULL", "full Pathfinder rate: N=256, 1024 channels, T=32768, sky+noise (rho 0.1, sigma 2.5)"),
    "pathfinder_small": ("PATHFINDER_SMALL", "Pathfinder-shaped small: N=256, 8 channels, T=4096, uniform nibbles"),
    "chime_slice": ("CHIME_SLICE", "16 channels of the full-CHIME shape (N=2048, T=8192): profiling case"),
    "pathfinder_slice": ("PATHFINDER_SLICE", "64 channels of the Pathfinder shape (N=256, T=32768): profiling case"),
    "mid_slice": ("MID_SLICE", "128 channels of N=640, T=8192, sky+noise: profiling case of the one pass over 128-input "
                               "block pairs"),
    "batched": (None, "64 independent jobs, N in {64..2048}, F in {1,16,64}, T log-uniform 1024..32768, uniform nibbles"),
    "serving": (None, "8 concurrent streams (3 x N=256, 3 x N=512, 2 x N=2048), 256 channels each, 256-sample blocks, "
                      "Poisson arrivals at r x real time, dumps every 65536 samples"),
}
METRIC = "Correlation TOPS (8 ops per complex MAC, bit-exact int32 visibilities)"

# DRAM bytes (read + write) per channel of one launch of a correlation kernel,
# from one ncu capture of the 16-channel slice of the same (N, T) shape
# (dram__bytes_read.sum + dram__bytes_write.sum); traffic grows in proportion to
# channels.  Keyed by (kernel, N, T); re-take (or remove) an entry whenever its
# kernel changes.
DRAM_BYTES_PER_CHANNEL = {
    ("correlate_pair", 2048, 8192): (300.792576e6 + 217.08416e6) / 16,  # 256-input block pairs, 16-channel slice
    ("correlate_tc", 2048, 8192): (607.22048e6 + 240.377344e6) / 16,   # planes engine, 16-channel slice
    ("correlate_small", 256, 32768): (821.3591e6 + 19.01209e6) / 64,  # N <= 256 kernel, 64-channel slice
    ("correlate_onepass", 640, 8192): (676.018944e6 + 184.502016e6) / 128,  # one pass, 128-channel slice
}


# The library's choice between its two single-pass kernels above 256 inputs, at
# its default build parameters: measured cost of one block pair (tens of us per
# 1024 channels x 8192 samples) times the upper-triangle block pairs.
PAIR_COST, ONEPASS_COST, FUSED_MAX_N = 118, 36, 3584


def use_pair_kernel(N):
    b2, b1 = -(-N // 256), -(-N // 128)
    return PAIR_COST * (b2 * (b2 + 1) // 2) < ONEPASS_COST * (b1 * (b1 + 1) // 2)


def correlate_kernel(engine, N):
    """(name, tile) of the correlation kernel an engine runs for N inputs (tile:
    the square of inputs one work item computes, lower halves of diagonal
    items included)."""
    fused = N % 16 == 0 and (engine == "fused" or (engine == "tensor" and N <= FUSED_MAX_N))
    if fused and N <= 256:
        return "correlate_small_kernel (decode fused; upper-triangle 128-input blocks, one CTA each)", 128
    if fused and use_pair_kernel(N):
        return "correlate_pair_kernel (decode fused; 256-input block pairs, 2-CTA clusters)", 256
    if fused:
        return "correlate_onepass_kernel (decode fused; 128-input block pairs, one CTA each)", 128
    return "correlate_tc_kernel (decoded planes; 128-input tile pairs)", 128


def max_over_ranks(x, dist=None):
    """Largest value of x over all ranks (x itself without a process group).
    Works on the gloo (CPU tensors) and nccl (CUDA tensors) backends."""
    if dist is None or not dist.is_initialized():
        return float(x)
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, seconds_max, world):
    """Throughput of the whole job: every rank processed units_per_rank in at most seconds_max."""
    return units_per_rank * world / seconds_max


def useful_ops(T, F, N):
    return 8.0 * T * F * N * (N + 1) / 2


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu_index = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu_index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.proc or not self.path or not os.path.exists(self.path):
            return None
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]) if parts[3] not in ("[N/A]", "") else 0.0,
                             parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k, v in enumerate(r[3]) if v.lower() == "active"})
        loaded = [r for r in rows if r[2] > 200.0] or rows
        return {"sm_mhz": statistics.median(r[0] for r in loaded), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows), "samples_under_load": len(loaded),
                "power_w_max": max(r[2] for r in rows)}


def gpu_index_for(local_rank):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    ids = [v for v in vis.split(",") if v.strip()]
    if ids and all(v.strip().isdigit() for v in ids) and local_rank < len(ids):
        return int(ids[local_rank])
    return local_rank


def cpu_oracle_sample(rec, T, F, N, out_dev=None):
    """Time the oracle (as it stands) on a bounded sample; check the GPU output on it."""
    import numpy as np
    import oracle
    # about 10 s of oracle work on 16 cores: 8 channels at N = 2048 (T = 8192),
    # 128 at N = 256 (T = 32768)
    nf = {2048: 8, 256: 128}.get(N, 8)
    nf = min(nf, F)
    host = rec.host(f0=0, nf=nf)
    t0 = time.perf_counter()
    want = oracle.correlate(host)
    dt = time.perf_counter() - t0
    ops = useful_ops(T, nf, N)
    exact = None
    if out_dev is not None:
        got = out_dev[:nf].cpu().numpy().astype(np.int64)
        exact = bool(np.array_equal(got, want))
    return {"value": ops / dt / 1e12, "unit": "TOPS", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": "channels 0..%d of the workload (all %d inputs, all %d samples), int64 oracle, %.1f s"
                      % (nf - 1, N, T, dt)}, exact


def run_reference(args, rank, world):
    """The oracle as the reference arm: each step correlates a bounded sample."""
    import synth
    import oracle
    rec = getattr(synth, WORKLOADS[args.workload][0])
    T, F, N = rec.T, rec.F, rec.N
    if rank != 0:
        return
    # sample: channel 0, all inputs, the first Ts samples (about a second or two per step)
    Ts = {2048: 512, 256: 8192}.get(N, T)
    Ts = min(Ts, T)
    host = rec.host(f0=0, nf=1, t0=0, nt=Ts)
    for _ in range(args.warmup):
        oracle.correlate(host)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.correlate(host)
    dt = (time.perf_counter() - t0) / args.steps
    ops = useful_ops(Ts, 1, N)
    value = ops / dt / 1e12
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "TOPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic (seeded generator)",
            "config": {"workload": args.workload, "description": WORKLOADS[args.workload][1],
                       "n_inputs": N, "n_freq": F, "t_integ": T, "step_sample": "channel 0, %d samples" % Ts},
            "sample_ops_per_step": ops, "workload_ops_per_step": useful_ops(T, F, N),
            "extrapolation": ("value = useful ops of the sample / its time; the oracle's work grows linearly with "
                              "channels and samples, so the whole workload (%.3g ops) would take %.1f s per step "
                              "on these cores" % (useful_ops(T, F, N), useful_ops(T, F, N) / (value * 1e12))),
            "cpu_baseline": {"value": value, "unit": "TOPS", "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": "channel 0, all %d inputs, %d samples per step" % (N, Ts)},
            "e2e": {"value": value, "unit": "TOPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def batch_launches(recipes):
    """Kernel launches of one batched run, as the library plans them: one
    persistent launch over every block pair of the jobs the 2-CTA pair kernel
    takes (up to 32,768 samples), one single-pass launch per 32,768 samples of
    each other job a single-pass kernel takes, and for the rest the TMA decode
    (N % 16 == 0 above FUSED_MAX_N), the thread-per-row decode (other N), the
    nibble-sums pass (with the TMA decode) and one listed tensor-core launch."""
    single = [r for r in recipes if r.N % 16 == 0 and r.N <= FUSED_MAX_N]
    listed = [r for r in single if r.N > 256 and use_pair_kernel(r.N) and r.T <= 32768]
    rest = [r for r in recipes if r not in single]
    n = (1 if listed else 0) + sum(-(-r.T // 32768) for r in single if r not in listed)
    tma = any(r.N % 16 == 0 for r in rest)
    if rest:
        n += (2 if tma else 0) + (1 if any(r.N % 16 for r in rest) else 0) + 1
    return n


def batched_record(args, steps, warmup, local_rank):
    """The batched workload (64 uneven jobs): one planned, graph-captured batch
    run per step, against one xeng_correlate call per job (tensor engine) and
    one dp4a launch per job on the same GPU.  Returns the record's fields."""
    import torch
    import synth
    import paper_1503_06202_gb300 as xe

    recipes = synth.batched_jobs()
    stream = torch.cuda.Stream()
    jobs = []
    with torch.cuda.stream(stream):
        for r in recipes:
            out = torch.empty((r.F, r.N * (r.N + 1) // 2, 2), dtype=torch.int32, device="cuda")
            jobs.append((r.device(stream), out))
    stream.synchronize()
    ops = sum(useful_ops(r.T, r.F, r.N) for r in recipes)
    cache = os.path.join(tempfile.gettempdir(), "xeng_batch_tune.jsonl")
    t0 = time.perf_counter()
    if args.batch_max_chunks > 0:  # a fixed plan (profiling runs), no tuning
        rc, opts, tuned_ms = 2, xe.xeng._opts(args.batch_max_chunks, args.batch_policy, True, args.batch_tile_order), None
    else:
        rc, opts, tuned_ms = xe.xeng_batch_autotune(jobs, cache, reps=3)
    tune_s = time.perf_counter() - t0
    if rc < 0:
        raise RuntimeError("autotune failed: %s" % xe.xeng_strerror(rc))
    b = xe.XBatch(jobs, opts)
    for _ in range(warmup):
        b.run(stream)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(gpu_index_for(local_rank)) as clk:
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(steps):
            b.run(stream)
        ev1.record(stream)
        ev1.synchronize()
    ms = ev0.elapsed_time(ev1) / steps
    clocks = clk.summary()
    info = b.info()

    # one plain call per job on the same GPU: tensor engine, then dp4a
    def per_job(engine, reps):
        engs = [xe.XEngine(r.N, r.F, r.T, engine) for r in recipes]
        for e_, (d, o) in zip(engs, jobs):
            e_.correlate(d, o, d.shape[0], stream)
        ev0.record(stream)
        for _ in range(reps):
            for e_, (d, o) in zip(engs, jobs):
                e_.correlate(d, o, d.shape[0], stream)
        ev1.record(stream)
        ev1.synchronize()
        t = ev0.elapsed_time(ev1) / reps
        for e_ in engs:
            e_.close()
        return t
    per_tc_ms = per_job(xe.XENG_ENGINE_TENSOR, 3)
    per_dp4a_ms = per_job(xe.XENG_ENGINE_DP4A, 1) if not args.no_per_job_dp4a else float("nan")
    b.close()
    del jobs
    torch.cuda.synchronize()
    peaks, peak_src = load_peaks()
    value = ops / (ms * 1e-3) / 1e12
    return {"value": value, "unit": "TOPS", "ms_per_step": ms, "steps": steps, "warmup": warmup,
            "config": {"workload": "batched", "description": WORKLOADS["batched"][1], "n_jobs": len(recipes),
                       "input_gb": sum(r.nbytes for r in recipes) / 1e9, "useful_ops": ops,
                       "l2": "inputs (%.1f GB) larger than L2; no flush" % (sum(r.nbytes for r in recipes) / 1e9)},
            "step_call": "xeng_batch_run (CUDA graph: one persistent 2-CTA pair-kernel launch over the block pairs "
                         "of every job it takes; single-pass launches for the other jobs with N % 16 == 0 (N <= 256: "
                         "on a side branch); the rest decoded to planes, then one persistent listed tensor-core "
                         "launch)",
            "gpu_launches": batch_launches(recipes) * steps,
            "autotune": {"opts": opts.as_dict(), "tuned_ms": tuned_ms, "from_cache": rc == 1, "fixed": rc == 2,
                         "tune_s": tune_s},
            "plan": info,
            "per_job_tensor": {"ms": per_tc_ms, "tops": ops / (per_tc_ms * 1e-3) / 1e12},
            "per_job_dp4a": {"ms": per_dp4a_ms, "tops": ops / (per_dp4a_ms * 1e-3) / 1e12, "launches": len(recipes)},
            "speedup_vs_per_job_tensor": per_tc_ms / ms, "speedup_vs_per_job_dp4a": per_dp4a_ms / ms,
            "roofline": {"bound": "tensor", "kernel": "single-pass kernels per job; decode + correlate_tc_kernel "
                                                      "(listed) for the rest",
                         "achieved": value, "peak": 2.0 * peaks["bf16_tflops_sustained"], "unit": "TFLOP/s",
                         "frac": value / (2.0 * peaks["bf16_tflops_sustained"]), "traffic": None,
                         "note": "whole batched run, useful ops; peak = 2 x %s sustained bf16" % peak_src},
            "clocks": clocks}


def run_batched(args, rank, world, local_rank):
    """--workload batched: the batched record as the contract's JSON line."""
    import torch
    torch.cuda.set_device(local_rank)
    r = batched_record(args, args.steps, args.warmup, local_rank)
    line = {"metric": METRIC, "value": r.pop("value"), "unit": r.pop("unit"), "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r.pop("ms_per_step"), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "fp8e4m3->f32 (exact integers)", "data": "synthetic (seeded on-device generator)",
            "config": r.pop("config"), "gpu_launches": r.pop("gpu_launches"), "clocks": r.pop("clocks"),
            "e2e": None, "cpu_baseline": None}
    line.update(r)
    if rank == 0:
        print(json.dumps(line), flush=True)


def serving_record(args, rates, seconds):
    """The streaming workload through the xserve_* service: Poisson block
    arrivals at r x the real-time rate per stream, continuous batching, dumps
    every 65536 samples; sustained TOPS and latency percentiles per rate,
    against one plain xeng_push per block.  Returns the record's fields."""
    import threading
    import numpy as np
    import torch
    import synth
    import paper_1503_06202_gb300 as xe

    BS, DUMP, POOL = 256, 65536, 16
    real_rate = 1.0 / (BS * 2.56e-6)  # blocks per second per stream at the 2.56 us sample period
    shapes = [(256, 256)] * 3 + [(512, 256)] * 3 + [(2048, 256)] * 2
    pools = []
    for k, (N, F) in enumerate(shapes):
        pools.append([synth.Recipe("uniform", T=BS, F=F, N=N, seed=4, stream=k * POOL + b).device() for b in range(POOL)])
    torch.cuda.synchronize()
    demand = [8.0 * BS * F * N * (N + 1) / 2 * real_rate / 1e12 for N, F in shapes]
    results = []
    rng = np.random.default_rng(5)
    for rate in rates:
        rc, sv = xe.xserve_create(hbm_budget_bytes=120 << 30, max_blocks=args.serve_max_blocks, max_streams=16,
                                  compute_budget_tops=args.serve_compute_budget)
        if rc != xe.XENG_OK:
            raise RuntimeError("xserve_create: " + xe.xeng_strerror(rc))
        ids, admitted = [], []
        for k, (N, F) in enumerate(shapes):
            rc, sid = xe.xserve_open_stream(sv, N, F, BS, DUMP, rate * real_rate)
            if rc == xe.XENG_ERR_NOMEM and args.serve_compute_budget > 0:
                continue  # refused by the compute budget: this stream is not served at this rate
            if rc != xe.XENG_OK:
                raise RuntimeError("admission refused: " + xe.xeng_strerror(rc))
            ids.append(sid)
            admitted.append(k)
        outs = [torch.empty((F, N * (N + 1) // 2, 2), dtype=torch.int32, device="cuda") for N, F in shapes]
        events = []
        for k in admitted:
            t = rng.exponential(1.0 / (rate * real_rate))
            while t < seconds:
                events.append((t, k))
                t += rng.exponential(1.0 / (rate * real_rate))
        events.sort()
        stop = threading.Event()
        dumps = [0] * len(shapes)
        sid_of = dict(zip(admitted, ids))

        def poller():
            while not stop.is_set():
                got = False
                for k in admitted:
                    r_, _ = xe.xserve_poll_dump(sv, sid_of[k], outs[k])
                    if r_ == 1:
                        dumps[k] += 1
                        got = True
                if not got:
                    time.sleep(5e-4)
        th = threading.Thread(target=poller, daemon=True)
        th.start()
        n_sub = [0] * len(shapes)
        t0 = xe.xserve_now()
        for t, k in events:
            while xe.xserve_now() - t0 < t:
                pass
            xe.xserve_submit(sv, sid_of[k], pools[k][n_sub[k] % POOL], 0.0)
            n_sub[k] += 1
        t_arr = xe.xserve_now() - t0
        _, st_end = xe.xserve_stats(sv)
        xe.xserve_drain(sv, 600.0)
        time.sleep(0.05)
        stop.set()
        th.join()
        rc, st = xe.xserve_stats(sv)
        xe.xserve_destroy(sv)
        results.append({"rate": rate, "admitted_streams": ["N=%d F=%d" % shapes[k] for k in admitted],
                        "offered_tops": rate * sum(demand[k] for k in admitted), "arrival_window_s": t_arr,
                        "blocks": sum(n_sub), "sustained_tops": st["useful_ops"] / st["busy_s"] / 1e12,
                        "busy_s": st["busy_s"], "rounds": st["rounds"], "dumps": st["dumps_done"],
                        "backlog_blocks_at_end_of_arrivals": st_end["backlog_blocks"],
                        "block_latency_p50_ms": st["block_p50_s"] * 1e3, "block_latency_p99_ms": st["block_p99_s"] * 1e3,
                        "dump_latency_p50_ms": st["dump_p50_s"] * 1e3, "dump_latency_p99_ms": st["dump_p99_s"] * 1e3,
                        "gpu_decode_ms": st["gpu_decode_ms"], "gpu_correlate_ms": st["gpu_correlate_ms"],
                        "host_plan_ms": st["host_plan_ms"]})
        del outs

    # plain comparison: one xeng_push per block, streams round-robin, closed loop
    engs = [xe.XEngine(N, F, DUMP) for N, F in shapes]
    nblk = 32
    for e_, pool in zip(engs, pools):
        e_.push(pool[0], BS)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for b in range(nblk):
        for e_, pool in zip(engs, pools):
            e_.push(pool[b % POOL], BS)
    torch.cuda.synchronize()
    plain_s = time.perf_counter() - t0
    plain_tops = nblk * sum(8.0 * BS * F * N * (N + 1) / 2 for N, F in shapes) / plain_s / 1e12
    for e_ in engs:
        e_.close()
    del pools
    torch.cuda.synchronize()
    head = results[0]
    return {"value": head["sustained_tops"], "unit": "TOPS", "ms_per_step": head["busy_s"] * 1e3,
            "config": {"workload": "serving", "description": WORKLOADS["serving"][1],
                       "streams": ["N=%d F=%d" % sh for sh in shapes], "block_samples": BS, "dump_samples": DUMP,
                       "max_blocks_per_round": args.serve_max_blocks, "arrival_seconds": seconds,
                       "compute_budget_tops": args.serve_compute_budget,
                       "real_time_blocks_per_s": real_rate, "real_time_demand_tops": sum(demand)},
            "per_rate": results, "plain_per_block_push_tops": plain_tops,
            "speedup_vs_plain_per_block": head["sustained_tops"] / plain_tops}


def run_serving(args, rank, world, local_rank):
    """--workload serving: the serving record as the contract's JSON line."""
    import torch
    torch.cuda.set_device(local_rank)
    r = serving_record(args, args.serve_rates, args.serve_seconds)
    line = {"metric": METRIC, "value": r.pop("value"), "unit": r.pop("unit"), "n_gpus": world,
            "steps": len(r["per_rate"]), "warmup": 0, "ms_per_step": r.pop("ms_per_step"), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "fp8e4m3->f32 (exact integers)",
            "data": "synthetic (seeded on-device block pools)", "config": r.pop("config"),
            "e2e": None, "cpu_baseline": None}
    line.update(r)
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="xeng", choices=["xeng", "reference"])
    ap.add_argument("--workload", default="chime_full", choices=sorted(WORKLOADS))
    ap.add_argument("--engine", default="tensor", choices=["tensor", "dp4a", "planes", "fused"],
                    help="tensor: the default engine; planes: always decode to HBM planes, then correlate; "
                         "fused: single pass (raw bytes split in shared memory) wherever N is a multiple of 16")
    ap.add_argument("--no-engine-compare", "--no-fused-compare", dest="no_engine_compare", action="store_true",
                    help="skip timing the two-pass (planes) engine beside the default one")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-peaks", action="store_true", help="skip the dense-throughput probes")
    ap.add_argument("--no-shift", action="store_true", help="skip the time-shift measurement")
    ap.add_argument("--no-gate", action="store_true", help="skip the gating + flags measurement")
    ap.add_argument("--no-beam", action="store_true", help="skip the beamforming measurement")
    ap.add_argument("--no-secondary", action="store_true", help="skip the Pathfinder-rate measurement")
    ap.add_argument("--no-dp4a", action="store_true", help="skip the plain dp4a comparison")
    ap.add_argument("--serve-rates", type=float, nargs="+", default=[1.0, 1.25, 1.5])
    ap.add_argument("--serve-seconds", type=float, default=1.5)
    ap.add_argument("--serve-max-blocks", type=int, default=128,
                    help="blocks a stream may contribute to one round (128 x 256 samples: one single-pass launch)")
    ap.add_argument("--serve-compute-budget", type=float, default=0.0, help="TOPS; > 0 admits streams by compute too")
    ap.add_argument("--batch-max-chunks", type=int, default=0, help="fixed batch plan instead of autotuning")
    ap.add_argument("--batch-policy", type=int, default=1)
    ap.add_argument("--batch-tile-order", type=int, default=0, help="with --batch-max-chunks: 0 row-major, 1 diagonal, 2 Morton")
    ap.add_argument("--no-per-job-dp4a", action="store_true")
    ap.add_argument("--no-systems", action="store_true",
                    help="skip the batched and served records of the default run")
    ap.add_argument("--systems-serve-seconds", type=float, default=0.75,
                    help="arrival window of the default run's serving record (one rate, 1.0x)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "batched":
        run_batched(args, rank, world, local_rank)
        return
    if args.workload == "serving":
        run_serving(args, rank, world, local_rank)
        return

    import torch
    import synth
    import paper_1503_06202_gb300 as xe

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    rec = getattr(synth, WORKLOADS[args.workload][0])
    T, F, N = rec.T, rec.F, rec.N
    B = N * (N + 1) // 2
    probes = None
    if not args.no_peaks:
        probes = {}
        for name, kind, iters in (("tc_f8f6f4", xe.XENG_PEAK_TC_F8F6F4, 1 << 21), ("tc_f16", xe.XENG_PEAK_TC_F16, 1 << 20),
                                  ("tc_f8f6f4_n128", xe.XENG_PEAK_TC_F8F6F4_N128, 1 << 21),
                                  ("tc_f8f6f4_correlator_mix", xe.XENG_PEAK_TC_F8F6F4_MIX, 1 << 20),
                                  ("tc_f8f6f4_live_data", xe.XENG_PEAK_TC_F8F6F4_LIVE, 1 << 21),
                                  ("tc_f8f6f4_live_raw_nibbles", xe.XENG_PEAK_TC_F8F6F4_LIVE_RAW, 1 << 21),
                                  ("mma_sync_s8", xe.XENG_PEAK_MMA_SYNC_S8, 200000), ("dp4a", xe.XENG_PEAK_DP4A, 500000)):
            rc, tf, pms = xe.xeng_peak_probe(kind, iters)
            probes[name] = round(tf, 1) if rc == 0 else None
    engine = {"tensor": xe.XENG_ENGINE_TENSOR, "dp4a": xe.XENG_ENGINE_DP4A,
              "planes": xe.XENG_ENGINE_TENSOR_PLANES, "fused": xe.XENG_ENGINE_TENSOR_FUSED}[args.engine]
    tensor_engine = args.engine != "dp4a"
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        block = rec.device(stream)
        out = torch.empty((F, B, 2), dtype=torch.int32, device="cuda")
    stream.synchronize()
    eng = xe.XEngine(N, F, T, engine)

    def step():
        eng.correlate(block, out, T, stream)

    for _ in range(args.warmup):
        step()
    stream.synchronize()
    eng.set_profiling(True)
    eng.stats(reset=True)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(gpu_index_for(local_rank)) as clk:
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        ev1.synchronize()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
    ms = ev0.elapsed_time(ev1) / args.steps
    st = eng.stats(reset=True)
    eng.set_profiling(False)
    clocks = clk.summary()
    # the same integration through xeng_push + xeng_dump (adds the triangle copy)
    def push_dump(reps=2):
        eng.set_profiling(True)
        eng.stats(reset=True)
        ev0.record(stream)
        for _ in range(reps):
            eng.push(block, T, stream)
            eng.dump(out, stream)
        ev1.record(stream)
        ev1.synchronize()
        s2 = eng.stats(reset=True)
        eng.set_profiling(False)
        return ev0.elapsed_time(ev1) / reps, s2["decode_ms"] / reps

    push_dump_ms, push_dump_decode_ms = push_dump()
    # the two-pass engine on the same block (decode to FP8 planes in HBM, then the
    # tensor-core GEMM), measured in the same run beside the default engine
    planes_cmp = None
    if args.engine == "tensor" and N > 256 and N % 16 == 0 and not args.no_engine_compare:
        eng_p = xe.XEngine(N, F, T, xe.XENG_ENGINE_TENSOR_PLANES)
        out_p = torch.empty_like(out)
        for _ in range(2):
            eng_p.correlate(block, out_p, T, stream)
        eng_p.set_profiling(True)
        eng_p.stats(reset=True)
        reps_p = 3
        ev0.record(stream)
        for _ in range(reps_p):
            eng_p.correlate(block, out_p, T, stream)
        ev1.record(stream)
        ev1.synchronize()
        sp = eng_p.stats(reset=True)
        p_ms = ev0.elapsed_time(ev1) / reps_p
        planes_cmp = {"engine": "tensor_planes", "ms_per_step": p_ms,
                      "value": useful_ops(T, F, N) / (p_ms * 1e-3) / 1e12, "unit": "TOPS",
                      "decode_ms_per_step": sp["decode_ms"] / reps_p,
                      "correlate_ms_per_step": sp["correlate_ms"] / reps_p,
                      "equals_default_engine_output": bool(torch.equal(out_p, out)),
                      "kernels": "decode_tma_kernel + plane_sums_kernel + correlate_tc_kernel (raw-nibble FP8 "
                                 "planes in HBM, 128-input tile pairs)"}
        eng_p.close()
        del out_p
        torch.cuda.synchronize()
    # time shifting (Sec. IV-C-5): two inputs of an outlying station delayed by
    # 168 ms (65,625 samples), the rest undelayed; the stream history carries
    # across the pushes
    shift = None
    if tensor_engine and not args.no_shift:
        import numpy as np
        d = np.zeros(N, np.int32)
        d[N - 2:] = 65625
        eng.set_delays(d)
        push_dump(1)
        sh_ms, sh_dec = push_dump()
        eng.set_delays(None)
        eng.correlate(block, out, T, stream)  # `out` holds the unshifted result again for the CPU check
        stream.synchronize()
        shift = {"delayed_inputs": 2, "delay_samples": 65625, "push_dump_ms_per_step": sh_ms,
                 "decode_ms_per_step": sh_dec, "unshifted_push_dump_ms_per_step": push_dump_ms,
                 "unshifted_decode_ms_per_step": push_dump_decode_ms,
                 "value": whole_job_rate(useful_ops(T, F, N), max_over_ranks(sh_ms, dist) * 1e-3, world) / 1e12,
                 "unit": "TOPS"}
    # gating and flags (Sec. IV-C-4, Sec. IV-A): the samples split into two phase
    # gates (on / off, alternating every 64 samples) and 1% of the (sample,
    # channel, input) bytes flagged; the counts of usable samples come back too
    gating = None
    if tensor_engine and not args.no_gate:
        import numpy as np
        G = 2
        gate = ((np.arange(T) // 64) % G).astype(np.int32)
        valid = torch.randint(0, 100, (T, F, N), dtype=torch.uint8, device="cuda")
        valid.clamp_(max=1)  # 0 (1 in 100: flagged) or 1
        gout = torch.empty((G, F, N * (N + 1) // 2, 2), dtype=torch.int32, device="cuda")
        gcounts = torch.empty((G, F, N), dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()

        def gated():
            rc = xe.xeng_correlate_gated(eng.h, block, T, gate, G, valid, gout, gcounts, stream)
            if rc != xe.XENG_OK:
                raise xe.XengError(rc, "xeng_correlate_gated")

        gated()
        eng.set_profiling(True)
        eng.stats(reset=True)
        greps = 2
        ev0.record(stream)
        for _ in range(greps):
            gated()
        ev1.record(stream)
        ev1.synchronize()
        gst = eng.stats(reset=True)
        eng.set_profiling(False)
        g_ms = ev0.elapsed_time(ev1) / greps
        gating = {"gates": G, "gate_period_samples": 128, "flagged_fraction": 0.01, "ms_per_step": g_ms,
                  "decode_ms_per_step": gst["decode_ms"] / greps,
                  "correlate_ms_per_step": gst["correlate_ms"] / greps,
                  "value": whole_job_rate(useful_ops(T, F, N), max_over_ranks(g_ms, dist) * 1e-3, world) / 1e12,
                  "unit": "TOPS", "ungated_ms_per_step": ms,
                  "kernels": "decode_gather_kernel (gate rows, flags, counts) + correlate_tc_kernel per gate"}
        del valid, gout, gcounts
        torch.cuda.synchronize()
    # beamforming (Sec. IV-C-3): 16 beams over the same block, int8 weights;
    # HBM-bound: reads the block once, writes T x F x 16 complex int32
    beam = None
    if tensor_engine and not args.no_beam:
        nb = 16
        bf = xe.XBeam(N, F, nb)
        g = torch.Generator(device="cuda").manual_seed(5)
        with torch.cuda.stream(stream):
            w_re = torch.randint(-128, 128, (F, nb, N), dtype=torch.int8, device="cuda", generator=g)
            w_im = torch.randint(-128, 128, (F, nb, N), dtype=torch.int8, device="cuda", generator=g)
            bout = torch.empty((T, F, nb, 2), dtype=torch.int32, device="cuda")
        bf.set_weights(w_re, w_im, stream)
        for _ in range(3):
            bf.run(block, bout, T, stream)
        reps = 10
        ev0.record(stream)
        for _ in range(reps):
            bf.run(block, bout, T, stream)
        ev1.record(stream)
        ev1.synchronize()
        bms = ev0.elapsed_time(ev1) / reps
        peaks_b, src_b = load_peaks()
        bytes_alg = T * F * N + T * F * nb * 8
        beam = {"n_beams": nb, "ms_per_step": bms, "bound": "hbm", "algorithmic_bytes": bytes_alg,
                "achieved": bytes_alg / (bms * 1e-3) / 1e9, "peak": peaks_b["hbm_gbs"], "unit": "GB/s",
                "cmac_per_s": T * F * N * nb / (bms * 1e-3), "kernel": "beamform_kernel<16>"}
        beam["frac"] = beam["achieved"] / beam["peak"]
        bf.close()
        del w_re, w_im, bout
    # the Pathfinder-rate configuration (N = 256, 1024 channels, 32768 samples)
    # beside the default one: its step is the fused decode + correlation
    secondary = None
    if args.workload == "chime_full" and args.engine == "tensor" and not args.no_secondary:
        r2 = synth.PATHFINDER_FULL
        with torch.cuda.stream(stream):
            blk2 = r2.device(stream)
            out2 = torch.empty((r2.F, r2.N * (r2.N + 1) // 2, 2), dtype=torch.int32, device="cuda")
        stream.synchronize()
        eng2 = xe.XEngine(r2.N, r2.F, r2.T, engine)
        for _ in range(3):
            eng2.correlate(blk2, out2, r2.T, stream)
        reps2 = 10
        ev0.record(stream)
        for _ in range(reps2):
            eng2.correlate(blk2, out2, r2.T, stream)
        ev1.record(stream)
        ev1.synchronize()
        ms2 = ev0.elapsed_time(ev1) / reps2
        secondary = {"workload": "pathfinder_full", "description": WORKLOADS["pathfinder_full"][1],
                     "ms_per_step": ms2, "value": useful_ops(r2.T, r2.F, r2.N) / (ms2 * 1e-3) / 1e12, "unit": "TOPS",
                     "steps": reps2, "kernel": "correlate_small_kernel (decode fused into the correlation; "
                                               "upper-triangle 128-input blocks)"}
        eng2.close()
        del blk2, out2
    # the plain single-instance CUDA-core (dp4a) correlator on the same GPU, on
    # a channel sample of the same block (its full step takes seconds): its
    # rate, and whether its output equals the tensor path's for those channels
    plain_dp4a = None
    if tensor_engine and not args.no_dp4a:
        fs = min(F, 16)
        with torch.cuda.stream(stream):
            blk_s = block[:, :fs, :].contiguous()
            out_s = torch.empty((fs, B, 2), dtype=torch.int32, device="cuda")
        eng_d = xe.XEngine(N, fs, T, xe.XENG_ENGINE_DP4A)
        eng_d.correlate(blk_s, out_s, T, stream)
        reps_d = 3
        ev0.record(stream)
        for _ in range(reps_d):
            eng_d.correlate(blk_s, out_s, T, stream)
        ev1.record(stream)
        ev1.synchronize()
        d_ms = ev0.elapsed_time(ev1) / reps_d
        d_full_ms = d_ms * F / fs
        plain_dp4a = {"kernel": "correlate_dp4a_kernel", "sample": "channels 0..%d of the same block, %d runs" % (fs - 1, reps_d),
                      "ms_per_sample_run": d_ms, "ms_per_step_extrapolated": d_full_ms,
                      "value": useful_ops(T, fs, N) / (d_ms * 1e-3) / 1e12, "unit": "TOPS",
                      "equals_tensor_output": bool(torch.equal(out_s, out[:fs]))}
        eng_d.close()
        del blk_s, out_s
    ms = max_over_ranks(ms, dist)
    ops = useful_ops(T, F, N)
    value = whole_job_rate(ops, ms * 1e-3, world) / 1e12
    if plain_dp4a:
        plain_dp4a["tensor_path_speedup"] = plain_dp4a["ms_per_step_extrapolated"] / ms

    # dominant kernel: the correlation launches, timed live over the timed region
    peaks, peak_src = load_peaks()
    corr_ms = st["correlate_ms"] / max(1, st["timed_correlate"])
    launches_per_step = st["correlate_launches"] / args.steps
    flops_per_launch = ops / launches_per_step
    if tensor_engine:
        peak = 2.0 * peaks["bf16_tflops_sustained"]
        kernel, tile = correlate_kernel(args.engine, N)
        peak_note = ("fp8 dense = 2 x %s sustained bf16 %.1f TFLOP/s (nominal fp8:bf16 = 4.5:2.25); "
                     "sm_103a has no tcgen05 kind::i8; the bf16 figure was sustained at a power-capped clock, "
                     "so frac can exceed 1 -- the fp8 probes measured in this run (peak_probe_*) are the "
                     "ceilings at this kernel's clock" % (peak_src, peaks["bf16_tflops_sustained"]))
        per_ch = DRAM_BYTES_PER_CHANNEL.get((kernel.split()[0].replace("_kernel", ""), N, T))
        traffic = per_ch * F / launches_per_step if per_ch else None
        roof = {"bound": "tensor", "kernel": kernel, "achieved": flops_per_launch / (corr_ms * 1e-3) / 1e12,
                "peak": peak, "unit": "TFLOP/s", "traffic": traffic, "peak_note": peak_note}
        if traffic:
            # algorithmic bytes of one launch: the operands read once (planes: 2 bytes per
            # input and sample; raw: 1 byte) and the triangle written once
            op_bytes = (2 if kernel.startswith("correlate_tc") else 1) * T * N * F / launches_per_step
            roof["algorithmic_bytes"] = op_bytes + 8.0 * B * F / launches_per_step
            roof["traffic_over_algorithmic"] = traffic / roof["algorithmic_bytes"]
            roof["traffic_source"] = "ncu capture of the 16-channel slice, scaled by channels"
        roof["frac"] = roof["achieved"] / peak
        if probes and probes.get("tc_f8f6f4"):
            roof["peak_probe_fp8"] = probes["tc_f8f6f4"]
            roof["frac_of_probe_fp8"] = roof["achieved"] / probes["tc_f8f6f4"]
            # useful ops exclude the lower halves of diagonal tiles (and the padding past N)
            # the MMAs also compute: nt (nt + 1) / 2 tiles of tile x tile per channel
            nt = -(-N // tile)
            executed = (nt * (nt + 1) // 2 * tile * tile) / (N * (N + 1) / 2)
            roof["executed_over_useful"] = executed
            roof["frac_executed_of_probe_fp8"] = roof["achieved"] * executed / probes["tc_f8f6f4"]
        if probes and probes.get("tc_f8f6f4_live_data"):
            roof["peak_probe_fp8_live_data"] = probes["tc_f8f6f4_live_data"]
            roof["frac_executed_of_probe_fp8_live_data"] = (roof["achieved"] * roof.get("executed_over_useful", 1.0)
                                                           / probes["tc_f8f6f4_live_data"])
        if probes and probes.get("tc_f8f6f4_live_raw_nibbles"):
            # the operands the tensor path feeds: codes of raw nibbles (u / 512)
            roof["peak_probe_fp8_live_raw_nibbles"] = probes["tc_f8f6f4_live_raw_nibbles"]
            roof["frac_executed_of_probe_fp8_live_raw_nibbles"] = (
                roof["achieved"] * roof.get("executed_over_useful", 1.0) / probes["tc_f8f6f4_live_raw_nibbles"])
        if probes and probes.get("mma_sync_s8"):
            roof["frac_of_probe_int8_mma_sync"] = roof["achieved"] / probes["mma_sync_s8"]
    else:
        roof = {"bound": "alu", "kernel": "correlate_dp4a_kernel",
                "achieved": flops_per_launch / (corr_ms * 1e-3) / 1e12, "peak": None, "unit": "TFLOP/s",
                "traffic": None, "frac": None}
    roof["avg_launch_ms"] = corr_ms
    roof["decode_ms_per_step"] = st["decode_ms"] / args.steps
    # the decode stage (HBM-bound): 1 byte read + 2 plane bytes written per (input, sample, channel)
    decode_roof = None
    if tensor_engine and st["decode_ms"] > 0:
        dec_ms = st["decode_ms"] / args.steps
        dec_bytes = 3 * T * F * N
        decode_roof = {"kernel": "decode_tma_kernel" if N % 16 == 0 else "decode_kernel", "bound": "hbm",
                       "ms_per_step": dec_ms, "algorithmic_bytes": dec_bytes,
                       "achieved": dec_bytes / (dec_ms * 1e-3) / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                       "frac": dec_bytes / (dec_ms * 1e-3) / 1e9 / peaks["hbm_gbs"], "peak_source": peak_src}

    # end to end through the ABI with host buffers: H2D of the block, D2H of the triangle
    e2e = None
    if not args.no_e2e:
        hblock = torch.empty((T, F, N), dtype=torch.uint8, pin_memory=True)
        hblock.copy_(block)
        hout = torch.empty((F, B, 2), dtype=torch.int32, pin_memory=True)
        eng.correlate(hblock, hout, T, stream)  # warm: staging allocation
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        each = []
        for _ in range(args.e2e_steps):
            t1 = time.perf_counter()
            eng.correlate(hblock, hout, T, stream)  # returns once the triangle is in host memory
            each.append(round((time.perf_counter() - t1) * 1e3, 1))
        dt = max_over_ranks((time.perf_counter() - t0) / args.e2e_steps, dist)
        # host-link copies from pinned memory vary from call to call on these hosts
        # (the same buffers: 122 to 314 ms per call for full CHIME), so each call's
        # time is kept beside the mean
        e2e = {"value": whole_job_rate(ops, dt, world) / 1e12, "unit": "TOPS", "h2d_bytes_per_step": T * F * N,
               "d2h_bytes_per_step": F * B * 8, "ms_per_step": dt * 1e3, "ms_each_step": each}
        del hblock, hout

    cpu = None
    exact = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu, exact = cpu_oracle_sample(rec, T, F, N, out)

    # the batched and served workloads (configs of 64 uneven jobs and of 8
    # concurrent streams) beside the plain per-instance kernels, in the same
    # run, after the default workload's buffers are freed
    batched = serving = None
    if args.workload == "chime_full" and args.engine == "tensor" and not args.no_systems:
        eng.close()
        eng = None
        del block, out
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        batched = batched_record(args, 5, 3, local_rank)
        torch.cuda.empty_cache()
        serving = serving_record(args, [1.0], args.systems_serve_seconds)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "TOPS", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "fp8e4m3->f32 (exact integers)" if tensor_engine else "int8->int32",
                "data": "synthetic (seeded on-device generator)",
                "config": {"workload": args.workload, "description": WORKLOADS[args.workload][1],
                           "n_inputs": N, "n_freq": F, "t_integ": T, "engine": args.engine,
                           "parallelism": "replicas" if world > 1 else "single GPU",
                           "l2": "inputs (%.1f GiB) larger than L2; no flush" % (T * F * N / 2 ** 30)},
                "cmac_per_s": value / 8.0 * 1e12, "ops_per_cmac": 8, "step_call": "xeng_correlate",
                "push_dump_ms_per_step": push_dump_ms, "two_pass_engine": planes_cmp, "time_shift": shift, "gating": gating, "beamform": beam,
                "pathfinder_rate": secondary, "plain_dp4a": plain_dp4a, "batched": batched, "serving": serving,
                "gpu_launches": int(st["launches"]), "roofline": roof, "decode_roofline": decode_roof,
                "peak_probes_tflops": probes, "clocks": clocks, "e2e": e2e,
                "cpu_baseline": cpu, "bit_exact_on_cpu_sample": exact}
        print(json.dumps(line), flush=True)
    if eng is not None:
        eng.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
