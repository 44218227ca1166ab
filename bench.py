#!/usr/bin/env python
"""Benchmark of the sketched proximal TT-ALS hot path (Algorithm 1, TT-TS) on one GB300.

One step = one outer iteration (sweep) of Algorithm 1 on the order-4 100^4 FP32 workload
(TT ranks (1,10,10,10,1), 1e-2 relative noise, J = 4096, lambda = 1e-3): right-to-left
orthogonalisation, a fresh TensorSketch draw, for every core the FFT interface sketch, the
data sketch of the unfolding (a full read of the 400 MB tensor per core), the proximal
update of Eq. (ite) and the QR step, then the relative error (one more read of the tensor).

Prints ONE JSON line (rank 0). `--impl reference` times the CPU FP64 oracle instead.
Under torchrun (N > 1) every rank runs an independent replica (the single-tensor path has no
data-parallel split without a collective) and rank 0 reports the aggregate.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ALS sweeps/s + unfold-sketch HBM GB/s at equal rel. error vs plain FP32 GPU"
# DRAM bytes (read + write) per data-sketch launch from an ncu capture of the current kernels,
# per (workload, storage); the roofline reports null for anything not captured.
UNFOLD_TRAFFIC = {("order4-100-r10", "f32"): 428.65e6}
UNIT = "sweeps/s"
DEFAULT_WORKLOAD = "order4-100-r10"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--storage", default=None, help="override the workload's storage type")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-patterns", action="store_true", help="skip the precision/batched/warm-start patterns")
    ap.add_argument("--only-pattern", default=None,
                    choices=["precision", "batched", "warmstart", "gemm", "sparse", "order3", "order5",
                             "deterministic", "gram", "window", "fixed"],
                    help="run one pattern and print its JSON")
    ap.add_argument("--ws-train", type=int, default=10240, help="warm-start training solves")
    ap.add_argument("--cpu-sample", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--cpu-columns", type=int, default=0, help=argparse.SUPPRESS)
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------------------------
# clocks during the timed region

class ClockSampler:
    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu_id: str):
        self.samples = []
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + ",".join(self.FIELDS), "--format=csv,noheader,nounits",
                 "-lms", "50", "-i", gpu_id], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._reader, daemon=True)
        self.thread.start()
        t0 = time.time()
        while not self.samples and time.time() - t0 < 5.0:
            time.sleep(0.02)

    def _reader(self):
        for line in self.proc.stdout:
            self.samples.append((time.time(), [x.strip() for x in line.split(",")]))

    def stop(self):
        if self.proc is not None:
            time.sleep(0.12)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, t0, t1):
        if self.proc is None:
            return None
        win = [s for (t, s) in self.samples if t0 - 0.06 <= t <= t1 + 0.06] or \
              [s for (t, s) in self.samples if t >= t0 - 0.2][:2]
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for s in win:
            try:
                sm.append(float(s[0]))
                mx.append(float(s[1]))
            except (ValueError, IndexError):
                continue
            for nm, val in zip(names, s[4:8]):
                if val.strip().lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------------------------
# CPU oracle legs

def _oracle_threads_env():
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[v] = "1"
    return env


def cpu_sample_main(args):
    """Child process: time one oracle sweep (Algorithm 1 outer iteration) of the workload, or
    `--cpu-columns q` columns of the oracle's data sketch per step (reference arm)."""
    sys.path.insert(0, os.path.join(ROOT, "oracle"))
    import numpy as np
    import tt_oracle as O
    from paper_2309_08093_gb300 import synth

    w = synth.WORKLOADS[args.workload]
    p = synth.make_problem(w, storage=args.storage)
    if args.cpu_columns == 0:  # (negative: the reference arm's automatic sample size)
        t = time.perf_counter()
        O.tt_ts_sweep(p.tensor, p.init_cores, p.sketch_seed, 0, w.J, w.lam)
        dt = time.perf_counter() - t
        hs, vs = O.draw_sketch(p.sketch_seed, 0, w.dims, w.J)  # the same columns, one thread
        t = time.perf_counter()
        for k in range(w.d):
            for i in range(w.dims[k]):
                O.sketch_unfolding_column(p.tensor, hs, vs, w.J, k, i)
        sk = time.perf_counter() - t
        del p
        all_s, cores, detail = cpu_all_cores(args, dt, sk)
        print(json.dumps({"sweep_s": dt, "sweep_all_cores_s": all_s, "cores": cores, **detail}))
        return
    # reference arm: each step sketches q columns of Y_k by definition, cycling over modes/columns
    hs, vs = O.draw_sketch(p.sketch_seed, 0, w.dims, w.J)
    cols = [(k, i) for k in range(w.d) for i in range(w.dims[k])]
    times = []
    pos = 0
    if args.cpu_columns < 0:  # size q so that the whole run takes about 150 s
        t = time.perf_counter()
        for j in range(2):
            O.sketch_unfolding_column(p.tensor, hs, vs, w.J, cols[j][0], cols[j][1])
        per = (time.perf_counter() - t) / 2
        args.cpu_columns = max(1, int(150.0 / ((args.steps + args.warmup) * max(per, 1e-3))))
    for step in range(args.warmup + args.steps):
        t = time.perf_counter()
        for _ in range(args.cpu_columns):
            k, i = cols[pos % len(cols)]
            pos += 1
            O.sketch_unfolding_column(p.tensor, hs, vs, w.J, k, i)
        times.append(time.perf_counter() - t)
    timed = times[args.warmup:]
    per_col = sum(timed) / (len(timed) * args.cpu_columns)
    print(json.dumps({"per_column_s": per_col, "columns_per_sweep": len(cols), "steps": len(timed),
                      "step_s": sum(timed) / len(timed), "q": args.cpu_columns}))


_W = {}


def _cols_worker(args):
    """Spawned worker (one numpy thread): the oracle's data-sketch columns (k, i_k) of one draw by
    their definition; the workload is built once per process. Returns the compute seconds."""
    workload, storage, cols, hold = args
    sys.path.insert(0, os.path.join(ROOT, "oracle"))
    import tt_oracle as O
    from paper_2309_08093_gb300 import synth

    if _W.get("name") != (workload, storage):
        w = synth.WORKLOADS[workload]
        p = synth.make_problem(w, storage=storage)
        _W.update(name=(workload, storage), p=p, w=w, hv=O.draw_sketch(p.sketch_seed, 0, w.dims, w.J))
    p, w = _W["p"], _W["w"]
    hs, vs = _W["hv"]
    t = time.perf_counter()
    for k, i in cols:
        O.sketch_unfolding_column(p.tensor, hs, vs, w.J, k, i)
    dt = time.perf_counter() - t
    time.sleep(hold)  # warm-up round: keeps this worker busy so that every worker gets one task
    return dt


def cpu_all_cores(args, sweep_1t_s, sketch_1t_s):
    """The sweep's data-sketch columns spread over one single-threaded process per available core
    (os.sched_getaffinity); the rest of the sweep (interface sketches, solves, QR: the one-thread
    sweep minus its one-thread data-sketch columns) stays serial. Returns (sweep seconds, cores,
    detail)."""
    import multiprocessing as mp

    from paper_2309_08093_gb300 import synth

    w = synth.WORKLOADS[args.workload]
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    cols = [(k, i) for k in range(w.d) for i in range(w.dims[k])]
    tasks = [cols[j::cores * 4] for j in range(cores * 4)]
    with mp.get_context("spawn").Pool(cores) as pool:
        pool.map(_cols_worker, [(args.workload, args.storage, [cols[0]], 2.0)] * cores, chunksize=1)
        t = time.perf_counter()
        busy = pool.map(_cols_worker, [(args.workload, args.storage, tk, 0.0) for tk in tasks], chunksize=1)
        wall = time.perf_counter() - t
    serial_rest = max(0.0, sweep_1t_s - sketch_1t_s)
    return wall + serial_rest, cores, {"sketch_wall_s": wall, "sketch_busy_s": sum(busy), "serial_rest_s": serial_rest,
                                       "sketch_one_thread_s": sketch_1t_s}


def run_cpu_child(extra):
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-sample"] + extra
    p = subprocess.run(cmd, capture_output=True, text=True, env=_oracle_threads_env(), timeout=1800)
    if p.returncode != 0:
        raise RuntimeError(p.stderr[-2000:])
    return json.loads(p.stdout.strip().splitlines()[-1])


def max_over_ranks(ms, dist, dev):
    """Timed-region length of the slowest rank (every rank gets it); ms itself on one process."""
    if dist is None:
        return ms
    import torch

    t = torch.tensor([float(ms)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world, steps, max_ms):
    """Whole-job sweeps/s: every rank sweeps its own replica `steps` times within max_ms."""
    return world * steps / (max_ms / 1e3)


def reference_main(args, rank, world):
    if rank != 0:
        return
    from paper_2309_08093_gb300 import synth

    w = synth.WORKLOADS[args.workload]
    res = run_cpu_child(["--workload", args.workload, "--cpu-columns", "-1", "--steps", str(args.steps),
                         "--warmup", str(args.warmup)] + (["--storage", args.storage] if args.storage else []))
    q = res["q"]
    sweep_s = res["per_column_s"] * res["columns_per_sweep"]
    value = 1.0 / sweep_s
    sample = (f"per step {q} column(s) of the data sketch Y_k = S A_(k)^T computed by the oracle's definition "
              f"(FP64 numpy, 1 thread), cycling over all {res['columns_per_sweep']} columns of the {w.d} modes; "
              f"sweep time = columns per sweep x mean column time (the data sketch is >95% of an oracle sweep "
              f"on this workload)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sweep_s * 1e3,
            "sample_ms_per_step": res["step_s"] * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(w, args.storage or w.storage),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def workload_config(w, storage):
    return {"workload": f"{w.name}: {'x'.join(map(str, w.dims))} {storage} tensor, TT ranks {list(w.ranks)}, "
                        f"J={w.J}, lambda={w.lam}, noise={w.noise}",
            "dims": list(w.dims), "ranks": list(w.ranks), "J": w.J, "lambda": w.lam, "storage": storage,
            "step": "one sweep of Algorithm 1 (d core updates) + relative error",
            "l2": "inputs larger than L2 (tensor %.0f MB > 129 MB)" % (w.numel * {"f64": 8, "f32": 4, "bf16": 2, "fp8": 1}[storage] / 1e6)}


# ---------------------------------------------------------------------------------------------
# precision pattern: the same workload with the tensor stored in BF16 (FP32 sketch accumulation,
# FP32 Gram, FP32 factorisation), compared with the plain FP32 form at equal relative error

def precision_pattern(w, p, dev, nsweeps):
    import numpy as np
    import torch
    from paper_2309_08093_gb300 import lib, synth

    stream = torch.cuda.current_stream()
    A32 = lib.device_tensor(p.storage, "f32", device=dev)
    ctx32 = lib.Context(w.dims, p.ranks, w.J, w.lam, p.sketch_seed, "f32")
    forms = {"f32": (ctx32, A32)}
    bits = synth.bf16_bits(np.asarray(p.storage, dtype=np.float32))
    ctx16 = lib.Context(w.dims, p.ranks, w.J, w.lam, p.sketch_seed, "bf16")
    forms["bf16"] = (ctx16, lib.device_tensor(bits, "bf16", device=dev))
    out = {}
    for name, (ctx, A) in forms.items():
        cores = lib.device_cores(p.init_cores, device=dev)
        errs, ms = [], 0.0
        for t in range(nsweeps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.tt_prox_als_sweep(A, cores, 1, t, rel_change=False)
            e1.record(stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
            errs.append(ctx32.tt_rel_error(A32, cores))  # always against the FP32 tensor
        out[name] = {"sweeps_per_s": nsweeps / (ms / 1e3), "rel_error_per_sweep": errs}
    target = out["f32"]["rel_error_per_sweep"][-1] * (1 + 1e-3)
    for name, r in out.items():
        hit = next((i + 1 for i, e in enumerate(r["rel_error_per_sweep"]) if e <= target), None)
        r["sweeps_to_tolerance"] = hit
        r["sweeps_to_tolerance_per_s"] = (r["sweeps_per_s"] / hit) if hit else None
        r["rel_error_final"] = r["rel_error_per_sweep"][-1]
        r["rel_error_per_sweep"] = [round(e, 8) for e in r["rel_error_per_sweep"]]
    for ctx, _ in forms.values():
        ctx.close()
    return {"tolerance": target, "sweeps": nsweeps,
            "note": "sweeps timed with CUDA events (no relative error inside the timed sweeps); errors "
                    "against the FP32 tensor; tolerance = FP32 form's final error x (1 + 1e-3)",
            "forms": out}


# ---------------------------------------------------------------------------------------------
# batched pattern: 256 independent tensors (orders 3-4, sizes 16-128, ranks 4-12, FP32 and BF16
# storage, about 12 GB) swept together, one graph launch per sweep

def batched_pattern(dev, nsweeps=10, count=256):
    import torch
    from paper_2309_08093_gb300 import lib, synth

    specs = synth.batched_specs(count=count)
    As, cores, inits = [], [], []
    for sp in specs:
        a, init = synth.batched_tensor_gpu(sp, device=dev)
        As.append(a)
        inits.append(init)
        cores.append(lib.device_cores(init, device=dev))
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    batch = lib.Batch(specs)
    t0 = time.perf_counter()
    batch.tt_batch_sweep(As, cores, 1, 0)          # autotune + capture + first sweep
    setup_s = time.perf_counter() - t0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    batch.tt_batch_sweep(As, cores, nsweeps, 1)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    errs = batch.tt_batch_rel_error(As, cores)
    batch.close()
    # the same sweeps with a fixed draw per tensor (TT_FLAG_FIXED_SKETCH): a call's first sweep
    # computes the data sketches, its later sweeps reuse them (a second graph)
    batch_f = lib.Batch([dict(sp, flags=lib.TT_FLAG_FIXED_SKETCH) for sp in specs])
    cores_f = [lib.device_cores(init, device=dev) for init in inits]
    batch_f.tt_batch_sweep(As, cores_f, 1, 0)    # capture + first sweep
    torch.cuda.synchronize()
    e0.record(stream)
    batch_f.tt_batch_sweep(As, cores_f, nsweeps, 1)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_f = e0.elapsed_time(e1)
    errs_f = sorted(batch_f.tt_batch_rel_error(As, cores_f))
    batch_f.close()
    del cores_f
    # the same sweeps one tensor at a time (a context per tensor, its own launches, no graph)
    ctxs = [lib.Context(sp["dims"], sp["ranks"], sp["J"], sp["lam"], sp["seed"], sp["dtype"]) for sp in specs]
    for c, a, cs in zip(ctxs, As, cores):
        c.tt_prox_als_sweep(a, cs, 1, 100, rel_change=False)  # warm: plans, tables
    torch.cuda.synchronize()
    e0.record(stream)
    for t in range(2):
        for c, a, cs in zip(ctxs, As, cores):
            c.tt_prox_als_sweep(a, cs, 1, 101 + t, rel_change=False)
    e1.record(stream)
    torch.cuda.synchronize()
    loop_ms = e0.elapsed_time(e1) / 2
    for c in ctxs:
        c.close()
    esz = {"f32": 4, "bf16": 2}
    tensor_bytes = sum(int(a.numel()) * esz[sp["dtype"]] for a, sp in zip(As, specs))
    unfold_bytes = sum(int(a.numel()) * esz[sp["dtype"]] * len(sp["dims"]) for a, sp in zip(As, specs))
    sweep_s = ms / 1e3 / nsweeps
    errs_sorted = sorted(errs)
    return {"tensors": count, "tensor_gb": tensor_bytes / 1e9, "sweeps": nsweeps,
            "tensor_sweeps_per_s": count / sweep_s, "ms_per_batched_sweep": sweep_s * 1e3,
            "ms_per_sweep_one_tensor_at_a_time": loop_ms,
            "tensor_sweeps_per_s_one_tensor_at_a_time": count / (loop_ms * 1e-3),
            "unfold_read_gbs_lower_bound": unfold_bytes / sweep_s / 1e9,
            "setup_s": setup_s,
            "rel_error_median": errs_sorted[len(errs) // 2], "rel_error_max": errs_sorted[-1],
            "fixed_draw": {"ms_per_batched_sweep": ms_f / nsweeps, "tensor_sweeps_per_s": count / (ms_f / 1e3 / nsweeps),
                           "rel_error_median": errs_f[len(errs_f) // 2], "rel_error_max": errs_f[-1],
                           "note": f"TT_FLAG_FIXED_SKETCH on every tensor; one call of {nsweeps} sweeps: the first "
                                   "computes the data sketches, the others reuse them"},
            "note": "noise 1e-3 (the floor); sweeps timed with CUDA events around one tt_batch_sweep call "
                    "(graph replays); unfold GB/s = tensor bytes x order / sweep time, everything else in "
                    "the sweep included"}


# ---------------------------------------------------------------------------------------------
# Gram of the proximal update: CUDA-core FP32 (the default), tensor cores TF32 x 3 (FP32-accurate)
# and TF32 x 1 (mixed precision), each timed over whole sweeps of the benchmark workload

def gram_pattern(w, p, dev, nsweeps=20):
    import torch
    from paper_2309_08093_gb300 import lib

    stream = torch.cuda.current_stream()
    A = lib.device_tensor(p.storage, "f32", device=dev)
    out = {}
    for name, flags in (("cuda_core_fp32", 0), ("tcgen05_tf32x3", lib.TT_FLAG_TC_GRAM),
                        ("tcgen05_tf32x1", lib.TT_FLAG_TF32_GRAM)):
        ctx = lib.Context(w.dims, p.ranks, w.J, w.lam, p.sketch_seed, "f32", flags=flags)
        cores = lib.device_cores(p.init_cores, device=dev)
        ctx.tt_prox_als_sweep(A, cores, 3, 0, rel_change=False)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.tt_prox_als_sweep(A, cores, nsweeps, 3, rel_change=False)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / nsweeps
        out[name] = {"ms_per_sweep": ms, "sweeps_per_s": 1e3 / ms, "rel_error": ctx.tt_rel_error(A, cores)}
        ctx.close()
    return {"sweeps": nsweeps, "forms": out,
            "note": "sweeps only (no relative error inside the timed region), CUDA events, after 3 warm-up "
                    "sweeps from the workload's initial cores"}


# ---------------------------------------------------------------------------------------------
# fixed draw: the sketches drawn once (TT_FLAG_FIXED_SKETCH) instead of once per sweep (Alg. 1 as
# written); the data sketches then depend on A alone and a call computes them in its first sweep

def fixed_sketch_pattern(w, p, dev, nsweeps=20):
    import torch
    from paper_2309_08093_gb300 import lib

    stream = torch.cuda.current_stream()
    A = lib.device_tensor(p.storage, "f32", device=dev)
    out = {}
    for name, flags in (("redraw_per_sweep", 0), ("fixed_draw", lib.TT_FLAG_FIXED_SKETCH)):
        ctx = lib.Context(w.dims, p.ranks, w.J, w.lam, p.sketch_seed, "f32", flags=flags)
        cores = lib.device_cores(p.init_cores, device=dev)
        warm = lib.device_cores(p.init_cores, device=dev)
        ctx.tt_prox_als_sweep(A, warm, 3, 0, rel_change=False)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.tt_prox_als_sweep(A, cores, nsweeps, 0, rel_change=False)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / nsweeps
        errs, _ = ctx.tt_prox_als_sweep_monitored(A, lib.device_cores(p.init_cores, device=dev), nsweeps, 0)
        out[name] = {"ms_per_sweep": ms, "sweeps_per_s": 1e3 / ms, "rel_error_after": ctx.tt_rel_error(A, cores),
                     "rel_error_per_sweep": [float(e) for e in errs]}
        ctx.close()
    return {"sweeps": nsweeps, "forms": out,
            "note": f"one call of {nsweeps} sweeps from the workload's initial cores, CUDA events (no relative "
                    "error inside the timed call); with the fixed draw the call's first sweep computes the data "
                    "sketches and the later sweeps reuse them; errors per sweep from a second, monitored call"}


# ---------------------------------------------------------------------------------------------
# deterministic mode: the same sweeps with fixed summation orders (TT_FLAG_DETERMINISTIC), timed,
# repeated from the same initial cores, and checked for identical bits

def deterministic_pattern(w, p, dev, nsweeps=5):
    import torch
    from paper_2309_08093_gb300 import lib

    stream = torch.cuda.current_stream()
    A = lib.device_tensor(p.storage, "f32", device=dev)
    runs = []
    for _ in range(2):
        ctx = lib.Context(w.dims, p.ranks, w.J, w.lam, p.sketch_seed, "f32", flags=lib.TT_FLAG_DETERMINISTIC)
        warm = lib.device_cores(p.init_cores, device=dev)
        ctx.tt_prox_als_sweep(A, warm, 1, 500, rel_change=False)
        cores = lib.device_cores(p.init_cores, device=dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.tt_prox_als_sweep(A, cores, nsweeps, 0, rel_change=False)
        e1.record(stream)
        torch.cuda.synchronize()
        err = ctx.tt_rel_error(A, cores)
        runs.append((e0.elapsed_time(e1) / nsweeps, cores, err))
        ctx.close()
    same = all(torch.equal(a, b) for a, b in zip(runs[0][1], runs[1][1])) and runs[0][2] == runs[1][2]
    ms = min(runs[0][0], runs[1][0])
    return {"sweeps_per_s": 1e3 / ms, "ms_per_sweep": ms, "sweeps": nsweeps, "rel_error": runs[0][2],
            "bitwise_identical_runs": same,
            "note": "TT_FLAG_DETERMINISTIC: data sketch with runs summed in index order and flushed in 64-bit "
                    "fixed point (int64 atomics), Gram K-chunks and partial sums in fixed order; sweeps only (no relative error "
                    "inside the timed region), CUDA events; two runs from the same initial cores compared"}


# ---------------------------------------------------------------------------------------------
# the other single-tensor workloads: the order-3 50^3 FP64 workload and the order-5 40^5 workload
# stored FP32 / BF16 / FP8-E4M3 (slice scales), each timed per sweep with its error against the
# FP64 tensor and its data-sketch bandwidth

def workload_pattern(name, storages, dev, nsweeps=None):
    import numpy as np
    import torch
    from paper_2309_08093_gb300 import lib, synth

    w = synth.WORKLOADS[name]
    nsweeps = nsweeps or w.sweeps
    hbm, peak_kind = peaks()
    stream = torch.cuda.current_stream()
    p64 = synth.make_problem(w, storage="f64")
    A64 = lib.device_tensor(p64.storage, "f64", device=dev)
    ctx64 = lib.Context(w.dims, p64.ranks, w.J, w.lam, p64.sketch_seed, "f64")  # errors vs the FP64 tensor
    nrm64 = float(np.linalg.norm(p64.tensor.ravel()))
    forms = {}
    for st in storages:
        flat, scales, exact = synth.quantize(p64.tensor, st)
        delta = float(np.linalg.norm((exact - p64.tensor).ravel()) / nrm64)
        del exact
        ctx = lib.Context(w.dims, p64.ranks, w.J, w.lam, p64.sketch_seed, st)
        A = lib.device_tensor(flat, st, device=dev)
        sd = torch.tensor(scales, device=dev) if scales is not None else None
        warm = lib.device_cores(p64.init_cores, device=dev)
        ctx.tt_prox_als_sweep(A, warm, 2, 1000, scales=sd, rel_change=False)  # plans, tables, kernels
        cores = lib.device_cores(p64.init_cores, device=dev)
        ms, errs, errs64 = [], [], []
        ctx.tt_profile_enable(True)
        for t in range(nsweeps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.tt_prox_als_sweep(A, cores, 1, t, scales=sd, rel_change=False)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
            errs.append(ctx.tt_rel_error(A, cores, scales=sd))  # (the counters record data sketches only)
            errs64.append(ctx64.tt_rel_error(A64, cores))
        prof = ctx.tt_profile_read()
        ctx.tt_profile_enable(False)
        Y = [torch.zeros(w.J * n, device=dev) for n in w.dims]
        ctx.tt_sketch_unfold(A, -1, 5000, Y, scales=sd)
        torch.cuda.synchronize()
        ctx.tt_profile_enable(True)
        for t in range(10):
            ctx.tt_sketch_unfold(A, -1, 5001 + t, Y, scales=sd)
        torch.cuda.synchronize()
        iso = ctx.tt_profile_read()
        ctx.tt_profile_enable(False)
        ctx.close()
        del A, Y

        def gbs(pr):
            n = max(1, pr["unfold_launches"])
            return (pr["unfold_bytes"] / n) / (pr["unfold_ms"] / n * 1e-3) / 1e9, pr["unfold_bytes"] / n

        g_in, bpl = gbs(prof)
        g_iso, _ = gbs(iso)
        sweep_ms = sorted(ms)[len(ms) // 2]
        forms[st] = {"sweeps_per_s": 1e3 / sweep_ms, "ms_per_sweep_median": sweep_ms,
                     "data_sketch": {"bytes_per_launch": bpl, "gbs_in_sweep": g_in, "frac_in_sweep": g_in / hbm,
                                     "gbs_alone": g_iso, "frac_alone": g_iso / hbm, "peak": hbm,
                                     "peak_kind": peak_kind},
                     "quantisation_delta": delta,
                     "rel_error_per_sweep": [round(e, 8) for e in errs],
                     "rel_error_vs_fp64_tensor_per_sweep": [round(e, 8) for e in errs64],
                     "rel_error_vs_fp64_tensor_final": errs64[-1]}
    ctx64.close()
    base = storages[0]
    target = forms[base]["rel_error_vs_fp64_tensor_final"] * (1 + 1e-3)
    for st, r in forms.items():
        hit = next((i + 1 for i, e in enumerate(r["rel_error_vs_fp64_tensor_per_sweep"]) if e <= target), None)
        r["sweeps_to_tolerance"] = hit
        r["sweeps_to_tolerance_per_s"] = (r["sweeps_per_s"] / hit) if hit else None
        r["final_error_minus_baseline"] = r["rel_error_vs_fp64_tensor_final"] - forms[base]["rel_error_vs_fp64_tensor_final"]
    return {"workload": f"{w.name}: {'x'.join(map(str, w.dims))}, TT ranks {list(p64.ranks)}, J={w.J}, "
                        f"lambda={w.lam}, noise={w.noise}, cores {w.core_kind}",
            "sweeps": nsweeps, "baseline_form": base, "tolerance": target, "forms": forms,
            "note": "each sweep timed alone with CUDA events (one tt_prox_als_sweep call, synchronised); errors "
                    "outside the timed sweeps, against the stored tensor and against the FP64 tensor; "
                    "quantisation_delta = ||A_q - A|| / ||A||; data-sketch GB/s from CUDA events around each "
                    "launch (algorithmic bytes: N x bytes per entry, plus n_0 scales for FP8)"}


def bf16_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured"
    except Exception:
        return 1900.0, "fallback"


def gemm_pattern(dev, reps=10):
    """The network's tcgen05 GEMM (C = A B^T, BF16 in, FP32 accumulators in tensor memory) timed
    alone with CUDA events: a large square problem and the warm-start network's training shapes."""
    import torch
    from paper_2309_08093_gb300 import lib

    peak, kind = bf16_peak()
    stream = torch.cuda.current_stream()
    out = {"peak_tflops": peak, "peak_kind": kind, "shapes": {}}
    for M, N, K in [(8192, 8192, 8192), (256, 23232, 512), (23232, 512, 256), (256, 512, 5184)]:
        A = torch.randn(M, K, device=dev).to(torch.bfloat16)
        B = torch.randn(N, K, device=dev).to(torch.bfloat16)
        C = torch.empty(M, N, device=dev)
        for _ in range(3):
            lib.tt_mlp_gemm_bf16(A, B, C, M, N, K, K, K, N, check=False)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            lib.tt_mlp_gemm_bf16(A, B, C, M, N, K, K, K, N, check=False)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        tf = 2.0 * M * N * K / (ms * 1e-3) / 1e12
        out["shapes"][f"{M}x{N}x{K}"] = {"ms": ms, "tflops": tf, "frac": tf / peak}
        del A, B, C
    out["note"] = ("one kernel per call, no split-K (the network splits K for its small-M shapes); "
                   "frac against the measured cuBLAS BF16 burst peak")
    return out


def sparse_pattern(dev, nnz=20_000_000, reps=10):
    """The data sketch of a sparse tensor in coordinate form (tt_sketch_unfold_coo, all four
    modes) on the 100^4 shape at J = 4096: nnz uniformly random coordinates (20% of the entries,
    repeats allowed) with N(0,1) values, seeded, device-resident. One draw (fixed sweep index)
    for all timed calls; each call zeroes the four sketches, runs one kernel and reads the device
    status back (a synchronisation, inside the timed region)."""
    import torch
    from paper_2309_08093_gb300 import lib

    dims, J = (100, 100, 100, 100), 4096
    g = torch.Generator(device=dev)
    g.manual_seed(20230921)
    idx = torch.randint(0, 100, (4, nnz), generator=g, device=dev, dtype=torch.int32)
    val = torch.randn(nnz, generator=g, device=dev)
    ctx = lib.Context(dims, (1, 10, 10, 10, 1), J, 1e-3, 5, "f32")
    Y = [torch.zeros(J * n, device=dev) for n in dims]
    stream = torch.cuda.current_stream()
    for _ in range(3):
        ctx.tt_sketch_unfold_coo(idx, val, nnz, -1, 3, Y)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        ctx.tt_sketch_unfold_coo(idx, val, nnz, -1, 3, Y)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    ctx.close()
    in_bytes = nnz * (4 * 4 + 4)
    return {"shape": "100^4", "nnz": nnz, "J": J, "ms_per_call": ms, "entries_per_s": nnz / (ms * 1e-3),
            "input_gbs": in_bytes / (ms * 1e-3) / 1e9, "atomic_adds_per_s": 4 * nnz / (ms * 1e-3),
            "note": "k_unfold_coo: one thread per entry, four FP32 atomics into L2-resident sketches "
                    "(6.5 MB per mode); input GB/s counts the int32 indices and FP32 values read"}


def window_pattern(dev, reps=10):
    """The data sketch of tensors whose mode-0 fibres are off the 16-byte grid (window staging),
    each mode alone (tt_sketch_unfold, CUDA events, `reps` calls after two warm-up calls): FP32
    with 101-entry fibres (404 bytes, on a 4-byte grid), BF16 with 101-entry fibres (202 bytes,
    on a 2-byte grid), and the FP32 100-entry fibres of the same shape (400 bytes, on the 16-byte
    grid) for comparison. Seeded N(0,1) entries, generated on the device; J = 1024, one draw."""
    import numpy as np
    import torch
    from paper_2309_08093_gb300 import lib

    hbm, hbm_src = peaks()
    cases = [((101, 84, 93, 50), "f32"), ((101, 84, 93, 100), "bf16"), ((100, 84, 93, 50), "f32")]
    stream = torch.cuda.current_stream()
    out = {"peak_gbs": hbm, "peak_source": hbm_src, "cases": []}
    for dims, dt in cases:
        n = int(np.prod(dims))
        g = torch.Generator(device=dev)
        g.manual_seed(20230923)
        a = torch.randn(n, generator=g, device=dev)
        if dt == "bf16":
            a = a.to(torch.bfloat16)
        ctx = lib.Context(dims, (1, 4, 4, 4, 1), 1024, 1e-3, 7, dt)
        Y = [torch.zeros(1024 * m, device=dev) for m in dims]
        nbytes = a.numel() * a.element_size()
        per_mode = []
        for k in range(len(dims)):
            Yk = [None] * len(dims)
            Yk[k] = Y[k]
            for _ in range(2):
                ctx.tt_sketch_unfold(a, k, 0, Yk)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(reps):
                ctx.tt_sketch_unfold(a, k, 0, Yk)
            e1.record(stream)
            torch.cuda.synchronize()
            us = e0.elapsed_time(e1) / reps * 1e3
            gbs = nbytes / us / 1e3
            per_mode.append({"mode": k, "us": us, "gbs": gbs, "frac": gbs / hbm})
        ctx.close()
        del a, Y
        out["cases"].append({"dims": list(dims), "storage": dt, "fibre_bytes": dims[0] * (4 if dt == "f32" else 2),
                             "tensor_mb": nbytes / 1e6, "modes": per_mode})
    out["note"] = ("each call zeroes Y_k and launches one data-sketch kernel; GB/s = tensor bytes / call time; "
                   "frac of the " + hbm_src + " copy peak")
    return out


# ---------------------------------------------------------------------------------------------
# learned-warm-start pattern: the network (summary of the data sketch -> initial cores) trained
# on method-generated solves of the 256 x 256 x 3 x 128 smooth-core family, then held-out tensors
# swept from its cores and from random cores until the error against the noise-free tensor is
# <= 1e-2

WS_SUMMARY_SWEEP = 0  # the summary uses sweep 0's draw (fixed for a fixed seed); the first sweep reuses its plans


def warmstart_pattern(dev, n_train=10240, n_eval=32, p=8, train_sweeps=4, epochs=40, mb=256, group=256,
                      tol=1e-2, max_sweeps=8):
    import numpy as np
    import torch
    from paper_2309_08093_gb300 import lib, synth

    spec = synth.warmstart_spec()
    dims, ranks, J = spec["dims"], spec["ranks"], spec["J"]
    stream = torch.cuda.current_stream()
    ctx = lib.Context(dims, ranks, J, spec["lam"], 1234, "f32")
    n_in, n_out = ctx.tt_ws_summary_dim(p), ctx.tt_ws_core_dim()
    n_train = (n_train + group - 1) // group * group
    X = torch.zeros(n_train, n_in, device=dev)
    T = torch.zeros(n_train, n_out, device=dev)
    S = torch.zeros(n_train, device=dev)
    Y = [torch.zeros(J * n, device=dev) for n in dims]
    bspecs = [{"dims": dims, "ranks": ranks, "J": J, "lam": spec["lam"], "seed": 5000 + i, "dtype": "f32"}
              for i in range(group)]
    batch = lib.Batch(bspecs)
    t0 = time.perf_counter()
    for g0 in range(0, n_train, group):
        As, cores = [], []
        for i in range(g0, g0 + group):
            A, _, init = synth.warmstart_tensor_gpu(spec, 100000 + i, device=dev)
            ctx.tt_sketch_unfold(A, -1, WS_SUMMARY_SWEEP, Y)
            ctx.tt_ws_summary(Y, p, X[i], S[i:i + 1])
            As.append(A)
            cores.append(lib.device_cores(init, device=dev))
        batch.tt_batch_sweep(As, cores, train_sweeps, 0)
        for j, i in enumerate(range(g0, g0 + group)):
            ctx.tt_canonicalize(cores[j])
            ctx.tt_ws_pack(cores[j], S[i:i + 1], T[i])
        del As, cores
    torch.cuda.synchronize()
    datagen_s = time.perf_counter() - t0
    batch.close()
    torch.cuda.empty_cache()

    net = lib.Mlp(n_in, 512, n_out, mb, lr=1e-3)
    net.tt_mlp_set_weights(*[torch.from_numpy(w).to(dev) for w in synth.mlp_init(n_in, 512, n_out, 7)])
    rng = np.random.default_rng(5)
    losses, steps = [], 0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    train_ms = 0.0
    for ep in range(epochs):
        perm = torch.from_numpy(rng.permutation(n_train).astype(np.int32)).to(dev)
        e0.record(stream)
        for b in range(0, n_train - mb + 1, mb):
            net.tt_mlp_train_step(X, T, mb, rows=perm[b:b + mb])
            steps += 1
        e1.record(stream)
        torch.cuda.synchronize()
        train_ms += e0.elapsed_time(e1)
        if ep in (0, epochs - 1):
            losses.append(net.tt_mlp_loss_grads(X, T, mb, rows=perm[:mb]))
    flops_per_step = 2.0 * mb * (net.in_dim * 512 + 512 * 512 + 512 * n_out) * 3 - 2.0 * mb * net.in_dim * 512

    def sweeps(A, Tn, cores, Ygiven=None):
        """Sweeps until the error against the noise-free tensor is <= tol; the first sweep uses
        the given sketches when the warm start already computed them (Y_k do not depend on the
        cores). Returns the sweep count (None if not reached) and the device time of each sweep."""
        errs, ms = [], []
        for t in range(max_sweeps):
            e0.record(stream)
            if t == 0 and Ygiven is not None:
                ctx.tt_prox_als_sweep_sketched(Ygiven, cores, 0)
            else:
                ctx.tt_prox_als_sweep(A, cores, 1, t, rel_change=False)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
            errs.append(ctx.tt_rel_error(Tn, cores))
            if errs[-1] <= tol:
                break
        return (len(errs) if errs[-1] <= tol else None), ms

    res = {"random": [], "warm": []}
    tt = {"random": [], "warm": []}
    sweep_ms, first_ms, init_ms, parts = [], {"random": [], "warm": []}, [], []
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    x1 = torch.zeros(1, n_in, device=dev)
    s1 = torch.zeros(1, device=dev)
    y1 = torch.zeros(1, n_out, device=dev)
    for e in range(n_eval):
        A, Tn, init = synth.warmstart_tensor_gpu(spec, 900000 + e, device=dev)
        h, ms = sweeps(A, Tn, lib.device_cores(init, device=dev))
        res["random"].append(h)
        tt["random"].append(sum(ms) if h else None)
        first_ms["random"].append(ms[0])
        sweep_ms += ms[1:]
        cores = lib.device_cores(init, device=dev)
        ev[0].record(stream)
        ctx.tt_sketch_unfold(A, -1, WS_SUMMARY_SWEEP, Y)
        ev[1].record(stream)
        ctx.tt_ws_summary(Y, p, x1[0], s1)
        ev[2].record(stream)
        net.tt_mlp_forward(x1, 1, y1)
        ev[3].record(stream)
        ctx.tt_ws_unpack(y1[0], s1, cores)
        ev[4].record(stream)
        torch.cuda.synchronize()
        init_ms.append(ev[0].elapsed_time(ev[4]))
        parts.append([ev[i].elapsed_time(ev[i + 1]) for i in range(4)])
        h, ms = sweeps(A, Tn, cores, Ygiven=Y)
        res["warm"].append(h)
        tt["warm"].append(init_ms[-1] + sum(ms) if h else None)
        first_ms["warm"].append(ms[0])
        sweep_ms += ms[1:]
    net.close()
    ctx.close()
    t_sweep = float(np.median(sweep_ms))
    t_init = float(np.median(init_ms))
    out = {"workload": f"{'x'.join(map(str, dims))} FP32, TT ranks {ranks}, cumsum cores, 1% noise, J={J}",
           "train_solves": n_train, "train_sweeps_per_solve": train_sweeps, "datagen_s": datagen_s,
           "summary_width": n_in, "network": f"{n_in} -> 512 -> 512 -> {n_out}, GELU, BF16 tcgen05 GEMMs",
           "train_steps": steps, "minibatch": mb, "train_ms": train_ms,
           "train_tflops": flops_per_step * steps / (train_ms * 1e-3) / 1e12,
           "loss_first_epoch": losses[0], "loss_last_epoch": losses[-1],
           "eval_tensors": n_eval, "tolerance": tol,
           "tolerance_note": "relative error against the noise-free tensor (1% noise: recovered to the noise level)",
           "sweep_ms_median": t_sweep, "warm_init_ms_median": t_init,
           "first_sweep_ms_median": {k: float(np.median(v)) for k, v in first_ms.items()},
           "warm_init_parts_ms": dict(zip(["summary_unfold", "summary", "mlp_forward", "unpack"],
                                          [float(x) for x in np.median(np.array(parts), axis=0)])),
           "note": "warm form: the summary's sketches are the first sweep's data sketches (same draw), so the "
                   "first sweep runs on them (tt_prox_als_sweep_sketched); times are CUDA-event sums per tensor"}
    for k, hits in res.items():
        ok = [h for h in hits if h is not None]
        times = [t for t in tt[k] if t is not None]
        mean_t = float(np.mean(times)) if times else None
        out[k] = {"sweeps_to_tolerance": hits, "mean_sweeps": float(np.mean(ok)) if ok else None,
                  "reached": len(ok), "time_to_tolerance_ms_mean": mean_t,
                  "solves_per_s": (1e3 / mean_t) if mean_t else None}
    return out


# ---------------------------------------------------------------------------------------------
# GPU arm

def main():
    args = parse()
    if args.cpu_sample:
        cpu_sample_main(args)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        reference_main(args, rank, world)
        return

    import numpy as np
    import torch

    if args.only_pattern:
        torch.cuda.set_device(0)
        dev = torch.device("cuda", 0)
        from paper_2309_08093_gb300 import build, synth

        build.build()
        if args.only_pattern == "batched":
            out = batched_pattern(dev)
        elif args.only_pattern == "warmstart":
            out = warmstart_pattern(dev, n_train=args.ws_train)
        elif args.only_pattern == "gemm":
            out = gemm_pattern(dev)
        elif args.only_pattern == "sparse":
            out = sparse_pattern(dev)
        elif args.only_pattern == "order3":
            out = workload_pattern("order3-50-r5", ["f64", "f32"], dev)
        elif args.only_pattern == "order5":
            out = workload_pattern("order5-40-r8", ["f32", "bf16", "fp8"], dev)
        elif args.only_pattern == "gram":
            w = synth.WORKLOADS[args.workload]
            out = gram_pattern(w, synth.make_problem(w, storage="f32"), dev)
        elif args.only_pattern == "window":
            out = window_pattern(dev)
        elif args.only_pattern == "fixed":
            w = synth.WORKLOADS[args.workload]
            out = fixed_sketch_pattern(w, synth.make_problem(w, storage="f32"), dev)
        elif args.only_pattern == "deterministic":
            w = synth.WORKLOADS[args.workload]
            out = deterministic_pattern(w, synth.make_problem(w, storage="f32"), dev)
        else:
            w = synth.WORKLOADS[args.workload]
            out = precision_pattern(w, synth.make_problem(w, storage="f32"), dev, w.sweeps)
        print(json.dumps({"pattern": args.only_pattern, **out}), flush=True)
        return

    dist = None
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    from paper_2309_08093_gb300 import build, lib, synth

    build.build()
    w = synth.WORKLOADS[args.workload]
    storage = args.storage or w.storage
    p = synth.make_problem(w, storage=storage)
    stream = torch.cuda.current_stream()
    ctx = lib.Context(w.dims, p.ranks, w.J, w.lam, p.sketch_seed, storage)
    A = lib.device_tensor(p.storage, storage, device=dev)
    scales = torch.tensor(p.scales, device=dev) if p.scales is not None else None
    cores = lib.device_cores(p.init_cores, device=dev)

    # A step is one sweep of Algorithm 1, then the relative error of the updated cores. The K
    # steps are one tt_prox_als_sweep_monitored call: the sweeps run back to back with the error
    # after each, and the errors come back with one synchronisation (measured 756 us per step,
    # against 771 us for a sweep call and an error call per step, each ending in a host round trip).
    def steps(first, k):
        errs, _ = ctx.tt_prox_als_sweep_monitored(A, cores, k, first, scales=scales)
        return errs[-1] if len(errs) else None

    steps(0, args.warmup)
    torch.cuda.synchronize()

    gpu_id = torch.cuda.get_device_properties(dev).uuid
    gpu_id = "GPU-" + str(gpu_id) if not str(gpu_id).startswith("GPU-") else str(gpu_id)
    clocks = ClockSampler(gpu_id)
    ctx.tt_profile_enable(True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_wall0 = time.time()
    e0.record(stream)
    err = steps(args.warmup, args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    t_wall1 = time.time()
    if dist:
        dist.barrier()
    prof = ctx.tt_profile_read()
    ctx.tt_profile_enable(False)
    # the same data-sketch kernels alone (no concurrent chain kernels), after the timed region
    Yiso = [torch.zeros(w.J * n, device=dev) for n in w.dims]
    for t in range(2):
        ctx.tt_sketch_unfold(A, -1, 10_000 + t, Yiso, scales=scales)
    torch.cuda.synchronize()
    ctx.tt_profile_enable(True)
    for t in range(10):
        ctx.tt_sketch_unfold(A, -1, 10_002 + t, Yiso, scales=scales)
    torch.cuda.synchronize()
    prof_iso = ctx.tt_profile_read()
    ctx.tt_profile_enable(False)
    del Yiso
    clocks.stop()
    clk = clocks.summary(t_wall0, t_wall1)
    ms = max_over_ranks(e0.elapsed_time(e1), dist, dev)
    sweeps_per_s = replica_throughput(world, args.steps, ms)

    hbm, peak_kind = peaks()
    unfold_avg_ms = prof["unfold_ms"] / max(1, prof["unfold_launches"])
    bytes_per_launch = prof["unfold_bytes"] / max(1, prof["unfold_launches"])
    achieved = bytes_per_launch / (unfold_avg_ms * 1e-3) / 1e9
    mode_gbs = [(bytes_per_launch / (m / n * 1e-3) / 1e9) if n else None
                for m, n in zip(prof["mode_ms"], prof["mode_launches"])]

    iso_ms = prof_iso["unfold_ms"] / max(1, prof_iso["unfold_launches"])
    iso_bytes = prof_iso["unfold_bytes"] / max(1, prof_iso["unfold_launches"])
    iso_ach = iso_bytes / (iso_ms * 1e-3) / 1e9
    iso = {"kernel": "data sketch kernels alone (tt_sketch_unfold, all modes, 10 draws, after the timed region)",
           "bound": "hbm", "achieved": iso_ach, "peak": hbm, "unit": "GB/s", "frac": iso_ach / hbm,
           "avg_launch_ms": iso_ms, "bytes_per_launch": iso_bytes,
           "per_mode_gbs": [(iso_bytes / (m / n * 1e-3) / 1e9) if n else None
                            for m, n in zip(prof_iso["mode_ms"], prof_iso["mode_launches"])]}
    line = None
    if rank == 0:
        line = {"metric": METRIC, "value": sweeps_per_s, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": storage, "data": "synthetic",
                "config": workload_config(w, storage),
                "rel_error_after": err,
                "roofline": {"kernel": "data sketch (k_unfold_gather mode 0 + k_unfold_cols modes >= 1)",
                             "bound": "hbm",
                             "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                             "peak_kind": peak_kind,
                             "traffic": UNFOLD_TRAFFIC.get((args.workload, storage)),
                             "traffic_note": "dram__bytes_read.sum + dram__bytes_write.sum per launch, mean over the "
                                             "four modes of one sweep (in-sweep launch shapes), from one ncu capture of "
                                             "these kernel versions; null for workloads not captured",
                             "bytes_per_launch": bytes_per_launch, "avg_launch_ms": unfold_avg_ms,
                             "per_mode_gbs": mode_gbs,
                             "share_of_step": prof["unfold_ms"] / ms,
                             "note": "CUDA events around every data-sketch launch in the timed region; the sweep "
                                     "runs these kernels on a side stream concurrently with the chain kernels, so "
                                     "their durations include that sharing (see roofline_isolated)"},
                "roofline_isolated": iso,
                "gpu_launches": prof["kernel_launches"],
                "clocks": clk}
    # end-to-end through the host-buffer entry point (pinned host memory)
    if rank == 0 and not args.no_e2e:
        A_h = torch.from_numpy(np.ascontiguousarray(p.storage)).pin_memory().numpy() if storage != "bf16" else \
            torch.from_numpy(np.ascontiguousarray(p.storage.view(np.int16))).pin_memory().numpy()
        cores_h = [torch.from_numpy(np.ascontiguousarray(np.asarray(g, np.float32).ravel(order="F"))).pin_memory().numpy()
                   for g in p.init_cores]
        sc_h = np.ascontiguousarray(p.scales, dtype=np.float32) if p.scales is not None else None
        ne = max(3, min(40, args.steps))
        ctx.tt_prox_als_sweep_host(A_h, cores_h, 1, 0, scales_host=sc_h)  # warm (allocates staging)
        # warm the asynchronous path too (its copy stream, events and buffers); its output arrays
        # stay referenced until the synchronisation
        warm = [ctx.tt_prox_als_sweep_host_async(A_h, cores_h, 1, 0, scales_host=sc_h) for _ in range(3)]
        ctx.tt_host_sync()
        del warm
        # one asynchronous call per step: each copies the step's tensor and cores in, sweeps, takes
        # the relative error and copies the cores and the error out; the next step's tensor copy
        # runs beside this step's sweep. One synchronisation at the end of the timed steps.
        t0 = time.perf_counter()
        outs = [ctx.tt_prox_als_sweep_host_async(A_h, cores_h, 1, t + 1, scales_host=sc_h) for t in range(ne)]
        ctx.tt_host_sync()
        e2e_s = (time.perf_counter() - t0) / ne
        assert all(np.isfinite(o[1][0]) for o in outs)
        # the same steps as synchronous calls (copy in, sweep, error, copy out, wait)
        t0 = time.perf_counter()
        for t in range(ne):
            ctx.tt_prox_als_sweep_host(A_h, cores_h, 1, ne + t + 1, scales_host=sc_h)
        sync_s = (time.perf_counter() - t0) / ne
        core_bytes = sum(int(g.size) * 4 for g in cores_h)
        line["e2e"] = {"value": 1.0 / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(A_h.nbytes) + core_bytes
                       + (int(sc_h.nbytes) if sc_h is not None else 0),
                       "d2h_bytes_per_step": core_bytes + 8 + 16 + 4,
                       "synchronous_call_value": 1.0 / sync_s,
                       "note": f"{ne} tt_prox_als_sweep_host_async calls from page-locked host memory (each: H2D "
                               "copy of the tensor and cores, one sweep, the relative error, D2H of the cores, "
                               "the error sums and the status), then tt_host_sync; wall clock. The tensor copy of "
                               "a step runs beside the previous step's sweep. synchronous_call_value: the same "
                               "steps as tt_prox_als_sweep_host calls, each waiting for its results"}
    ctx.close()
    if rank == 0 and world == 1 and not args.no_patterns and storage == "f32":
        line["patterns"] = {"precision": precision_pattern(w, p, dev, w.sweeps)}
        torch.cuda.empty_cache()
        line["patterns"]["batched"] = batched_pattern(dev)
        torch.cuda.empty_cache()
        line["patterns"]["warmstart"] = warmstart_pattern(dev, n_train=args.ws_train)
        torch.cuda.empty_cache()
        line["patterns"]["gemm"] = gemm_pattern(dev)
        line["patterns"]["sparse"] = sparse_pattern(dev)
        torch.cuda.empty_cache()
        line["patterns"]["order3"] = workload_pattern("order3-50-r5", ["f64", "f32"], dev)
        line["patterns"]["order5"] = workload_pattern("order5-40-r8", ["f32", "bf16", "fp8"], dev)
        torch.cuda.empty_cache()
        line["patterns"]["deterministic"] = deterministic_pattern(w, p, dev)
        line["patterns"]["gram"] = gram_pattern(w, p, dev)
        torch.cuda.empty_cache()
        line["patterns"]["window"] = window_pattern(dev)
        line["patterns"]["fixed"] = fixed_sketch_pattern(w, p, dev)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            res = run_cpu_child(["--workload", args.workload] + (["--storage", args.storage] if args.storage else []))
            line["cpu_baseline"] = {
                "value": 1.0 / res["sweep_all_cores_s"], "unit": UNIT, "cores": res["cores"], "kind": "oracle",
                "sample": (f"one oracle sweep (Algorithm 1 outer iteration, FP64 numpy) on the same workload: its "
                           f"data-sketch columns by definition spread over {res['cores']} single-threaded "
                           f"processes (one per core of os.sched_getaffinity; {res['sketch_wall_s']:.2f} s wall "
                           f"for {res['sketch_busy_s']:.2f} s of column work), plus the rest of the sweep serial "
                           f"({res['serial_rest_s']:.2f} s: the one-thread sweep minus its "
                           f"{res['sketch_one_thread_s']:.2f} s of data-sketch columns)"),
                "one_thread": {"value": 1.0 / res["sweep_s"], "unit": UNIT, "cores": 1,
                               "sample": "one full oracle sweep, FP64 numpy, 1 thread, timed once"}}
        except Exception as e:  # report, do not hide
            line["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle",
                                    "sample": f"failed: {str(e)[-200:]}"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
