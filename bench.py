"""Benchmark of the Fast Count Sketch hot path on GB300.

Default workload (one step): CP-route FCS of one order-3 CP tensor,
I_n = 1000, rank R = 100, factors N(0,1), weights U(0.5, 1.5), J_n = 5000
(Jt = 14998, FFT length 16384), D = 10 independent sketches -- the hash
tables are generated on the device (fcs_make_hashes) and the sketches
computed (fcs_sketch_cp).  Throughput unit: sketches/s (one sketch = one
FCS_d vector of length Jt, so a step yields D sketches).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl fcs|reference]

N > 1 runs under torch.distributed.run as independent replicas (the path has
no exchange step); `value` is the sketches all ranks produced divided by the
slowest rank's time.  `--impl reference` times the FP64 CPU oracle on the host
cores on a bounded sample of the same workload (rank 0 only).

Prints one JSON line.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

WORKLOAD = {"workload": "cp_fcs_order3_I1000_R100_J5000_D10", "order": 3,
            "I": 1000, "R": 100, "J": 5000, "D": 10, "seed": 2}
METRIC = "FCS sketches/s (CP route, order 3, I=1000, R=100, J=5000, D=10)"
L2_FLUSH_BYTES = 256 << 20


def jt_of(w):
    return w["order"] * w["J"] - w["order"] + 1


def fft_len(jt):
    return 1 << max(4, math.ceil(math.log2(jt)))


def cp_flops(w):
    """Algorithmic flops of one fcs_sketch_cp launch: 2.5 P log2 P per real
    FFT of length P (D*R*N forward + D inverse) plus the pointwise mode
    products and rank accumulation (6 flops per complex multiply, 4 per
    real-weighted complex accumulate) over P/2+1 bins."""
    N, R, D = w["order"], w["R"], w["D"]
    P = fft_len(jt_of(w))
    fft = D * (R * N + 1) * 2.5 * P * math.log2(P)
    pointwise = D * R * (P // 2 + 1) * (6 * (N - 1) + 4)
    return fft + pointwise


def cp_bytes(w):
    """Algorithmic bytes of one step: factors and weights read once, hash
    tables written once (by fcs_make_hashes) and read once, sketches
    written once."""
    N, I, R, D = w["order"], w["I"], w["R"], w["D"]
    return N * I * R * 4 + R * 4 + 2 * D * N * I * 5 + D * jt_of(w) * 4


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clock / throttle-reason sampling during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.15)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k, v in enumerate(r[2])
                          if v.lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


# ------------------------------------------------------------------ CPU oracle
def oracle_sample(w, budget_s: float = 12.0):
    """Time the FP64 oracle (CP route by direct convolution) on a bounded
    sample of the workload: sketch d = 0 over the first R_s ranks, R_s grown
    until about `budget_s` seconds.  Returns (sketches/s, R_s, seconds)."""
    import oracle
    N, I, R, J = w["order"], w["I"], w["R"], w["J"]
    U, lam = synth.cp_factors(w["seed"], [I] * N, R)
    h, s = oracle.make_hashes(w["seed"], [I] * N, [J] * N, 1)
    Ud = [u.astype(np.float64) for u in U]
    lamd = lam.astype(np.float64)
    rs, spent = 1, 0.0
    while True:
        t0 = time.perf_counter()
        oracle.fcs_cp([u[:, :rs] for u in Ud], lamd[:rs], [J] * N, h, s)
        dt = time.perf_counter() - t0
        if dt * 2 > budget_s or rs >= R:
            spent = dt
            break
        rs = min(R, max(rs + 1, int(rs * budget_s / max(dt, 1e-3) / 3)))
    per_sketch = dt * R / rs
    return 1.0 / per_sketch, rs, spent


def omp_threads():
    v = os.environ.get("OMP_NUM_THREADS")
    if v and v.isdigit():
        return int(v)
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ------------------------------------------------------------------ arms
def run_reference(args, rank, world):
    """The oracle timed as the reference arm: each step computes one rank's
    contribution to one sketch (CS of three columns, two direct FP64
    convolutions); throughput scales that to sketches/s."""
    import oracle
    if rank != 0:
        return None
    w = WORKLOAD
    N, I, R, J = w["order"], w["I"], w["R"], w["J"]
    U, lam = synth.cp_factors(w["seed"], [I] * N, R)
    h, s = oracle.make_hashes(w["seed"], [I] * N, [J] * N, 1)
    Ud = [u.astype(np.float64) for u in U]
    lamd = lam.astype(np.float64)

    def step(k):
        r = k % R
        oracle.fcs_cp([u[:, r:r + 1] for u in Ud], lamd[r:r + 1], [J] * N, h, s)

    for k in range(args.warmup):
        step(k)
    t0 = time.perf_counter()
    for k in range(args.steps):
        step(k)
    dt = time.perf_counter() - t0
    ms = dt * 1e3 / args.steps
    value = (args.steps / R) / dt
    cores = omp_threads()
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "sketches/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(WORKLOAD, Jt=jt_of(w), fft_len=fft_len(jt_of(w)),
                       parallelism="cpu oracle"),
        "cpu_baseline": {"value": value, "unit": "sketches/s", "cores": cores,
                         "kind": "oracle",
                         "sample": f"each step: one rank's term of sketch d=0 "
                                   f"(3 count sketches + 2 direct FP64 convolutions), "
                                   f"{args.steps} steps = {args.steps / R:.2f} sketches"},
        "e2e": {"value": value, "unit": "sketches/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }


def run_fcs(args, rank, world, local_rank):
    import torch
    import paper_2106_13062_gb300 as fcs

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    w = WORKLOAD
    N, I, R, J, D = w["order"], w["I"], w["R"], w["J"], w["D"]
    Is, Js = [I] * N, [J] * N
    Jt = jt_of(w)
    U, lam = synth.cp_factors(w["seed"], Is, R)
    ctx = fcs.Context(local_rank)
    Ug = [torch.from_numpy(u).to(dev) for u in U]
    lamg = torch.from_numpy(lam).to(dev)
    out = torch.empty((D, Jt), dtype=torch.float32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(seed):
        h, s = fcs.fcs_make_hashes(ctx, seed, Is, Js, D)
        fcs.fcs_sketch_cp(ctx, Ug, lamg, Js, h, s, out=out)

    for k in range(args.warmup):
        step(w["seed"] + k)
    torch.cuda.synchronize()

    # ---- device-resident timed region
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sampler = ClockSampler(local_rank)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler.start()
    for k in range(args.steps):
        flush.zero_()                                    # L2 flush, untimed
        e0, e1, e2 = ev[k]
        e0.record(stream)
        h, s = fcs.fcs_make_hashes(ctx, w["seed"] + k, Is, Js, D)
        e1.record(stream)
        fcs.fcs_sketch_cp(ctx, Ug, lamg, Js, h, s, out=out)
        e2.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    if world > 1:
        torch.distributed.barrier()
    step_ms = [a.elapsed_time(c) for a, b, c in ev]
    cp_ms = [b.elapsed_time(c) for a, b, c in ev]
    total_ms = sum(step_ms)

    # ---- end to end through the C ABI with host buffers
    Uh = [torch.from_numpy(u).pin_memory() for u in U]
    lamh = torch.from_numpy(lam).pin_memory()
    outh = torch.empty((D, Jt), dtype=torch.float32).pin_memory()
    e2e_steps = max(3, min(args.steps, 200))
    eev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(e2e_steps)]
    Ud2 = [torch.empty_like(u) for u in Ug]
    lam2 = torch.empty_like(lamg)
    torch.cuda.synchronize()
    for k in range(e2e_steps):
        flush.zero_()
        a, b = eev[k]
        a.record(stream)
        for dst, src in zip(Ud2, Uh):
            dst.copy_(src, non_blocking=True)
        lam2.copy_(lamh, non_blocking=True)
        h, s = fcs.fcs_make_hashes(ctx, w["seed"] + k, Is, Js, D)
        fcs.fcs_sketch_cp(ctx, Ud2, lam2, Js, h, s, out=out)
        outh.copy_(out, non_blocking=True)
        b.record(stream)
    torch.cuda.synchronize()
    e2e_ms = sum(a.elapsed_time(b) for a, b in eev) / e2e_steps
    h2d = sum(u.numel() * 4 for u in Uh) + lamh.numel() * 4
    d2h = outh.numel() * 4

    # correctness guard on the last device-timed output: finite values
    if not torch.isfinite(out).all():
        raise RuntimeError("non-finite sketch output")

    # ---- max over ranks
    tmax = total_ms
    if world > 1:
        t = torch.tensor([total_ms, e2e_ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        tmax, e2e_ms = float(t[0]), float(t[1])
    ctx.close()
    if rank != 0:
        return None

    ms_per_step = tmax / args.steps
    value = world * D * args.steps / (tmax / 1e3)
    props = torch.cuda.get_device_properties(local_rank)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak = props.multi_processor_count * 128 * 2 * sm_mhz * 1e6 / 1e12  # TFLOP/s
    cp_avg_ms = statistics.mean(cp_ms)
    achieved = cp_flops(w) / (cp_avg_ms / 1e3) / 1e12
    roof = {"kernel": "cp_kernel (fcs_sketch_cp)", "bound": "alu",
            "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
            "frac": achieved / fp32_peak, "traffic": None,
            "peak_source": f"derived: {props.multi_processor_count} SMs x 128 FP32 lanes "
                           f"x 2 flop x {sm_mhz:.0f} MHz",
            "flops_per_launch": cp_flops(w), "avg_launch_ms": cp_avg_ms,
            "hbm_gbs_algorithmic": cp_bytes(w) / (cp_avg_ms / 1e3) / 1e9}
    res = {
        "impl": "fcs", "metric": METRIC, "value": value, "unit": "sketches/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(WORKLOAD, Jt=Jt, fft_len=fft_len(Jt),
                       parallelism=f"replicas x{world}" if world > 1 else "single GPU",
                       l2="flushed between timed steps (256 MiB write)"),
        "roofline": roof,
        "e2e": {"value": world * D / (e2e_ms / 1e3), "unit": "sketches/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": e2e_ms},
        "gpu_launches": 2 * args.steps,
        "clocks": clocks,
    }
    if world == 1 and not args.no_cpu_baseline:
        v, rs, secs = oracle_sample(w)
        res["cpu_baseline"] = {"value": v, "unit": "sketches/s", "cores": omp_threads(),
                               "kind": "oracle",
                               "sample": f"sketch d=0 over the first {rs} of {R} ranks "
                                         f"({secs:.1f} s), scaled to one sketch"}
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["fcs", "reference"], default="fcs")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        # the CPU oracle runs on rank 0 only; other ranks exit without work
        res = run_reference(args, rank, world)
        if res is not None:
            print(json.dumps(res), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    res = run_fcs(args, rank, world, local_rank)
    if res is not None:
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
