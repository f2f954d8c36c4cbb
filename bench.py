"""Benchmark of the Fast Count Sketch hot path on GB300.

Default workload `cp` (one step): CP-route FCS of one order-3 CP tensor,
I_n = 1000, rank R = 100, factors N(0,1), weights U(0.5, 1.5), J_n = 5000
(Jt = 14998, FFT length 16384), D = 10 independent sketches -- one call of
fcs_sketch_cp_seeded generates the step's hash tables on the device (in the
factor-transpose launch) and computes the sketches.  Unit: sketches/s (one sketch = one FCS_d vector of length
Jt, so a step yields D sketches).

With N = 1 the default line also carries the metric's other parts as
sub-results under the keys `dense`, `kron`, `batch` and `serve` (skip them with
--no-extra); each has its own roofline, clock record, end-to-end leg and CPU
baseline (serve: capacity, p50/p99 latency and an accuracy check of served
results against direct calls).

Workloads (`--workload`; the default line is `cp`):
  dense  the robust-tensor-power-method step: dense-route FCS of a symmetric
         500^3 FP32 tensor (rank 10, noise 0.01), J_n = 2000, D = 5, then
         T(u,u,u) and T(I,u,u) for 64 unit vectors with the median over D.
  kron   Kronecker compression: 32 pairs of 512x512 matrices, order-4 hashes
         J_n = 1024, D = 10; sketch every A and B (dense route, batched),
         combine FCS(A o B) by FFT, recover 2^20 sampled entries per pair.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl fcs|reference]
                    [--workload cp|dense|kron]

N > 1 runs under torch.distributed.run as independent replicas (the path has
no exchange step); `value` is the sketches all ranks produced divided by the
slowest rank's time.  `--impl reference` times the FP64 CPU oracle on the host
cores on a bounded sample of the same workload (rank 0 only).

Prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
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

L2_FLUSH_BYTES = 256 << 20
CSRC = os.path.join(ROOT, "paper_2106_13062_gb300", "csrc")


def fft_len(jt):
    return 1 << max(4, math.ceil(math.log2(jt)))


def jt_of(J):
    return int(sum(J) - len(J) + 1)


def sources_digest(files):
    """sha256 over the kernel's source files (to tell whether an ncu capture
    still describes the current kernel)."""
    hsh = hashlib.sha256()
    for f in files:
        with open(os.path.join(CSRC, f), "rb") as fh:
            hsh.update(fh.read())
    return hsh.hexdigest()[:16]


def profiled_traffic(profile_name, files):
    """DRAM bytes per launch from a committed ncu summary, or None when the
    summary is absent or the kernel's sources changed since the capture."""
    path = os.path.join(ROOT, "profiles", profile_name)
    try:
        text = open(path).read()
    except OSError:
        return None
    m1 = re.search(r"dram_bytes_per_launch\s*=\s*([0-9.eE+]+)", text)
    m2 = re.search(r"sources_sha256\s*=\s*([0-9a-f]+)", text)
    if not (m1 and m2) or m2.group(1) != sources_digest(files):
        return None
    return float(m1.group(1))


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


def omp_threads():
    v = os.environ.get("OMP_NUM_THREADS")
    if v and v.isdigit():
        return int(v)
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# ================================================================== workloads
class CpWorkload:
    """Order-3 CP tensor, I_n = 1000, R = 100, J_n = 5000, D = 10."""
    name = "cp_fcs_order3_I1000_R100_J5000_D10"
    metric = "FCS sketches/s (CP route, order 3, I=1000, R=100, J=5000, D=10)"
    N, I, R, J, D, seed = 3, 1000, 100, 5000, 10, 2

    def __init__(self):
        self.Is, self.Js = [self.I] * self.N, [self.J] * self.N
        self.Jt = jt_of(self.Js)
        self.P = fft_len(self.Jt)

    def config(self):
        return {"workload": self.name, "order": self.N, "I": self.I, "R": self.R,
                "J": self.J, "D": self.D, "Jt": self.Jt, "fft_len": self.P,
                "seed": self.seed}

    def sketches_per_step(self):
        return self.D

    def launches_per_step(self):
        return 2                     # prep (transpose, clear, hash tables), sketch kernel

    def flops(self):
        """2.5 P log2 P per real FFT of length P (D*R*N forward + D inverse)
        plus the pointwise mode products and rank sum (6 flops per complex
        multiply, 2 per complex add) over P/2+1 bins."""
        P = self.P
        fft = self.D * (self.R * self.N + 1) * 2.5 * P * math.log2(P)
        pointwise = self.D * self.R * (P // 2 + 1) * (6 * (self.N - 1) + 2)
        return fft + pointwise

    def bytes(self):
        """Factors and weights read once, hash tables (int32 + int8) read
        once, sketches written once."""
        return (self.N * self.I * self.R * 4 + self.R * 4 +
                self.D * self.N * self.I * 5 + self.D * self.Jt * 4)

    # -- device
    def setup(self, fcs, ctx, dev):
        import torch
        U, lam = synth.cp_factors(self.seed, self.Is, self.R)
        self.host = {"U": U, "lam": lam}
        self.Ug = [torch.from_numpy(u).to(dev) for u in U]
        self.lamg = torch.from_numpy(lam).to(dev)
        self.out = torch.empty((self.D, self.Jt), dtype=torch.float32, device=dev)
        self.h = torch.empty((self.D, self.N * self.I), dtype=torch.int32, device=dev)
        self.s = torch.empty((self.D, self.N * self.I), dtype=torch.int8, device=dev)
        self.fcs, self.ctx, self.dev = fcs, ctx, dev

    def step(self, k, marks):
        # one library call: the hash tables of this step's seed (written by
        # the factor-transpose launch) and the sketch
        marks("cp_kernel")
        self.fcs.fcs_sketch_cp_seeded(self.ctx, self.Ug, self.lamg, self.Js, self.D, self.seed + k,
                                      out=self.out, h=self.h, s=self.s)
        marks(None)

    def e2e_prepare(self):
        """Inputs staged as one pinned host buffer [U_1 | ... | U_N | lambda]
        whose views go to fcs_sketch_cp_host (the library merges the adjacent
        ranges into one copy), output into a pinned host buffer."""
        import torch
        parts = [u.reshape(-1) for u in self.host["U"]] + [self.host["lam"]]
        self.inh = torch.from_numpy(np.concatenate(parts)).pin_memory()
        offs = np.cumsum([0] + [p.size for p in parts])
        self.Uh = [self.inh[offs[n]:offs[n + 1]].view(self.I, self.R) for n in range(self.N)]
        self.lamh = self.inh[offs[self.N]:offs[self.N + 1]]
        self.outh = torch.empty((self.D, self.Jt), dtype=torch.float32).pin_memory()
        return self.inh.numel() * 4, self.outh.numel() * 4

    def e2e_step(self, k):
        """One library call with host buffers: copies in, hash tables from
        the seed, the sketch, and the copy out, all on the current stream."""
        self.fcs.fcs_sketch_cp_host(self.ctx, self.Uh, self.lamh, self.Js, self.D,
                                    self.seed + k, out=self.outh)

    def check(self):
        import torch
        return bool(torch.isfinite(self.out).all())

    def roofline(self, times_ms, props):
        t = statistics.mean(times_ms["cp_kernel"])
        sm_mhz = float(measured_peaks().get("sm_max_mhz", 2070.0))
        peak = props.multi_processor_count * 128 * 2 * sm_mhz * 1e6 / 1e12
        ach = self.flops() / (t / 1e3) / 1e12
        files = ["fcs_cp.cu", "fcs_cp_run.cuh", "fcs_fft.cuh", "fcs_hash.cuh", "fcs_internal.cuh"]
        return {"kernel": "cp13_kernel (fcs_sketch_cp_seeded: prep launch with the hash "
                          "tables + fused sketch)",
                "bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak,
                "traffic": profiled_traffic("cp_kernel_order3_I1000_R100_J5000_D10.txt", files),
                "peak_source": f"derived: {props.multi_processor_count} SMs x 128 FP32 lanes "
                               f"x 2 flop/FMA x {sm_mhz:.0f} MHz (recipe unit counts, max clock)",
                "flops_per_launch": self.flops(), "avg_launch_ms": t,
                "hbm_gbs_algorithmic": self.bytes() / (t / 1e3) / 1e9}

    # -- oracle
    def oracle_sample(self, budget_s=12.0):
        """FP64 oracle (direct convolutions) on whole sketches d = 0, 1, ...
        until about budget_s seconds have been spent."""
        import oracle
        U, lam = synth.cp_factors(self.seed, self.Is, self.R)
        h, s = oracle.make_hashes(self.seed, self.Is, self.Js, self.D)
        Ud = [u.astype(np.float64) for u in U]
        lamd = lam.astype(np.float64)
        t0 = time.perf_counter()
        done = 0
        while done < self.D:
            oracle.fcs_cp(Ud, lamd, self.Js, h[done:done + 1], s[done:done + 1])
            done += 1
            if time.perf_counter() - t0 > budget_s:
                break
        dt = time.perf_counter() - t0
        return done / dt, f"{done} whole sketch(es) (d = 0..{done - 1}, all {self.R} ranks), {dt:.1f} s"

    def reference_setup(self):
        import oracle
        U, lam = synth.cp_factors(self.seed, self.Is, self.R)
        self.rh, self.rs = oracle.make_hashes(self.seed, self.Is, self.Js, 1)
        self.rU = [u.astype(np.float64) for u in U]
        self.rlam = lam.astype(np.float64)

    def reference_step(self, k):
        """One rank's term of sketch d = 0 (three count sketches and two direct
        FP64 convolutions); R such steps make one sketch."""
        import oracle
        r = k % self.R
        oracle.fcs_cp([u[:, r:r + 1] for u in self.rU], self.rlam[r:r + 1], self.Js,
                      self.rh, self.rs)
        return 1.0 / self.R

    reference_sample = "each step: one rank's term of sketch d=0 (3 count sketches + 2 direct FP64 convolutions); R steps = 1 sketch"


class DenseWorkload:
    """Robust tensor power method step: 500^3, J_n = 2000, D = 5, B = 64."""
    name = "rtpm_step_dense_order3_I500_J2000_D5_B64"
    metric = "FCS sketches/s (dense route 500^3, J=2000, D=5, + T(u,u,u), T(I,u,u) for 64 u)"
    N, I, J, D, B, seed = 3, 500, 2000, 5, 64, 3

    def __init__(self):
        self.Is, self.Js = [self.I] * self.N, [self.J] * self.N
        self.Jt = jt_of(self.Js)
        self.P = fft_len(self.Jt)

    def config(self):
        return {"workload": self.name, "order": self.N, "I": self.I, "J": self.J,
                "D": self.D, "vectors": self.B, "Jt": self.Jt, "fft_len": self.P,
                "tensor": "symmetric rank 10, weights 10..1, noise sigma 0.01",
                "contractions": "fcs_contract_both: T(u,u,u) and T(I,u,u) from one set of "
                                "transforms",
                "seed": self.seed}

    def sketches_per_step(self):
        return self.D

    def launches_per_step(self):
        # hashes, zero + dense, spectrum, fused contraction, 2 medians
        return 1 + 2 + 1 + 1 + 2

    def bytes(self):
        """Dense kernel: the tensor read once, tables read once, sketches
        written once."""
        return self.I ** 3 * 4 + self.D * self.N * self.I * 5 + self.D * self.Jt * 4

    def setup(self, fcs, ctx, dev):
        import torch
        T, _, _ = synth.rtpm_tensor(self.seed, I=self.I, R=10, sigma=0.01)
        u = synth.unit_vectors(self.seed + 1, self.B, self.I)
        self.host = {"T": T, "u": u}
        self.Tg = torch.from_numpy(T).to(dev)
        self.ug = torch.from_numpy(u).to(dev)
        self.fT = torch.empty((self.D, self.Jt), dtype=torch.float32, device=dev)
        self.fcs, self.ctx, self.dev = fcs, ctx, dev

    def step(self, k, marks, T=None, u=None):
        fcs = self.fcs
        T = self.Tg if T is None else T
        u = self.ug if u is None else u
        h, s = fcs.fcs_make_hashes(self.ctx, self.seed + k, self.Is, self.Js, self.D)
        marks("dense_kernel")
        fcs.fcs_sketch_dense(self.ctx, T, self.Js, h, s, out=self.fT)
        marks("contract")
        # T(u,u,u) and T(I,u,u) from one set of transforms
        a, b = fcs.fcs_contract_both(self.ctx, self.fT, [u, u, u], self.Is, self.Js, h, s,
                                     free_mode=0)
        marks(None)
        return a, b

    def e2e_prepare(self):
        import torch
        self.Th = torch.from_numpy(self.host["T"]).pin_memory()
        self.uh = torch.from_numpy(self.host["u"]).pin_memory()
        self.Td = torch.empty_like(self.Tg)
        self.ud = torch.empty_like(self.ug)
        self.ah = torch.empty((self.B,), dtype=torch.float32).pin_memory()
        self.bh = torch.empty((self.B, self.I), dtype=torch.float32).pin_memory()
        return (self.Th.numel() * 4 + self.uh.numel() * 4,
                self.ah.numel() * 4 + self.bh.numel() * 4)

    def e2e_step(self, k):
        self.Td.copy_(self.Th, non_blocking=True)
        self.ud.copy_(self.uh, non_blocking=True)
        a, b = self.step(k, lambda _: None, T=self.Td, u=self.ud)
        self.ah.copy_(a, non_blocking=True)
        self.bh.copy_(b, non_blocking=True)

    def check(self):
        import torch
        return bool(torch.isfinite(self.fT).all())

    def roofline(self, times_ms, props):
        t = statistics.mean(times_ms["dense_kernel"])
        peak = float(measured_peaks().get("hbm_gbs", 6787.6))
        ach = self.bytes() / (t / 1e3) / 1e9
        files = ["fcs_dense.cu", "fcs_internal.cuh"]
        return {"kernel": "dense_kernel (fcs_sketch_dense, incl. output zeroing)",
                "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                "frac": ach / peak,
                "traffic": profiled_traffic("dense_kernel_rtpm_I500_J2000_D5.txt", files),
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy)",
                "bytes_per_launch": self.bytes(), "avg_launch_ms": t,
                "contract_ms": statistics.mean(times_ms["contract"])}

    def oracle_sample(self, budget_s=12.0):
        """FP64 oracle dense route on leading slabs T[0:k] (all D sketches),
        scaled by I/k to one step's sketches."""
        import oracle
        T, _, _ = synth.rtpm_tensor(self.seed, I=self.I, R=10, sigma=0.01)
        h, s = oracle.make_hashes(self.seed, self.Is, self.Js, self.D)
        k = 10
        while True:
            t0 = time.perf_counter()
            sub = T[:k]
            hs = np.concatenate([h[:, :k], h[:, self.I:]], axis=1)
            ss = np.concatenate([s[:, :k], s[:, self.I:]], axis=1)
            oracle.fcs_dense(sub, self.Js, hs, ss)
            dt = time.perf_counter() - t0
            if dt > budget_s / 4 or k >= self.I:
                break
            k = min(self.I, k * 4)
        per_step = dt * self.I / k
        return self.D / per_step, f"dense route on slabs T[0:{k}] of {self.I} (all {self.D} sketches), {dt:.1f} s, scaled x{self.I / k:.0f}"


class KronWorkload:
    """Kronecker compression: 32 pairs 512x512, J_n = 1024, D = 10, 2^20
    recovered entries per pair."""
    name = "kron_32pairs_512x512_J1024_D10_M1M"
    metric = "FCS sketches/s (Kronecker compression, 32 pairs 512x512, J=1024, D=10, recover 2^20/pair)"
    pairs, n, J, D, Msamp, seed = 32, 512, 1024, 10, 1 << 20, 4

    def __init__(self):
        self.I4, self.J4 = [self.n] * 4, [self.J] * 4
        self.Ja = 2 * self.J - 1
        self.Jt = jt_of(self.J4)

    def config(self):
        return {"workload": self.name, "pairs": self.pairs, "matrix": [self.n, self.n],
                "J": self.J, "D": self.D, "Jt": self.Jt, "fft_len": fft_len(self.Jt),
                "samples_per_pair": self.Msamp, "seed": self.seed}

    def sketches_per_step(self):
        return self.pairs * self.D     # FCS(A o B) sketches per step

    def launches_per_step(self):
        return 1 + 2 * 2 + 1 + 1       # hashes, 2 x (zero + dense), outer, recover

    def bytes_recover(self):
        return self.pairs * self.Msamp * (4 * 4 + 4)

    def bytes_dense(self):
        return 2 * self.pairs * self.n * self.n * 4 + 2 * self.D * 2 * self.n * 5 + \
            2 * self.pairs * self.D * self.Ja * 4

    def setup(self, fcs, ctx, dev):
        import torch
        A = synth.gaussian(self.seed, (self.pairs, self.n, self.n))
        B = synth.gaussian(self.seed + 1, (self.pairs, self.n, self.n))
        idx = np.stack([synth.sample_indices(self.seed + 2 + p, self.Msamp, self.I4)
                        for p in range(self.pairs)])
        self.host = {"A": A, "B": B, "idx": idx}
        self.Ag = torch.from_numpy(A).to(dev)
        self.Bg = torch.from_numpy(B).to(dev)
        self.idxg = torch.from_numpy(idx).to(dev)
        self.fa = torch.empty((self.pairs, self.D, self.Ja), dtype=torch.float32, device=dev)
        self.fb = torch.empty_like(self.fa)
        self.fcs, self.ctx, self.dev = fcs, ctx, dev
        # the outer combine's block shape, tuned for this batch and for the
        # end-to-end leg's chunks (untimed)
        h, s = fcs.fcs_make_hashes(ctx, self.seed, self.I4, self.J4, self.D)
        ld, n = 4 * self.n, self.n
        fcs.fcs_sketch_dense(ctx, self.Ag, self.J4[:2], h[:, :2 * n], s[:, :2 * n], ldh=ld,
                             batched=True, out=self.fa)
        fcs.fcs_sketch_dense(ctx, self.Bg, self.J4[2:], h[:, 2 * n:], s[:, 2 * n:], ldh=ld,
                             batched=True, out=self.fb)
        self.outer_threads, _ = fcs.fcs_outer_autotune(ctx, self.fa, self.fb)
        per = self.pairs // 8
        fcs.fcs_outer_autotune(ctx, self.fa[:per], self.fb[:per])

    def step(self, k, marks, A=None, B=None, idx=None):
        fcs = self.fcs
        A = self.Ag if A is None else A
        B = self.Bg if B is None else B
        idx = self.idxg if idx is None else idx
        h, s = fcs.fcs_make_hashes(self.ctx, self.seed + k, self.I4, self.J4, self.D)
        ld = 4 * self.n
        marks("dense_kernel")
        fcs.fcs_sketch_dense(self.ctx, A, self.J4[:2], h[:, :2 * self.n],
                             s[:, :2 * self.n], ldh=ld, batched=True, out=self.fa)
        fcs.fcs_sketch_dense(self.ctx, B, self.J4[2:], h[:, 2 * self.n:],
                             s[:, 2 * self.n:], ldh=ld, batched=True, out=self.fb)
        marks("outer")
        sk = fcs.fcs_sketch_outer(self.ctx, self.fa, self.fb)
        marks("recover_kernel")
        rec = fcs.fcs_recover(self.ctx, sk, self.I4, self.J4, h, s, idx)
        marks(None)
        self.sk = sk
        return rec

    def e2e_prepare(self):
        import torch
        self.Ah = torch.from_numpy(self.host["A"]).pin_memory()
        self.Bh = torch.from_numpy(self.host["B"]).pin_memory()
        self.ih = torch.from_numpy(self.host["idx"]).pin_memory()
        self.Ad, self.Bd = torch.empty_like(self.Ag), torch.empty_like(self.Bg)
        self.idd = torch.empty_like(self.idxg)
        self.rh = torch.empty((self.pairs, self.Msamp), dtype=torch.float32).pin_memory()
        return ((self.Ah.numel() + self.Bh.numel() + self.ih.numel()) * 4,
                self.rh.numel() * 4)

    def e2e_step(self, k):
        """Pipelined over chunks of pairs on three streams: the upload of
        chunk c + 1 runs while chunk c is sketched, combined and recovered and
        chunk c - 1 is read back (the link is the bound: its two directions
        overlap, and the compute hides under the upload)."""
        import torch
        fcs, n = self.fcs, self.n
        main = torch.cuda.current_stream(self.dev)
        if not hasattr(self, "st_in"):
            self.st_in, self.st_cmp, self.st_out = (torch.cuda.Stream(self.dev) for _ in range(3))
        st_in, st_cmp, st_out = self.st_in, self.st_cmp, self.st_out
        for st in (st_in, st_cmp, st_out):
            st.wait_stream(main)
        chunks = 8
        per = self.pairs // chunks
        with torch.cuda.stream(st_cmp):
            h, s = fcs.fcs_make_hashes(self.ctx, self.seed + k, self.I4, self.J4, self.D)
        for c in range(chunks):
            lo, hi = c * per, (c + 1) * per
            with torch.cuda.stream(st_in):
                self.Ad[lo:hi].copy_(self.Ah[lo:hi], non_blocking=True)
                self.Bd[lo:hi].copy_(self.Bh[lo:hi], non_blocking=True)
                self.idd[lo:hi].copy_(self.ih[lo:hi], non_blocking=True)
                ev_in = torch.cuda.Event()
                ev_in.record(st_in)
            with torch.cuda.stream(st_cmp):
                st_cmp.wait_event(ev_in)
                fcs.fcs_sketch_dense(self.ctx, self.Ad[lo:hi], self.J4[:2], h[:, :2 * n],
                                     s[:, :2 * n], ldh=4 * n, batched=True, out=self.fa[lo:hi])
                fcs.fcs_sketch_dense(self.ctx, self.Bd[lo:hi], self.J4[2:], h[:, 2 * n:],
                                     s[:, 2 * n:], ldh=4 * n, batched=True, out=self.fb[lo:hi])
                sk = fcs.fcs_sketch_outer(self.ctx, self.fa[lo:hi], self.fb[lo:hi])
                rec = fcs.fcs_recover(self.ctx, sk, self.I4, self.J4, h, s, self.idd[lo:hi])
                ev_out = torch.cuda.Event()
                ev_out.record(st_cmp)
            with torch.cuda.stream(st_out):
                st_out.wait_event(ev_out)
                self.rh[lo:hi].copy_(rec, non_blocking=True)
                rec.record_stream(st_out)
                sk.record_stream(st_out)
        for st in (st_in, st_cmp, st_out):
            main.wait_stream(st)

    def check(self):
        import torch
        return bool(torch.isfinite(self.sk).all())

    def roofline(self, times_ms, props):
        peak = float(measured_peaks().get("hbm_gbs", 6787.6))
        tr = statistics.mean(times_ms["recover_kernel"])
        td = statistics.mean(times_ms["dense_kernel"])
        if tr >= td:
            name, t, by = "recover_kernel (fcs_recover, batched)", tr, self.bytes_recover()
            prof, files = "recover_kernel_kron_D10_M1M.txt", ["fcs_recover.cu", "fcs_internal.cuh"]
        else:
            name, t, by = "dense_kernel (fcs_sketch_dense, batched A and B)", td, self.bytes_dense()
            prof, files = "dense_kernel_kron_512x512_D10.txt", ["fcs_dense.cu", "fcs_internal.cuh"]
        ach = by / (t / 1e3) / 1e9
        return {"kernel": name, "bound": "hbm", "achieved": ach, "peak": peak,
                "unit": "GB/s", "frac": ach / peak,
                "traffic": profiled_traffic(prof, files),
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy)",
                "bytes_per_launch": by, "avg_launch_ms": t,
                "dense_ms": td, "outer_ms": statistics.mean(times_ms["outer"]),
                "outer_threads": self.outer_threads,
                "recover_ms": tr}

    def oracle_sample(self, budget_s=12.0):
        """FP64 oracle for one pair: dense sketches of A and B, direct
        convolution combine, recovery of a 2^16-entry sample; scaled to 32
        pairs and 2^20 samples."""
        import oracle
        A = synth.gaussian(self.seed, (1, self.n, self.n))[0]
        B = synth.gaussian(self.seed + 1, (1, self.n, self.n))[0]
        idx = synth.sample_indices(self.seed + 2, 1 << 16, self.I4)
        h, s = oracle.make_hashes(self.seed, self.I4, self.J4, self.D)
        t0 = time.perf_counter()
        fa = oracle.fcs_dense(A, self.J4[:2], h[:, :2 * self.n], s[:, :2 * self.n])
        fb = oracle.fcs_dense(B, self.J4[2:], h[:, 2 * self.n:], s[:, 2 * self.n:])
        sk = oracle.outer_combine(fa, fb)
        t1 = time.perf_counter()
        oracle.recover(sk, self.I4, self.J4, h, s, idx)
        t2 = time.perf_counter()
        per_pair = (t1 - t0) + (t2 - t1) * (self.Msamp / (1 << 16))
        return self.D / per_pair, f"one pair: dense sketches + combine ({t1 - t0:.2f} s) and 2^16 recoveries ({t2 - t1:.2f} s), scaled to 2^20"


def mixed_cp_shapes(seed: int, count: int):
    """Heterogeneous CP problems: order 3 or 4, I_n log-uniform in [50, 2000],
    rank log-uniform in [1, 256], J_n log-uniform in [256, 8192] (so Jt up to
    32765 and FFT lengths up to 32768), D uniform in 1..10."""
    g = np.random.default_rng(seed)
    shapes = []
    for _ in range(count):
        N = int(g.integers(3, 5))
        I = [int(round(math.exp(g.uniform(math.log(50), math.log(2000))))) for _ in range(N)]
        R = int(round(math.exp(g.uniform(0.0, math.log(256)))))
        J = [int(round(math.exp(g.uniform(math.log(256), math.log(8192))))) for _ in range(N)]
        D = int(g.integers(1, 11))
        shapes.append((I, J, max(1, R), D))
    return shapes


def long_cp_launches(J) -> int:
    """Kernels of one CP-route sketch with P > 16384.  P = 32768: the one
    fused kernel.  Longer (two-pass FFT route): Count Sketches, pass 1,
    pass 2, accumulate per chunk of transforms, then pack, pass 1, pass 2,
    unpack for the inverse (one chunk here)."""
    P = fft_len(jt_of(J))
    return 1 if P == 32768 else 8


class BatchWorkload:
    """64 heterogeneous CP problems per step in one batched launch chain (a
    transpose, then one kernel per FFT size; CUDA graph replay of a prepared
    plan); the plain path runs one fcs_sketch_cp per problem.  Unit:
    sketches/s."""
    name = "batch_cp_mixed64"
    metric = "FCS sketches/s (64 mixed CP problems per step, batched launch chain)"
    count, seed = 64, 5

    def __init__(self):
        self.shapes = mixed_cp_shapes(self.seed, self.count)

    def config(self):
        return {"workload": self.name, "problems": self.count,
                "order": "3-4", "I": "log-U[50,2000]", "R": "log-U[1,256]",
                "J": "log-U[256,8192] (Jt up to 32765, P up to 32768)", "D": "U{1..10}",
                "long_problems": sum(1 for _, J, _, _ in self.shapes if fft_len(jt_of(J)) > 16384),
                "sketches_per_step": self.sketches_per_step(), "seed": self.seed}

    def sketches_per_step(self):
        return sum(D for _, _, _, D in self.shapes)

    def launches_per_step(self):
        # batched transpose + one kernel per FFT size; problems with
        # P > 16384 run on the two-pass long-FFT route after them
        sizes = {fft_len(jt_of(J)) for _, J, _, _ in self.shapes if fft_len(jt_of(J)) <= 16384}
        return 1 + len(sizes) + sum(long_cp_launches(J) for _, J, _, _ in self.shapes
                                    if fft_len(jt_of(J)) > 16384)

    def setup(self, fcs, ctx, dev):
        import torch
        self.fcs, self.ctx, self.dev = fcs, ctx, dev
        self.items = []
        probs = []
        # every problem's factors and weights are views of one device buffer,
        # and every output of another, so the end-to-end step moves each way
        # in one transfer (segments padded to 16 bytes)
        data = []
        for k, (I, J, R, D) in enumerate(self.shapes):
            U, lam = synth.cp_factors(self.seed * 1000 + k, I, R)
            data.append((U, lam))
        pad4 = lambda n: (n + 3) // 4 * 4  # noqa: E731
        n_in = sum(pad4(u.size) for U, lam in data for u in U) + \
            sum(pad4(lam.size) for U, lam in data)
        n_out = sum(pad4(D * jt_of(J)) for I, J, R, D in self.shapes)
        self.inbuf = torch.empty(n_in, dtype=torch.float32, device=dev)
        self.outbuf = torch.zeros(n_out, dtype=torch.float32, device=dev)
        pos_in = pos_out = 0
        for k, ((I, J, R, D), (U, lam)) in enumerate(zip(self.shapes, data)):
            Ug = []
            for u in U:
                v = self.inbuf[pos_in:pos_in + u.size].view(u.shape)
                v.copy_(torch.from_numpy(u))
                Ug.append(v)
                pos_in += pad4(u.size)
            lamg = self.inbuf[pos_in:pos_in + lam.size]
            lamg.copy_(torch.from_numpy(lam))
            pos_in += pad4(lam.size)
            out = self.outbuf[pos_out:pos_out + D * jt_of(J)].view(D, jt_of(J))
            pos_out += pad4(D * jt_of(J))
            h, s = fcs.fcs_make_hashes(ctx, k, I, J, D)
            pr, out = fcs.cp_problem(Ug, lamg, J, h, s, out=out)
            probs.append(pr)
            self.items.append((Ug, lamg, h, s, out, J))
        # the tuning table of an earlier run is reused when FCS_AUTOTUNE_CACHE
        # names an existing file (the plan then takes the stored grain and
        # class shapes); otherwise the batch is autotuned here
        cache = os.environ.get("FCS_AUTOTUNE_CACHE")
        if cache and os.path.exists(cache):
            self.plan = fcs.BatchPlan(ctx, probs)
            self.grain = self.plan.config()[0]
        else:
            self.grain = fcs.fcs_batch_autotune(ctx, probs)
            self.plan = fcs.BatchPlan(ctx, probs, grain=self.grain)
        self.plan.launch()
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        st = torch.cuda.Stream(dev)
        with torch.cuda.stream(st):
            self.plan.launch()
            torch.cuda.synchronize()
            with torch.cuda.graph(self.graph, stream=st):
                self.plan.launch()
        torch.cuda.synchronize()

    def step(self, k, marks):
        marks("batch")
        self.graph.replay()
        marks(None)

    def plain_step(self):
        for Ug, lamg, h, s, out, J in self.items:
            self.fcs.fcs_sketch_cp(self.ctx, Ug, lamg, J, h, s, out=out)

    def e2e_prepare(self):
        import torch
        self.inh = self.inbuf.cpu().pin_memory()
        self.outh = torch.empty(self.outbuf.shape, dtype=torch.float32).pin_memory()
        return self.inh.numel() * 4, self.outh.numel() * 4

    def e2e_step(self, k):
        self.inbuf.copy_(self.inh, non_blocking=True)
        self.graph.replay()
        self.outh.copy_(self.outbuf, non_blocking=True)

    def check(self):
        import torch
        return all(bool(torch.isfinite(it[4]).all()) for it in self.items)

    def roofline(self, times_ms, props):
        import torch
        t = statistics.mean(times_ms["batch"])
        flops = 0.0
        for I, J, R, D in self.shapes:
            P = fft_len(jt_of(J))
            flops += D * (R * len(I) + 1) * 2.5 * P * math.log2(P) + \
                D * R * (P // 2 + 1) * (6 * (len(I) - 1) + 2)
        # the plain path on the same problems, same stream, for comparison
        stream = torch.cuda.current_stream(self.dev)
        for _ in range(3):
            self.plain_step()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        torch.cuda.synchronize()
        ev[0].record(stream)
        for _ in range(10):
            self.plain_step()
        ev[1].record(stream)
        torch.cuda.synchronize()
        plain_ms = ev[0].elapsed_time(ev[1]) / 10
        sm_mhz = float(measured_peaks().get("sm_max_mhz", 2070.0))
        peak = props.multi_processor_count * 128 * 2 * sm_mhz * 1e6 / 1e12
        ach = flops / (t / 1e3) / 1e12
        return {"kernel": "batch (transpose + batch_class_kernel per FFT size, graph replay)",
                "bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak,
                "traffic": profiled_traffic("batch_class_kernels_mixed64.txt",
                                            ["fcs_batch.cu", "fcs_batch_kernels.cuh",
                                             "fcs_batch_k0.cu", "fcs_batch_k1.cu",
                                             "fcs_batch_k2.cu", "fcs_batch_k3.cu",
                                             "fcs_batch_k4.cu", "fcs_cp_run.cuh", "fcs_fft.cuh",
                                             "fcs_internal.cuh"]),
                "peak_source": f"derived: {props.multi_processor_count} SMs x 128 FP32 lanes "
                               f"x 2 flop/FMA x {sm_mhz:.0f} MHz",
                "avg_launch_ms": t, "grain": self.grain,
                "classes": [{"fft_len": P, "engine": "warp-DIT" if e else "slot FFT",
                             "thread_mult": m, "items_per_cta": i, "threads": n}
                            for P, m, i, n, e in self.plan.config()[1]],
                "plain_per_problem_ms": plain_ms,
                "plain_sketches_per_s": self.sketches_per_step() / (plain_ms / 1e3),
                "batched_over_plain": plain_ms / t}

    def oracle_sample(self, budget_s=12.0):
        import oracle
        t0 = time.perf_counter()
        done = 0
        for k, (I, J, R, D) in enumerate(self.shapes):
            U, lam = synth.cp_factors(self.seed * 1000 + k, I, R)
            h, s = oracle.make_hashes(k, I, J, 1)
            oracle.fcs_cp([u.astype(np.float64) for u in U], lam.astype(np.float64), J, h, s)
            done += 1
            if time.perf_counter() - t0 > budget_s:
                break
        dt = time.perf_counter() - t0
        return done / dt, f"sketch d=0 of the first {done} problems, {dt:.1f} s"


WORKLOADS = {"cp": CpWorkload, "dense": DenseWorkload, "kron": KronWorkload,
             "batch": BatchWorkload}


# ================================================================== serving
def run_serve(args, rank, world, local_rank):
    """Serving workload: 10,000 requests with Poisson arrivals, half CP-route
    sketches (order 3-4, I_n log-U[50,2000], rank log-U[1,256], J_n
    log-U[256,8192], so FFT lengths up to 32768, D U{1..10}; 96 shape
    templates), half
    contractions (T(u,u,u) : T(I,u,u) = 1 : 1, 1-16 vectors) against 16
    resident sketches.  The offered rate is 0.8 x the capacity of the plain
    path (one request at a time: copy in, hashes, one launch, copy out,
    synchronise), measured first.  Both paths see the same arrival
    schedule; the server's capacity is also measured at saturation."""
    import threading
    import torch
    import paper_2106_13062_gb300 as fcs
    if rank != 0:
        return None
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    g = np.random.default_rng(7)
    nreq = args.requests
    templates = []
    for k, (I, J, R, D) in enumerate(mixed_cp_shapes(70, 96)):
        U, lam = synth.cp_factors(7000 + k, I, R)
        templates.append((I, J, R, D, U, lam))
    res_shapes = []
    for k in range(16):
        I = [int(g.integers(50, 500))] * 3
        J = [int(g.integers(256, 2000))] * 3
        U, lam = synth.cp_factors(8000 + k, I, 8)
        res_shapes.append((I, J, 8, 5, U, lam, 9000 + k))
    reqs = []
    for i in range(nreq):
        if g.random() < 0.5:
            reqs.append(("cp", int(g.integers(0, len(templates))), 1000 + i))
        else:
            k = int(g.integers(0, len(res_shapes)))
            kind = fcs.FCS_CONTRACT_ALL if g.random() < 0.5 else fcs.FCS_CONTRACT_FREE
            B = int(g.integers(1, 17))
            vec = synth.unit_vectors(20000 + i, B, res_shapes[k][0][0])
            reqs.append(("ct", k, kind, vec))

    # ---- plain path: one request per launch, synchronised
    ctx = fcs.Context(local_rank)
    dU = [[torch.from_numpy(u).to(dev) for u in t[4]] for t in templates]
    hU = [[torch.from_numpy(u).pin_memory() for u in t[4]] for t in templates]
    dlam = [torch.from_numpy(t[5]).to(dev) for t in templates]
    hlam = [torch.from_numpy(t[5]).pin_memory() for t in templates]
    douts = [torch.empty((t[3], jt_of(t[1])), device=dev) for t in templates]
    houts = [torch.empty((t[3], jt_of(t[1]))).pin_memory() for t in templates]
    resident = []
    for I, J, R, D, U, lam, seed in res_shapes:
        h, s_ = fcs.fcs_make_hashes(ctx, seed, I, J, D)
        sk = fcs.fcs_sketch_cp(ctx, [torch.from_numpy(u).to(dev) for u in U],
                               torch.from_numpy(lam).to(dev), J, h, s_)
        resident.append((I, J, h, s_, sk))
    torch.cuda.synchronize()

    def plain(r):
        if r[0] == "cp":
            k, seed = r[1], r[2]
            I, J, R, D, _, _ = templates[k]
            for d_, h_ in zip(dU[k], hU[k]):
                d_.copy_(h_, non_blocking=True)
            dlam[k].copy_(hlam[k], non_blocking=True)
            fcs.fcs_sketch_cp_seeded(ctx, dU[k], dlam[k], J, D, seed, out=douts[k])
            houts[k].copy_(douts[k], non_blocking=True)
        else:
            _, k, kind, vec = r
            I, J, h, s_, sk = resident[k]
            v = torch.from_numpy(vec).to(dev, non_blocking=True)
            vv = [None if (kind == fcs.FCS_CONTRACT_FREE and m == 0) else v for m in range(3)]
            out = fcs.fcs_contract(ctx, kind, sk, vv, I, J, h, s_, free_mode=0)
            out.cpu()
        torch.cuda.synchronize()

    for r in reqs[:20]:
        plain(r)
    sampler = ClockSampler(local_rank)
    sampler.start()
    t0 = time.perf_counter()
    ncap = min(400, nreq)
    for r in reqs[:ncap]:
        plain(r)
    mu = ncap / (time.perf_counter() - t0)              # requests/s
    lam_rate = 0.8 * mu
    arrivals = np.cumsum(g.exponential(1.0 / lam_rate, size=nreq))
    sk_per_req = [templates[r[1]][3] if r[0] == "cp" else 0 for r in reqs]

    # plain path under the arrival schedule
    lat_plain = np.empty(nreq)
    start = time.perf_counter()
    for i, r in enumerate(reqs):
        while time.perf_counter() - start < arrivals[i]:
            pass
        plain(r)
        lat_plain[i] = time.perf_counter() - start - arrivals[i]
    plain_wall = time.perf_counter() - start

    # ---- served path under the same schedule
    srv = fcs.FcsServer(device=local_rank, streams=4, max_inflight=128, max_batch=48,
                        arena_bytes=6 << 30, staging_bytes=2 << 30)
    sids = []
    for I, J, R, D, U, lam, seed in res_shapes:
        t = srv.submit_cp(U, lam, J, D, seed=seed, keep_resident=True)
        sids.append(srv.wait(t, 120.0).sketch_id)

    def submit(r, out_store, idx):
        if r[0] == "cp":
            I, J, R, D, U, lam = templates[r[1]]
            out = np.empty((D, jt_of(J)), dtype=np.float32)
            out_store[idx] = out
            return srv.submit_cp(U, lam, J, D, seed=r[2], out=out)
        _, k, kind, vec = r
        I, J = res_shapes[k][0], res_shapes[k][1]
        out = np.empty((vec.shape[0],) if kind == fcs.FCS_CONTRACT_ALL
                       else (vec.shape[0], I[0]), dtype=np.float32)
        out_store[idx] = out
        vv = [None if (kind == fcs.FCS_CONTRACT_FREE and m == 0) else vec for m in range(3)]
        return srv.submit_contract(sids[k], I, J, kind, vv, out)

    # warm-up, as the plain path had: the first request of every CP template
    # and of every (resident sketch, contraction kind) once, so the server's
    # device workspace reaches its final size before the timed runs
    seen, warm_out, warm_t = set(), {}, []
    for i, r in enumerate(reqs):
        key = ("cp", r[1]) if r[0] == "cp" else (r[1], r[2])
        if key not in seen:
            seen.add(key)
            warm_t.append(submit(r, warm_out, i))
    for t in warm_t:
        if srv.wait(t, 120.0).state != 2:
            raise RuntimeError("serving warm-up request failed")

    def served_run(sched):
        srv.reset_stats()
        tickets = [None] * nreq
        outs = [None] * nreq

        def producer():
            st0 = time.perf_counter()
            for i, r in enumerate(reqs):
                if sched is not None:
                    while time.perf_counter() - st0 < sched[i]:
                        time.sleep(0)
                tickets[i] = submit(r, outs, i)
        th = threading.Thread(target=producer)
        t_start = time.perf_counter()
        th.start()
        lat = np.empty(nreq)
        for i in range(nreq):
            while tickets[i] is None:
                time.sleep(0)
            res = srv.wait(tickets[i], 600.0)
            if res.state != 2:
                raise RuntimeError(f"request {i} ended in state {res.state}")
            lat[i] = res.latency_s
        th.join()
        wall = time.perf_counter() - t_start
        st = srv.stats()
        return lat, wall, st, outs

    lat_srv, srv_wall, st_srv, outs_srv = served_run(arrivals)
    lat_sat, sat_wall, st_sat, _ = served_run(None)
    clocks = sampler.stop()
    srv.close()
    accuracy = serve_accuracy(fcs, ctx, dev, reqs, outs_srv, templates, res_shapes, resident)
    ctx.close()
    sk_total = float(sum(sk_per_req))
    plain_cap_sk = mu * sk_total / nreq
    res = {
        "impl": "fcs",
        "metric": "served sketch requests: sketches/s at saturation, p50/p99 latency at 0.8x plain capacity",
        "value": sk_total / sat_wall, "unit": "sketches/s", "n_gpus": world,
        "steps": nreq, "warmup": 20, "ms_per_step": 1e3 * sat_wall / nreq,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "serve_10k_poisson_mixed", "requests": nreq,
                   "mix": "50% CP sketch (96 templates, order 3-4, I log-U[50,2000], R log-U[1,256], J log-U[256,8192] so P up to 32768, D U{1..10}); 50% contractions UUU:IUU 1:1, B U{1..16}, 16 resident sketches",
                   "arrivals": "Poisson, rate 0.8 x measured plain capacity", "seed": 7,
                   "server": "4 streams, 128 slots, 48 CP per round"},
        "serving": {
            "offered_rate_req_s": lam_rate,
            "plain_capacity_req_s": mu, "plain_capacity_sketches_s": plain_cap_sk,
            "served_capacity_req_s": nreq / sat_wall,
            "served_capacity_sketches_s": sk_total / sat_wall,
            "capacity_ratio_served_over_plain": (nreq / sat_wall) / mu,
            "plain_p50_s": float(np.percentile(lat_plain, 50)),
            "plain_p99_s": float(np.percentile(lat_plain, 99)),
            "served_p50_s": float(np.percentile(lat_srv, 50)),
            "served_p99_s": float(np.percentile(lat_srv, 99)),
            "plain_wall_s": plain_wall, "served_wall_s": srv_wall,
            "served_rounds": st_srv.rounds, "served_max_inflight": st_srv.max_inflight_seen,
            "saturation_rounds": st_sat.rounds,
            "saturation_p50_s": float(np.percentile(lat_sat, 50)),
            "saturation_p99_s": float(np.percentile(lat_sat, 99)),
        },
        "accuracy": accuracy,
        "clocks": clocks,
        # saturation run: per round a batched transpose + one kernel per FFT
        # size (counted by the server), per CP request a hash kernel, per
        # contraction spectrum + contract + median kernels
        "gpu_launches": int(st_sat.batch_launches + sum(1 for r in reqs if r[0] == "cp")
                            + 3 * sum(1 for r in reqs if r[0] == "ct")),
    }
    return res


def serve_accuracy(fcs, ctx, dev, reqs, outs, templates, res_shapes, resident, sample=48):
    """Served results against direct library calls on the same inputs, for a
    sample of the requests of the scheduled run: CP sketches in relative L2
    per sketch (bar 1e-5); T(u,u,u) medians on the Cauchy-Schwarz scale
    max_d ||FCS_d T|| ||FCS_d(u o u o u)|| (bar 1e-4); T(I,u,u) medians in
    relative L2 per vector (bar 1e-4).  The served contractions read the
    server's resident copy of each sketch, the direct ones the plain path's."""
    import torch
    cp_err = all_err = free_err = 0.0
    n_cp = n_ct = 0
    for i, r in enumerate(reqs):
        if r[0] == "cp" and n_cp < sample:
            I, J, R, D, U, lam = templates[r[1]]
            h, s_ = fcs.fcs_make_hashes(ctx, r[2], I, J, D)
            ref = fcs.fcs_sketch_cp(ctx, [torch.from_numpy(u).to(dev) for u in U],
                                    torch.from_numpy(lam).to(dev), J, h, s_).cpu().numpy()
            got = outs[i]
            for d in range(D):
                den = np.linalg.norm(ref[d]) or 1.0
                cp_err = max(cp_err, float(np.linalg.norm(got[d] - ref[d]) / den))
            n_cp += 1
        elif r[0] == "ct" and n_ct < sample:
            _, k, kind, vec = r
            I, J, h, s_, sk = resident[k]
            v = torch.from_numpy(vec).to(dev)
            got = outs[i]
            if kind == fcs.FCS_CONTRACT_ALL:
                ref = fcs.fcs_contract(ctx, kind, sk, [v, v, v], I, J, h, s_).cpu().numpy()
                nT = torch.linalg.norm(sk, dim=1)
                for b in range(vec.shape[0]):
                    ub = v[b].reshape(-1, 1).contiguous()
                    r1 = fcs.fcs_sketch_cp(ctx, [ub, ub, ub], None, J, h, s_)
                    scale = float((nT * torch.linalg.norm(r1, dim=1)).max())
                    all_err = max(all_err, abs(float(got[b]) - float(ref[b])) / scale)
            else:
                ref = fcs.fcs_contract(ctx, kind, sk, [None, v, v], I, J, h, s_,
                                       free_mode=0).cpu().numpy()
                for b in range(vec.shape[0]):
                    den = np.linalg.norm(ref[b]) or 1.0
                    free_err = max(free_err, float(np.linalg.norm(got[b] - ref[b]) / den))
            n_ct += 1
        if n_cp >= sample and n_ct >= sample:
            break
    return {"checked_cp": n_cp, "checked_contractions": n_ct,
            "cp_max_rel_l2": cp_err, "contract_all_max_err_cs_scale": all_err,
            "contract_free_max_rel_l2": free_err,
            "bars": {"cp": 1e-5, "contract_all": 1e-4, "contract_free": 1e-4},
            "pass": cp_err <= 1e-5 and all_err <= 1e-4 and free_err <= 1e-4}


# ================================================================== arms
def run_reference(args, rank, world):
    """The FP64 oracle as the reference arm, on the host cores, rank 0 only."""
    if rank != 0:
        return None
    w = WORKLOADS[args.workload]() if args.workload in WORKLOADS else None
    if w is None or not hasattr(w, "reference_step"):
        return {"impl": "reference", "unavailable":
                f"reference arm only defined for the default workload (cp), not {args.workload}"}
    w.reference_setup()
    for k in range(args.warmup):
        w.reference_step(k)
    t0 = time.perf_counter()
    units = 0.0
    for k in range(args.steps):
        units += w.reference_step(k)
    dt = time.perf_counter() - t0
    value = units / dt
    return {
        "impl": "reference", "metric": w.metric, "value": value, "unit": "sketches/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(w.config(), parallelism="cpu oracle"),
        "cpu_baseline": {"value": value, "unit": "sketches/s", "cores": omp_threads(),
                         "kind": "oracle", "sample": w.reference_sample},
        "e2e": {"value": value, "unit": "sketches/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }


def reduce_max_over_ranks(values, world):
    """Per-rank timings -> their maxima over all ranks (replicas: the slowest
    rank sets the job's time).  Works with NCCL (device tensors) and gloo."""
    if world <= 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist
    dev = (torch.device("cuda", torch.cuda.current_device())
           if dist.get_backend() == "nccl" else torch.device("cpu"))
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


def job_rate(world, units_per_step, steps, time_ms):
    """Whole-job throughput: units all ranks processed / the slowest rank's time."""
    return world * units_per_step * steps / (time_ms / 1e3)


def measure(wname, args, rank, world, local_rank, steps, warmup, cpu_baseline=True):
    """One workload on the FCS path: `warmup` untimed steps, then a loaded
    clock window (the same steps, untimed, for about args.clock_window_s
    seconds while nvidia-smi samples the clocks), then exactly `steps` timed
    steps (CUDA events on the launching stream, L2 flushed between steps),
    then the end-to-end leg with host buffers.  Returns the JSON dict (rank 0)."""
    import torch
    import paper_2106_13062_gb300 as fcs

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    w = WORKLOADS[wname]()
    ctx = fcs.Context(local_rank)
    w.setup(fcs, ctx, dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    for k in range(warmup):
        w.step(k, lambda _: None)
    torch.cuda.synchronize()

    # ---- device-resident timed region: per-step events, per-kernel marks
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    marks_all = []
    sampler = ClockSampler(local_rank)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler.start()
    window = clock_window(w, flush, args.clock_window_s, warmup)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    for k in range(steps):
        flush.zero_()                                   # L2 flush, untimed
        starts[k].record(stream)
        marks = []

        def mark(name, marks=marks):
            e = torch.cuda.Event(enable_timing=True)
            e.record(stream)
            marks.append((name, e))
        w.step(warmup + k, mark)
        ends[k].record(stream)
        marks_all.append(marks)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    clocks["window"] = window
    if world > 1:
        torch.distributed.barrier()
    total_ms = sum(a.elapsed_time(b) for a, b in zip(starts, ends))
    times = {}
    for marks in marks_all:
        for (name, e0), (_, e1) in zip(marks, marks[1:]):
            times.setdefault(name, []).append(e0.elapsed_time(e1))
    if not w.check():
        raise RuntimeError("non-finite output")

    # ---- end to end with host buffers (inputs H2D and results D2H per step)
    h2d, d2h = w.e2e_prepare()
    e2e_steps = max(3, min(steps, 50 if wname != "cp" else 200))
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(e2e_steps)]
    torch.cuda.synchronize()
    for k in range(e2e_steps):
        flush.zero_()
        ev[k][0].record(stream)
        w.e2e_step(k)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    e2e_ms = sum(a.elapsed_time(b) for a, b in ev) / e2e_steps

    tmax, e2e_ms = reduce_max_over_ranks([total_ms, e2e_ms], world)
    props = torch.cuda.get_device_properties(local_rank)
    roof = w.roofline(times, props)
    ctx.close()
    if rank != 0:
        return None
    per_step = w.sketches_per_step()
    res = {
        "impl": "fcs", "metric": w.metric, "value": job_rate(world, per_step, steps, tmax),
        "unit": "sketches/s", "n_gpus": world, "steps": steps, "warmup": warmup,
        "ms_per_step": tmax / steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(w.config(),
                       parallelism=f"replicas x{world}" if world > 1 else "single GPU",
                       l2="flushed between timed steps (256 MiB write)"),
        "roofline": roof,
        "e2e": {"value": job_rate(world, per_step, 1, e2e_ms), "unit": "sketches/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": e2e_ms},
        "gpu_launches": w.launches_per_step() * steps,
        "clocks": clocks,
        "kernel_ms": {k: statistics.mean(v) for k, v in times.items()},
    }
    if world == 1 and cpu_baseline and not args.no_cpu_baseline:
        v, sample = w.oracle_sample(budget_s=args.cpu_budget_s)
        res["cpu_baseline"] = {"value": v, "unit": "sketches/s", "cores": omp_threads(),
                               "kind": "oracle", "sample": sample}
    return res


def clock_window(w, flush, seconds, k0):
    """Untimed steps of the workload for about `seconds` (L2 flushed between
    them, as in the timed region) so that the clock sampler sees the GPU under
    this load; the timed steps follow directly.  Returns what ran."""
    import torch
    if seconds <= 0:
        return {"steps": 0, "s": 0.0}
    t0 = time.perf_counter()
    n = 0
    while True:
        for _ in range(8):
            flush.zero_()
            w.step(k0 + n, lambda _: None)
            n += 1
        torch.cuda.synchronize()
        if time.perf_counter() - t0 >= seconds:
            break
    return {"steps": n, "s": round(time.perf_counter() - t0, 3),
            "what": "untimed steps of this workload directly before the timed ones; "
                    "the clock samples span them and the timed region"}


def run_fcs(args, rank, world, local_rank):
    return measure(args.workload, args, rank, world, local_rank, args.steps, args.warmup)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["fcs", "reference"], default="fcs")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["serve"], default="cp")
    ap.add_argument("--requests", type=int, default=10000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="default workload only: skip the dense, kron, batch and serve sub-results")
    ap.add_argument("--clock-window-s", type=float, default=1.0,
                    help="seconds of untimed steps, sampled for clocks, before the timed ones")
    ap.add_argument("--cpu-budget-s", type=float, default=10.0,
                    help="seconds of CPU oracle work per cpu_baseline sample")
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
    res = (run_serve if args.workload == "serve" else run_fcs)(args, rank, world, local_rank)
    if res is not None and args.workload == "cp" and world == 1 and not args.no_extra:
        # the metric's other parts on one GPU: the dense route and both
        # contractions (RTPM step), Kronecker compression with recovery (HBM
        # rooflines), the batched launch chain against one launch per
        # problem, and the served path against the plain one (p50/p99)
        extra = {}
        for name in ("dense", "kron", "batch"):
            extra[name] = measure(name, args, rank, world, local_rank, args.steps, args.warmup)
        extra["serve"] = run_serve(args, rank, world, local_rank)
        res.update(extra)
        res["extra_keys"] = sorted(extra)
    if res is not None:
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
