#!/usr/bin/env python3
"""Benchmark of the Polar Express online stage on GB300.

One "step" is one Muon orthogonalisation step of the workload: every matrix
of the set normalised and taken through T polynomial steps by one
``pe_polar_batched`` call (prepare launch + one persistent grouped tcgen05
launch per polynomial step, replayed from a CUDA graph).

The headline workload is the large dense set (8192 x 8192, 4096 x 14336,
14336 x 4096; Haar singular vectors, singular values log-uniform in
[1e-4, 1]; l = 1e-4, T = 6), generated on the GPU from a seeded generator.
Reported ``value``: algorithmic polar TFLOP/s, sum over matrices of
T (3 s^2 L + s^3) per step (s = min(m, n), L = max(m, n); the Gram and A^2
products are symmetric and counted once), divided by the device time of the
step, with inputs resident in HBM. ``e2e`` repeats the measurement through
the host-buffer entry ``pe_polar_batched_host`` with the inputs copied from
pinned host memory and the factors copied back inside the timed region.
``roofline`` attributes device time to the dominant kernel from CUDA events
bracketing each launch (library tracing) over the same steps.
``cpu_baseline`` times the FP64 oracle on the host cores on a bounded
sample. ``fp32_plain`` and ``speedup_vs_fp32_plain`` compare with the plain
FP32 path at equal restricted max|sigma - 1| (the smallest BF16 T whose
error is no larger than the FP32 one at the workload's T). The GPT-2-small
Muon step is reported beside it (``gpt2_small``) with its own roofline,
e2e and CPU baseline.

Launch: ``python bench.py [--gpus N] [--steps K] [--warmup W]``; for N > 1
under torchrun every rank runs its own set of the workload (same shapes,
own seeds; no collective in the timed region; weak scaling, ``value`` = all
ranks' flops over the slowest rank's time), and beside it one shared set is
taken through the distributed-Muon form (LPT ownership of whole matrices,
one NCCL all-gather of the results inside the timed region;
``sharded_exchange``, strong scaling). Rank 0 prints the line.
``--impl reference`` times the FP64 oracle on the host (the reference arm).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

METRIC = "polar TFLOP/s & µs/Muon-step, BF16 grouped vs FP32 plain at equal max|σ−1|"
L2_BYTES = 129 * 1024 * 1024
LARGE_SHAPES = ((8192, 8192), (4096, 14336), (14336, 4096))
LARGE_NAME = "large_dense_8192sq_4096x14336_14336x4096"

CPU_WORKLOADS = {
    "gpt2_small": lambda: synth.gpt2_small(),
    "uneven_d1024": lambda: synth.uneven_d1024(),
    "gpt2_heads": lambda: synth.gpt2_heads(),
    "ill_conditioned": lambda: synth.ill_conditioned(),
    "plain_small": lambda: synth.plain_small(),
}
WORKLOADS = sorted(list(CPU_WORKLOADS) + ["large_dense"])


def algorithmic_flops(shapes, T):
    f = 0.0
    for m, n in shapes:
        s, L = min(m, n), max(m, n)
        f += 3.0 * s * s * L + float(s) ** 3
    return f * T


def dense_equiv_flops(shapes, T):
    f = 0.0
    for m, n in shapes:
        s, L = min(m, n), max(m, n)
        f += 4.0 * s * s * L + 2.0 * float(s) ** 3
    return f * T


def algorithmic_bytes_bf16(shapes, T):
    """Compulsory bytes per polynomial step with BF16 operands only
    (read X twice, write X, read/write A and B once each): 6 s L + 6 s^2."""
    b = 0.0
    for m, n in shapes:
        s, L = min(m, n), max(m, n)
        b += 6.0 * s * L + 6.0 * s * s
    return b * T


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return {"hbm_gbs": d.get("hbm_gbs", 6800.0), "bf16_tflops": d.get("bf16_tflops", 1900.0),
                "bf16_tflops_sustained": d.get("bf16_tflops_sustained", 1700.0),
                "sm_max_mhz": d.get("sm_max_mhz", 2070.0), "source": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0,
            "source": "fallback"}


# --------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, power = [], [], []
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                    power.append(float(parts[3]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power)}


# ------------------------------------------------------------ CPU oracle

def cpu_cores():
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads") for i in threadpool_info() if i.get("user_api") == "blas"]
        if n and n[0]:
            return int(n[0])
    except Exception:
        pass
    for v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS"):
        if os.environ.get(v):
            return int(os.environ[v])
    return os.cpu_count() or 1


def oracle_sample(mats, table, budget_s: float):
    """Time the FP64 oracle iteration over ``mats`` (host arrays) in order
    until ``budget_s`` has elapsed (at least one matrix). A matrix whose full
    iteration would overrun the budget (at an assumed 100 GFLOP/s FP64) is
    sampled with its first polynomial step only. Returns (TFLOP/s, seconds,
    matrices done, steps per matrix)."""
    import oracle as O
    done, flops, steps_used = 0, 0.0, []
    t0 = time.perf_counter()
    for G in mats:
        steps = len(table)
        if dense_equiv_flops([G.shape], steps) / 1e11 > max(budget_s, 1.0):
            steps = 1
        O.polar_express(np.asarray(G, dtype=np.float64), table[:steps])
        done += 1
        steps_used.append(steps)
        flops += algorithmic_flops([G.shape], steps)
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    return flops / dt / 1e12, dt, done, steps_used


def cpu_baseline_line(mats, table, budget_s, what):
    tf, secs, done, steps = oracle_sample(mats, table, budget_s)
    if all(s == len(table) for s in steps):
        how = f"T={len(table)}"
    else:
        how = "the first polynomial step of each"
    return {"value": tf, "unit": "TFLOP/s", "cores": cpu_cores(), "kind": "oracle",
            "sample": f"FP64 numpy oracle iteration of the first {done} of {len(mats)} matrices of {what}, "
                      f"{how} ({secs:.1f} s)"}


# ------------------------------------------------------------ workloads

class Work:
    """A workload resident on the GPU: FP32 inputs (never overwritten), known
    factors where drawn that way (for restricted error metrics), host copies
    on demand."""

    def __init__(self, name, shapes, l, T, dev_in, facs=None, note="", svd=None, host=None):
        self.name, self.shapes, self.l, self.T = name, [tuple(s) for s in shapes], l, T
        self.dev_in, self.facs, self.note, self.svd = dev_in, facs, note, svd
        self._host = host

    def host(self):
        if self._host is None:
            self._host = [d.cpu().numpy() for d in self.dev_in]
        return self._host


def large_dense_gpu(torch, seed=3, shapes=LARGE_SHAPES):
    """The large dense set on the GPU: G = U diag(s) V^T with U, V from the
    QR of seeded Gaussian matrices (Haar) and s i.i.d. log-uniform in
    [1e-4, 1], sorted; FP32. Keeps U1, V1: the singular directions with
    s_i >= 1e-3 s_max (restricted metric)."""
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    mats, facs = [], []
    for m, n in shapes:
        k = min(m, n)
        U, _ = torch.linalg.qr(torch.randn(m, k, device="cuda", generator=gen))
        V, _ = torch.linalg.qr(torch.randn(n, k, device="cuda", generator=gen))
        e = torch.rand(k, device="cuda", generator=gen) * 4.0 - 4.0
        sv = torch.sort(10.0 ** e, descending=True).values
        mats.append(((U * sv) @ V.T).contiguous())
        keep = sv >= 1e-3 * sv[0]
        facs.append((U[:, keep].contiguous(), V[:, keep].contiguous()))
        del U, V
    torch.cuda.empty_cache()
    return Work(LARGE_NAME, shapes, 1e-4, 6, mats, facs,
                "Haar U,V (QR of seeded Gaussians on the GPU); s log-uniform [1e-4,1]; l=1e-4, T=6")


# per-rank sets of the multi-GPU weak-scaling run: the same shapes and
# distributions, other seeds (rank 0 keeps the single-GPU set)
RANK_WORKLOADS = {
    "gpt2_small": lambda r: synth.gpt2_small(first_seed=1 + 100 * r),
    "gpt2_heads": lambda r: synth.gpt2_heads(first_seed=5000 + 1000 * r),
}


def load_workload(name, torch, rank=0):
    if name == "large_dense":
        return large_dense_gpu(torch, seed=3 + 1009 * rank)
    wl = RANK_WORKLOADS[name](rank) if (rank and name in RANK_WORKLOADS) else CPU_WORKLOADS[name]()
    host = [G.astype(np.float32) for G in wl.matrices]
    dev = [torch.from_numpy(h).cuda() for h in host]
    return Work(wl.name, wl.shapes, wl.l, wl.T, dev, None, wl.note, svd=wl.svd, host=host)


def restricted_err(torch, xs, facs):
    """max |sigma_i - 1| over the directions kept in facs: singular values
    of U1^T X V1 (FP32 products, TF32 off)."""
    worst = 0.0
    for X, (U1, V1) in zip(xs, facs):
        C = U1.T @ X @ V1
        worst = max(worst, float((torch.linalg.svdvals(C) - 1.0).abs().max()))
    return worst


# ------------------------------------------------------------ reference arm

def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_reference(args, world, rank):
    """The FP64 oracle on the host cores, the same metric and unit. Each step
    is a bounded sample of the workload: the large dense set at a quarter of
    its sides (2048^2, 1024 x 3584, 3584 x 1024, same spectrum law, l, T),
    one matrix per step, cycling; other workloads: one of their matrices per
    step."""
    if rank != 0:
        return 0
    import oracle as O
    if args.workload == "large_dense":
        mats = []
        for j, (m, n) in enumerate([(2048, 2048), (1024, 3584), (3584, 1024)]):
            rng = np.random.default_rng(3 + j)
            s = synth.spectrum_loguniform(rng, min(m, n), 1e-4, 1.0)
            mats.append(synth.svd_matrix(rng, m, n, s).G)
        name, l, T = LARGE_NAME, 1e-4, 6
        sample = "FP64 numpy oracle iteration, T=6, of one quarter-side matrix of the large dense set per step"
    else:
        wl = CPU_WORKLOADS[args.workload]()
        mats, name, l, T = wl.matrices, wl.name, wl.l, wl.T
        sample = f"FP64 numpy oracle iteration, one matrix of {name} per step, T={T}"
    table, _ = O.optimal_composition(l, T, safety=1.01)
    n = len(mats)
    for i in range(args.warmup):
        O.polar_express(mats[i % n], table[:1])
    tot_f, tot_t = 0.0, 0.0
    for i in range(args.steps):
        G = mats[i % n]
        t0 = time.perf_counter()
        O.polar_express(G, table)
        tot_t += time.perf_counter() - t0
        tot_f += algorithmic_flops([G.shape], T)
    val = tot_f / tot_t / 1e12
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "TFLOP/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": name, "T": T, "l": l, "matrices": n,
                   "step": "one matrix of the sample per step, cycling"},
        "cpu_baseline": {"value": val, "unit": "TFLOP/s", "cores": cpu_cores(), "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------- roofline

# source files whose contents decide each kernel's DRAM traffic
KERNEL_SOURCES = {
    "umma_step": ("pe_umma.cu", "pe_umma.h", "pe_internal.h"),
    "prepare": ("pe_prep.cu", "pe_internal.h"),
}


def kernel_source_hash(kernel: str = "umma_step"):
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_2505_16932_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def committed_traffic(workload: str, kernel: str):
    """Per-launch DRAM bytes from a committed ncu summary, if it was taken on
    the current kernel source (profiles/traffic.txt: workload kernel hash bytes)."""
    p = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(p):
        return None
    hsh = kernel_source_hash(kernel) if kernel in KERNEL_SOURCES else None
    with open(p) as f:
        for line in f:
            parts = line.split()
            if len(parts) == 4 and parts[0] == workload and parts[1] == kernel and parts[2] == hsh:
                return float(parts[3])
    return None


def roofline_line(trace, shapes, dtype, flops_step, in_bytes, workload, peaks, fp32_peak=None):
    """Roofline of the dominant kernel (largest traced time): algorithmic
    flops (or bytes) per launch over its mean CUDA-event launch time, against
    the measured burst peak (and the sustained one for tensor-bound kernels);
    FP32 SIMT kernels against the measured cuBLAS FP32 (no TF32) rate when
    given, else the derived SIMT roof; DRAM traffic from the committed ncu
    figure while the source matches."""
    dom_name, (dom_n, dom_ms) = max(trace.items(), key=lambda kv: kv[1][1])
    dom_avg_ms = dom_ms / dom_n
    tot_trace_ms = sum(v[1] for v in trace.values())
    peak_source = peaks["source"] + " burst"
    if dom_name in ("umma_step", "simt_update", "umma_update", "umma_gram", "umma_square", "simt_gram",
                    "simt_square"):
        if dom_name == "umma_step":
            f_launch = flops_step
        else:
            f_launch = 0.0
            key = dom_name.split("_")[1]
            for m, n in shapes:
                s, L = min(m, n), max(m, n)
                f_launch += {"gram": s * s * L, "square": float(s) ** 3, "update": 2.0 * s * s * L}[key]
        achieved = f_launch / (dom_avg_ms * 1e-3) / 1e12
        if dtype == "fp32":
            if fp32_peak:
                peak, unit, bound = fp32_peak, "TFLOP/s", "alu"
                peak_source = "measured cuBLAS FP32 (TF32 off) 8192^3"
            else:
                # FP32 SIMT roof: 152 SMs x 128 FP32 lanes x 2 flop x max SM clock
                peak, unit, bound = 152 * 128 * 2 * peaks["sm_max_mhz"] * 1e6 / 1e12, "TFLOP/s", "alu"
                peak_source = "derived (152 SMs x 128 lanes x 2 x max SM clock)"
        else:
            peak, unit, bound = peaks["bf16_tflops"], "TFLOP/s", "tensor"
    else:
        achieved = in_bytes * 2 / (dom_avg_ms * 1e-3) / 1e9
        peak, unit, bound = peaks["hbm_gbs"], "GB/s", "hbm"
    roofline = {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit, "frac": achieved / peak,
                "traffic": committed_traffic(workload, dom_name), "kernel": dom_name, "kernel_ms_avg": dom_avg_ms,
                "launches_traced": dom_n, "share_of_step": dom_ms / tot_trace_ms,
                "peak_source": peak_source,
                "algorithmic_bytes_per_launch_bf16": algorithmic_bytes_bf16(shapes, 1)}
    if bound == "tensor":
        roofline["peak_sustained"] = peaks["bf16_tflops_sustained"]
        roofline["frac_sustained"] = achieved / peaks["bf16_tflops_sustained"]
    return roofline


# ------------------------------------------------------------ measurement

class Ctx:
    def __init__(self, pe, torch, world, rank, local):
        self.pe, self.torch = pe, torch
        self.world, self.rank, self.local = world, rank, local
        self.stream = torch.cuda.current_stream()
        self.flush = torch.empty(max(2 * L2_BYTES, 256 << 20) // 4, dtype=torch.float32, device="cuda")

    def barrier(self):
        self.torch.cuda.synchronize()
        if self.world > 1:
            import torch.distributed as dist
            dist.barrier()
        self.torch.cuda.synchronize()

    def max_over_ranks(self, x):
        if self.world == 1:
            return x
        import torch.distributed as dist
        t = self.torch.tensor([x], dtype=self.torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())


def time_calls(ctx, xs, src, table, dtype, n, flags=0):
    """Mean CUDA-event time (ms) of ``n`` pe_polar_batched calls, each on
    restored inputs after an L2 flush (restore and flush outside the events)."""
    torch, pe = ctx.torch, ctx.pe
    for _ in range(2):
        for d, s in zip(xs, src):
            d.copy_(s)
        pe.pe_polar_batched(xs, table, dtype, flags=flags)
    tot = 0.0
    for _ in range(n):
        for d, s in zip(xs, src):
            d.copy_(s)
        ctx.flush.fill_(3.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(ctx.stream)
        pe.pe_polar_batched(xs, table, dtype, flags=flags)
        b.record(ctx.stream)
        b.synchronize()
        tot += a.elapsed_time(b)
    return tot / n


def measure(ctx, wl, table, dtype, steps, warmup, flags=0, peaks=None, fp32_peak=None, clocks=True):
    """The timed region (``steps`` grouped calls on resident inputs, each
    restored and followed by an L2 flush outside the step's events), a traced
    pass for the per-kernel roofline, and the end-to-end pass through the
    host-buffer entry."""
    torch, pe = ctx.torch, ctx.pe
    T = len(table)
    flops = algorithmic_flops(wl.shapes, T)
    xs = [d.clone() for d in wl.dev_in]
    in_bytes = sum(d.numel() * 4 for d in wl.dev_in)

    def restore():
        for d, s in zip(xs, wl.dev_in):
            d.copy_(s, non_blocking=True)

    for _ in range(warmup):
        restore()
        ctx.flush.fill_(1.0)
        pe.pe_polar_batched(xs, table, dtype, flags=flags)
    pe.pe_sync_status()
    sampler = ClockSampler(ctx.local)
    if clocks and ctx.rank == 0:
        sampler.start()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    ctx.barrier()
    l0 = pe.pe_launch_count()
    wall0 = time.perf_counter()
    for k in range(steps):
        restore()
        ctx.flush.fill_(1.0)
        evs[k][0].record(ctx.stream)
        pe.pe_polar_batched(xs, table, dtype, flags=flags)
        evs[k][1].record(ctx.stream)
    ctx.barrier()
    wall = time.perf_counter() - wall0
    launches = pe.pe_launch_count() - l0
    pe.pe_sync_status()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    dev_ms = ctx.max_over_ranks(sum(step_ms))
    ms_per_step = dev_ms / steps
    value = flops * steps / (dev_ms * 1e-3) / 1e12

    # per-kernel trace pass (CUDA events around each launch on the call's stream)
    pe.pe_trace_enable(True)
    for _ in range(steps):
        restore()
        ctx.flush.fill_(1.0)
        pe.pe_polar_batched(xs, table, dtype, flags=flags)
    trace = pe.pe_trace_read()
    pe.pe_trace_enable(False)
    pe.pe_sync_status()

    # end-to-end pass: pinned host inputs and outputs, copies inside the timed region
    host_in = [torch.from_numpy(np.ascontiguousarray(h, dtype=np.float32)).pin_memory() for h in wl.host()]
    host_out = [torch.empty_like(h).pin_memory() for h in host_in]
    e2e_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for _ in range(max(1, warmup)):   # builds and tunes the per-group plans outside the timed region
        pe.pe_polar_batched_host(host_in, host_out, table, dtype)
    ctx.barrier()
    for k in range(steps):
        ctx.flush.fill_(1.0)
        e2e_ev[k][0].record(ctx.stream)
        pe.pe_polar_batched_host(host_in, host_out, table, dtype)
        e2e_ev[k][1].record(ctx.stream)
    ctx.barrier()
    e2e_ms = ctx.max_over_ranks(sum(a.elapsed_time(b) for a, b in e2e_ev))
    clk = sampler.stop() if (clocks and ctx.rank == 0) else None
    pe.pe_sync_status()
    del host_in, host_out
    roof = roofline_line(trace, wl.shapes, dtype, flops / T, in_bytes, wl.name, peaks or measured_peaks(),
                         fp32_peak)
    return {
        "value": value, "ms_per_step": ms_per_step, "us_per_muon_step_median": 1e3 * statistics.median(step_ms),
        "us_per_poly_step": 1e3 * ms_per_step / T, "wall_s_timed": wall, "gpu_launches": int(launches),
        "flops_per_step": flops, "in_bytes": in_bytes, "xs": xs,
        "e2e": {"value": flops * steps / (e2e_ms * 1e-3) / 1e12, "unit": "TFLOP/s", "h2d_bytes_per_step": in_bytes,
                "d2h_bytes_per_step": in_bytes, "ms_per_step": e2e_ms / steps},
        "roofline": roof, "trace": {k: {"launches": v[0], "ms_total": v[1]} for k, v in trace.items()},
        "clocks": clk,
    }


def matmul_peaks(torch, n=8192, reps=6):
    """cuBLAS rates on this GPU at n^3: FP32 with TF32 off (the SIMT rate the
    plain FP32 path is measured against), FP32 with TF32 on, BF16."""
    out = {}
    old = torch.backends.cuda.matmul.allow_tf32
    try:
        for name, dt, tf32 in (("fp32_simt", torch.float32, False), ("tf32", torch.float32, True),
                               ("bf16", torch.bfloat16, False)):
            torch.backends.cuda.matmul.allow_tf32 = tf32
            a = torch.randn(n, n, device="cuda").to(dt)
            b = torch.randn(n, n, device="cuda").to(dt)
            for _ in range(2):
                torch.matmul(a, b)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                torch.matmul(a, b)
            e1.record()
            e1.synchronize()
            ms = e0.elapsed_time(e1) / reps
            out[name + "_tflops"] = 2.0 * n ** 3 / (ms * 1e-3) / 1e12
            del a, b
    finally:
        torch.backends.cuda.matmul.allow_tf32 = old
    out["n"] = n
    torch.cuda.empty_cache()
    return out


NS5_ROW = (15.0 / 8.0, -10.0 / 8.0, 3.0 / 8.0)   # the fixed Newton-Schulz quintic (Sec. 2)


def listing_steps(torch, wl, table):
    """The paper's online code (App. A) in PyTorch: X, A and B stored in BF16,
    one batched product call per product for each stack of same-shape
    matrices, the combinations b A + c A A and a X + B X folded into the
    product calls (baddbmm's beta and alpha). Returns (run, outputs)."""
    groups = {}
    for i, sh in enumerate(wl.shapes):
        groups.setdefault(sh, []).append(i)
    stacks = [(sh, idx, torch.stack([wl.dev_in[i] for i in idx])) for sh, idx in groups.items()]
    outs = [torch.empty_like(G) for _, _, G in stacks]
    coef = [tuple(float(v) for v in row) for row in table]

    def one(G, tall):
        nrm = torch.linalg.vector_norm(G, dim=(1, 2), keepdim=True)
        X = (G / (1.01 * nrm + 1e-7)).to(torch.bfloat16)
        if tall:
            X = X.mT
        for a, b, c in coef:
            A = torch.bmm(X, X.mT)
            B = torch.baddbmm(A, A, A, beta=b, alpha=c)
            X = torch.baddbmm(X, B, X, beta=a, alpha=1.0)
        return X.mT if tall else X

    return stacks, outs, one


def listing_line(ctx, wl, table, ours_ms, compiled, n=5):
    """The App. A listing on the same inputs, either eager cuBLAS calls
    replayed from a CUDA graph or under torch.compile; time per Muon step."""
    torch = ctx.torch
    stacks, outs, one = listing_steps(torch, wl, table)
    kind = "torch bmm/baddbmm (cuBLAS) in BF16 per same-shape stack, CUDA graph"
    try:
        if compiled:
            fn = torch.compile(one, dynamic=False)
            kind = "the App. A listing under torch.compile (default mode), BF16 per same-shape stack"

            def run():
                for (sh, _, G), out in zip(stacks, outs):
                    out.copy_(fn(G, sh[0] > sh[1]))
            for _ in range(3):
                run()
            torch.cuda.synchronize()
            replay = run
        else:
            def run():
                for (sh, _, G), out in zip(stacks, outs):
                    out.copy_(one(G, sh[0] > sh[1]))
            side = torch.cuda.Stream()
            side.wait_stream(ctx.stream)
            with torch.cuda.stream(side):
                for _ in range(3):
                    run()
            ctx.stream.wait_stream(side)
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph):
                run()
            replay = graph.replay
        replay()
        tot = 0.0
        for _ in range(n):
            ctx.flush.fill_(3.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(ctx.stream)
            replay()
            b.record(ctx.stream)
            b.synchronize()
            tot += a.elapsed_time(b)
        ms = tot / n
    except Exception as e:   # noqa: BLE001 - a comparison point only
        return {"unavailable": f"{type(e).__name__}: {str(e).splitlines()[0][:200] if str(e) else ''}", "kind": kind}
    res = {"value": algorithmic_flops(wl.shapes, len(table)) / (ms * 1e-3) / 1e12, "unit": "TFLOP/s",
           "ms_per_step": ms, "T": len(table), "kind": kind, "speedup_of_this_library": ms / ours_ms}
    if wl.facs is not None:
        xs = []
        for (sh, idx, _), out in zip(stacks, outs):
            for k in range(len(idx)):
                xs.append((idx[k], out[k]))
        xs.sort(key=lambda t: t[0])
        res["restricted_max_sigma_err"] = restricted_err(torch, [x for _, x in xs], wl.facs)
    del stacks, outs
    torch.cuda.empty_cache()
    return res


def _rel_fro(X, Y):
    return float(np.linalg.norm(X - Y) / np.linalg.norm(Y))


def _err_fro(X, P):
    return float(np.linalg.norm(X - P) / np.sqrt(min(X.shape)))


def _max_sigma_err(X):
    return float(np.max(np.abs(np.linalg.svd(X, compute_uv=False) - 1.0)))


def accuracy_sample(wl, table, xs, k=4):
    """First matrix of each distinct shape (up to k): relative Frobenius
    distance to the FP64 iterate (the oracle's spectral form where the factors
    are known, else its iteration on the FP32-cast input), error against the
    true factor and max|sigma - 1|."""
    import oracle as O
    seen = {}
    for i, sh in enumerate(wl.shapes):
        seen.setdefault(sh, i)
    rows = []
    for i in list(seen.values())[:k]:
        got = xs[i].cpu().numpy().astype(np.float64)
        sv = wl.svd[i] if wl.svd else None
        if sv is not None:
            ref, P = O.polar_express_spectral(sv.U, sv.s, sv.V, table), sv.U @ sv.V.T
        else:
            G = wl.host()[i].astype(np.float64)
            ref, P = O.polar_express(G, table), O.polar_svd(G)
        rows.append({"shape": list(wl.shapes[i]), "rel_fro_vs_fp64_iteration": _rel_fro(got, ref),
                     "err_fro_per_sqrt_n": _err_fro(got, P), "max_sigma_err": _max_sigma_err(got),
                     "fp64_max_sigma_err": _max_sigma_err(ref)})
    return rows


def large_extras(ctx, wl, table, res, dtype, peaks, mm, args):
    """Large dense set: restricted max|sigma - 1| of the BF16 result, the plain
    FP32 path at the same T, and the smallest BF16 T whose restricted error is
    no larger than FP32's (speed-up at equal error)."""
    torch, pe = ctx.torch, ctx.pe
    out = {}
    e16 = restricted_err(torch, res["xs"], wl.facs)
    xs = [d.clone() for d in wl.dev_in]
    ms32 = time_calls(ctx, xs, wl.dev_in, table, "fp32", 2)
    e32 = restricted_err(torch, xs, wl.facs)
    t16, ms16, err16 = wl.T, res["ms_per_step"], e16
    tries = []
    while err16 > 1.05 * e32 + 1e-4 and t16 < wl.T + 4:
        t16 += 1
        tab16 = pe.pe_coeffs(5, wl.l, t16, 1.01)
        ms16 = time_calls(ctx, xs, wl.dev_in, tab16, dtype, 3)
        err16 = restricted_err(torch, xs, wl.facs)
        tries.append({"T": t16, "ms": ms16, "restricted_max_sigma_err": err16})
    f = algorithmic_flops(wl.shapes, wl.T)
    fp32 = {"value": f / (ms32 * 1e-3) / 1e12, "unit": "TFLOP/s", "ms_per_step": ms32, "T": wl.T,
            "restricted_max_sigma_err": e32}
    if mm and mm.get("fp32_simt_tflops"):
        fp32["frac_of_measured_fp32_simt"] = fp32["value"] / mm["fp32_simt_tflops"]
    out["fp32_plain"] = fp32
    out["accuracy"] = {"restricted_max_sigma_err_bf16": e16, "restricted_max_sigma_err_fp32": e32,
                       "gamma": 1e-3, "note": "max|sigma_i - 1| over the directions with s_i >= 1e-3 s_max "
                                               "(singular values of U1^T X V1)"}
    out["speedup_vs_fp32_plain"] = {"value": ms32 / ms16, "T_bf16": t16, "T_fp32": wl.T,
                                    "restricted_max_sigma_err_bf16": err16,
                                    "restricted_max_sigma_err_fp32": e32, "equal_error": bool(err16 <= 1.05 * e32 + 1e-4),
                                    "search": tries}
    tab_ns = np.array([NS5_ROW] * wl.T)
    ms_ns = time_calls(ctx, xs, wl.dev_in, tab_ns, dtype, 3)
    out["newton_schulz5"] = {"value": f / (ms_ns * 1e-3) / 1e12, "unit": "TFLOP/s", "ms_per_step": ms_ns, "T": wl.T,
                             "dtype": dtype, "restricted_max_sigma_err": restricted_err(torch, xs, wl.facs)}
    del xs
    torch.cuda.empty_cache()
    return out


def small_extras(ctx, wl, table, res, dtype, args):
    """Workloads generated on the CPU: accuracy sample against the FP64
    oracle, the FP32 path, the Newton-Schulz quintic through the same
    kernels."""
    torch, pe = ctx.torch, ctx.pe
    out = {"accuracy": {dtype: accuracy_sample(wl, table, res["xs"])}}
    xs = [d.clone() for d in wl.dev_in]
    n = max(3, min(20, args.steps // 5))
    ms32 = time_calls(ctx, xs, wl.dev_in, table, "fp32", n)
    out["accuracy"]["fp32"] = accuracy_sample(wl, table, xs)
    f = algorithmic_flops(wl.shapes, wl.T)
    w16 = max(r["max_sigma_err"] for r in out["accuracy"][dtype])
    w32 = max(r["max_sigma_err"] for r in out["accuracy"]["fp32"])
    out["fp32_plain"] = {"value": f / (ms32 * 1e-3) / 1e12, "unit": "TFLOP/s", "ms_per_step": ms32, "T": wl.T,
                         "max_sigma_err_sample": w32}
    # both paths apply the same table, so at equal T the BF16 error must
    # not exceed the FP32 one by more than 5%
    out["speedup_vs_fp32_plain"] = {"value": ms32 / res["ms_per_step"], "T_bf16": wl.T, "T_fp32": wl.T,
                                    "max_sigma_err_bf16": w16, "max_sigma_err_fp32": w32,
                                    "equal_error": bool(w16 <= 1.05 * w32 + 1e-4)}
    tab_ns = np.array([NS5_ROW] * wl.T)
    ms_ns = time_calls(ctx, xs, wl.dev_in, tab_ns, dtype, n)
    errs = [_max_sigma_err(xs[r].cpu().numpy().astype(np.float64)) for r in range(min(4, len(xs)))]
    out["newton_schulz5"] = {"value": f / (ms_ns * 1e-3) / 1e12, "unit": "TFLOP/s", "ms_per_step": ms_ns, "T": wl.T,
                             "dtype": dtype, "max_sigma_err_first4": max(errs)}
    del xs
    return out


def side_line(ctx, name, args, peaks, fp32_peak, cpu_budget):
    """Another workload, measured the same way (own roofline, e2e, CPU
    baseline), for the ``gpt2_small`` key of the headline line."""
    wl = load_workload(name, ctx.torch)
    table = ctx.pe.pe_coeffs(5, wl.l, wl.T, 1.01)
    res = measure(ctx, wl, table, "bf16", args.steps, args.warmup, peaks=peaks, fp32_peak=fp32_peak, clocks=False)
    line = {k: res[k] for k in ("value", "ms_per_step", "us_per_muon_step_median", "us_per_poly_step", "gpu_launches",
                                 "e2e", "roofline", "trace")}
    line.update({"unit": "TFLOP/s", "config": {"workload": wl.name, "matrices": len(wl.shapes), "T": wl.T, "l": wl.l,
                                               "flops_per_step": res["flops_per_step"], "note": wl.note}})
    line["cpu_baseline"] = cpu_baseline_line(wl.host(), table, cpu_budget, wl.name)
    line.update(small_extras(ctx, wl, table, res, "bf16", args))
    line["torch_cublas_bf16"] = listing_line(ctx, wl, table, res["ms_per_step"], compiled=False)
    del res["xs"]
    return line


def error_sweep(ctx, wl, Ts=(2, 4, 6, 8, 10, 12), gamma=1e-3):
    """Error against the truth U V^T vs iteration count T and vs time, for the
    Polar Express tables (FP32 plain, BF16, BF16x3) and the Newton-Schulz
    quintic (BF16), on a workload with known factors. Errors per T: the
    largest over the workload's matrices of max|sigma_i - 1| restricted to the
    directions with s_i >= gamma s_max (singular values of U1^T X V1, FP64 on
    the GPU) and of ||X - U V^T||_F / sqrt(n)."""
    torch, pe = ctx.torch, ctx.pe
    kept = []
    for sv in wl.svd:
        k = sv.s >= gamma * sv.s.max()
        U = torch.from_numpy(sv.U).cuda()
        V = torch.from_numpy(sv.V).cuda()
        kept.append((U[:, k].contiguous(), V[:, k].contiguous(), U, V))
    rows = []
    for T in Ts:
        for path in ("fp32", "bf16", "bf16x3", "ns5"):
            table = np.array([NS5_ROW] * T) if path == "ns5" else pe.pe_coeffs(5, wl.l, T, 1.01)
            dt = "bf16" if path == "ns5" else path
            xs = [d.clone() for d in wl.dev_in]
            ms = time_calls(ctx, xs, wl.dev_in, table, dt, 3)
            rmax, efro = 0.0, 0.0
            for X, (U1, V1, U, V) in zip(xs, kept):
                Xd = X.double()
                sig = torch.linalg.svdvals(U1.T @ Xd @ V1)
                rmax = max(rmax, float((sig - 1).abs().max()))
                efro = max(efro, float(torch.linalg.norm(Xd - U @ V.T) / np.sqrt(min(X.shape))))
            rows.append({"path": path, "T": T, "ms": ms, "restricted_max_sigma_err": rmax,
                         "err_fro_per_sqrt_n": efro})
            del xs
    return {"gamma": gamma, "rows": rows}


def spectrum_bound_line(pe, wl, iters=10):
    """Cost of the App. H bound (the power method, ``iters`` steps, on G) for
    one matrix of each distinct shape: host wall time of the blocking call
    (its buffers, about five launches per step and the read-back of z), and
    z / f, which decides whether the cubic applies (z / f > 1 / sqrt 2)."""
    seen = {}
    for i, sh in enumerate(wl.shapes):
        seen.setdefault(sh, i)
    rows = []
    for sh, i in list(seen.items())[:4]:
        v0 = np.random.default_rng(i).standard_normal(min(sh)).astype(np.float32)
        pe.pe_spectrum_bound(wl.dev_in[i], v0, iters)
        t0 = time.perf_counter()
        z, f = pe.pe_spectrum_bound(wl.dev_in[i], v0, iters)
        rows.append({"shape": list(sh), "ms": 1e3 * (time.perf_counter() - t0), "z_over_f": z / f if f else None})
    return {"iters": iters, "rows": rows}


def fast_rectangular_line(ctx, n=1024, alphas=(4, 8, 32), T=6, reps=3):
    """Alg. 4 (fast rectangular iteration, FP32 path) against the ordinary
    FP32 iteration on n x (alpha n) Gaussian matrices, T degree-5 steps
    (the paper's runtime comparison of restart intervals T, 3 and 1): time
    per call with inputs resident, after an L2 flush, and its ratio."""
    torch, pe = ctx.torch, ctx.pe
    table = pe.pe_coeffs(5, 1e-3, T, 1.01)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(12)

    def timed(fn, x, src):
        for _ in range(2):
            x.copy_(src)
            fn(x)
        tot = 0.0
        for _ in range(reps):
            x.copy_(src)
            ctx.flush.fill_(5.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(ctx.stream)
            fn(x)
            b.record(ctx.stream)
            b.synchronize()
            tot += a.elapsed_time(b)
        return tot / reps

    rows = []
    for al in alphas:
        G = torch.randn(n, al * n, device="cuda", generator=gen)
        x = G.clone()
        base = timed(lambda t: pe.pe_polar_batched([t], table, "fp32", flags=pe.PE_BATCH_NO_GRAPH), x, G)
        bf16 = timed(lambda t: pe.pe_polar_batched([t], table, "bf16", flags=pe.PE_BATCH_NO_GRAPH), x, G)
        row = {"shape": [n, al * n], "alpha": al, "T": T, "fp32_ordinary_ms": base, "bf16_ordinary_ms": bf16}
        for rs in (3, T):
            ms = timed(lambda t: pe.pe_polar_fast_batched([t], table, restart=rs, flags=pe.PE_BATCH_NO_GRAPH), x, G)
            row[f"fast_restart{rs}_ms"] = ms
            row[f"speedup_restart{rs}_vs_fp32_ordinary"] = base / ms
        rows.append(row)
        del G, x
    torch.cuda.empty_cache()
    return {"path": "fp32 (SIMT) products; Gaussian inputs", "rows": rows}


# ------------------------------------------------------------------ multi-GPU

def run_multi(ctx, args, dtype, peaks):
    """N GPUs, one process each. The matrices are independent problems, so
    the timed run shards units with no exchange: every rank owns a set of
    the workload's shape (its own seeds), runs the single-GPU measurement on
    it (CUDA events, barrier + synchronize around the timed region, max over
    ranks) and the value is the units of all ranks over that time (weak
    scaling). Beside it, the distributed-Muon form of one shared set: LPT
    ownership of whole matrices and one NCCL all-gather of the results per
    step (shard.polar_sharded), timed with the exchange inside. Rank 0
    prints the line."""
    from paper_2505_16932_gb300 import shard
    torch, pe = ctx.torch, ctx.pe
    wl = load_workload(args.workload, torch, ctx.rank)
    table = pe.pe_coeffs(5, wl.l, wl.T, 1.01)
    res = measure(ctx, wl, table, dtype, args.steps, args.warmup, 0, peaks)
    res.pop("xs", None)
    flops = res["flops_per_step"]
    value = ctx.world * res["value"]
    e2e = dict(res["e2e"])
    e2e["value"] = ctx.world * e2e["value"]
    e2e["note"] = "every rank through pe_polar_batched_host on its own pinned buffers; bytes per rank"
    del wl
    torch.cuda.empty_cache()

    # distributed-Muon exchange: one set shared by all ranks (rank 0's seeds)
    ws = load_workload(args.workload, torch, 0)
    xs = [d.clone() for d in ws.dev_in]
    owners = shard.assign(ws.shapes, ctx.world, len(table))
    fl_set = algorithmic_flops(ws.shapes, len(table))

    def restore():
        for d, s0 in zip(xs, ws.dev_in):
            d.copy_(s0)
        ctx.flush.fill_(1.0)

    for _ in range(args.warmup):
        restore()
        shard.polar_sharded(xs, table, dtype)
    ctx.barrier()
    tot = 0.0
    for _ in range(args.steps):
        restore()
        ctx.barrier()
        t0 = time.perf_counter()
        shard.polar_sharded(xs, table, dtype)
        torch.cuda.synchronize()
        tot += time.perf_counter() - t0
    ex_ms = ctx.max_over_ranks(1e3 * tot / args.steps)
    pe.pe_sync_status()
    if ctx.rank != 0:
        return 0
    line = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": ctx.world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic",
            "config": {"workload": ws.name, "matrices": len(ws.shapes), "matrices_all_ranks": ctx.world * len(ws.shapes),
                       "T": ws.T, "l": ws.l,
                       "parallelism": f"{ctx.world} ranks, one set of the workload per rank (own seeds), "
                                      "no collective in the timed region",
                       "flops_per_step_per_rank": flops,
                       "l2": "inputs larger than L2 and a 258 MB L2 flush before each step"},
            "gpu_launches": res["gpu_launches"], "e2e": e2e, "roofline": res["roofline"], "trace": res["trace"],
            "clocks": res["clocks"],
            "sharded_exchange": {
                "value": fl_set / (ex_ms * 1e-3) / 1e12, "unit": "TFLOP/s", "ms_per_step": ex_ms,
                "scaling": "strong", "owners": owners,
                "what": "one set over the ranks: LPT ownership of whole matrices, one grouped call per rank, "
                        "one NCCL all-gather of the results; host clock between barriers, max over ranks"}}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ main

def role_cycles(ctx, wl, table, dtype):
    """Per-role cycle counters of the tcgen05 step kernel (debug key 4) over
    one grouped call, as fractions of the kernel's own cycles, averaged over
    the persistent CTAs: where the producer, MMA and epilogue warps spend their
    time (a diagnostic, printed instead of the bench line)."""
    torch, pe = ctx.torch, ctx.pe
    xs = [m.clone() for m in wl.dev_in]
    src = [x.clone() for x in xs]
    for _ in range(3):
        for d, s in zip(xs, src):
            d.copy_(s)
        pe.pe_polar_batched(xs, table, dtype)
    torch.cuda.synchronize()
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    prof = torch.zeros(32 * 4096, dtype=torch.int64, device="cuda")
    pe.pe_debug_set(4, prof.data_ptr())
    try:
        for d, s in zip(xs, src):
            d.copy_(s)
        pe.pe_polar_batched(xs, table, dtype)
        torch.cuda.synchronize()
    finally:
        pe.pe_debug_set(4, 0)
    pe.pe_sync_status()
    P = prof.view(4096, 32)[:nsm].double().cpu().numpy()
    names = {0: "total", 11: "producer", 1: "producer_wait_dependency", 2: "producer_wait_free_stage",
             12: "mma", 3: "mma_wait_operands", 4: "mma_wait_free_accumulator",
             5: "epilogue_wait_accumulator", 9: "epilogue_wait_dependency", 6: "epilogue_gram_tiles",
             7: "epilogue_square_tiles", 8: "epilogue_update_tiles", 18: "update_tmem_load",
             14: "update_wait_prefetched_operand", 13: "update_operand_read_and_arithmetic",
             10: "update_wait_output_box", 15: "update_output_staging", 16: "update_proxy_fence",
             17: "update_store_and_prefetch_issue"}
    tot = P[:, 0].mean()
    # 2-SM UMMA: only the even CTA of a pair issues MMAs, so the MMA slots
    # average over the CTAs that recorded any
    issuers = P[:, 12] > 0
    frac = {}
    for k, v in names.items():
        rows = P[issuers, k] if k in (3, 4, 12) and issuers.any() else P[:, k]
        frac[v] = float(rows.mean() / tot)
    return {"workload": wl.name, "dtype": dtype, "ctas": nsm, "mma_issuing_ctas": int(issuers.sum()),
            "fractions_of_kernel_cycles": frac}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large_dense", choices=WORKLOADS)
    ap.add_argument("--dtype", default=None, choices=["fp32", "bf16", "bf16x3"])
    ap.add_argument("--phased", action="store_true", help="three grouped launches per step")
    ap.add_argument("--no-extras", action="store_true",
                    help="only the timed line (no comparisons, accuracy, side workload)")
    ap.add_argument("--no-compile", action="store_true", help="skip the torch.compile run of the App. A listing")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--sweep", action="store_true",
                    help="error vs iteration count and vs time for FP32, BF16, BF16x3 and Newton-Schulz "
                         "(workloads with known factors)")
    ap.add_argument("--role-cycles", action="store_true",
                    help="print the step kernel's per-role cycle fractions (debug counters) instead of timing")
    args = ap.parse_args()
    if args.steps < 1:
        ap.error("--steps must be >= 1")
    args.warmup = max(args.warmup, 3)   # at least 3 untimed warm-up steps

    world, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, world, rank)

    import torch
    import paper_2505_16932_gb300 as pe
    from paper_2505_16932_gb300 import build as B

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    B.build()
    pe.lib()
    ctx = Ctx(pe, torch, world, rank, local)
    dtype = args.dtype or ("fp32" if args.workload == "plain_small" else "bf16")
    if world > 1:
        return run_multi(ctx, args, dtype, measured_peaks())
    wl = load_workload(args.workload, torch)
    table = pe.pe_coeffs(5, wl.l, wl.T, 1.01)
    if args.role_cycles:
        print(json.dumps(role_cycles(ctx, wl, table, dtype)))
        return 0
    peaks = measured_peaks()
    flags = pe.PE_BATCH_PHASED if args.phased else 0

    mm = None if args.no_extras else matmul_peaks(torch)
    fp32_peak = mm["fp32_simt_tflops"] if mm else None
    res = measure(ctx, wl, table, dtype, args.steps, args.warmup, flags, peaks, fp32_peak)
    cpu = cpu_baseline_line(wl.host(), table, args.cpu_budget, wl.name)
    extras = {}
    if not args.no_extras:
        if wl.facs is not None:
            extras.update(large_extras(ctx, wl, table, res, dtype, peaks, mm, args))
        else:
            extras.update(small_extras(ctx, wl, table, res, dtype, args))
        extras["torch_cublas_bf16"] = listing_line(ctx, wl, table, res["ms_per_step"], compiled=False)
        extras["torch_compile_bf16"] = (listing_line(ctx, wl, table, res["ms_per_step"], compiled=True)
                                        if not args.no_compile else {"skipped": "--no-compile"})
        extras["matmul_peaks"] = mm
        if args.workload == "large_dense":
            del res["xs"]
            extras["gpt2_small"] = side_line(ctx, "gpt2_small", args, peaks, fp32_peak, 5.0)
            extras["spectrum_bound"] = spectrum_bound_line(pe, load_workload("gpt2_small", torch))
        extras["fast_rectangular"] = fast_rectangular_line(ctx)
        if args.sweep or args.workload == "ill_conditioned":
            extras["error_vs_T"] = error_sweep(ctx, wl)
    res.pop("xs", None)
    line = {
        "metric": METRIC, "value": res["value"], "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": res["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": dtype, "data": "synthetic",
        "config": {"workload": wl.name, "matrices": len(wl.shapes), "T": wl.T, "l": wl.l,
                   "path": dtype + (" grouped phased" if args.phased
                                    else " grouped persistent (one launch per step), CUDA graph"),
                   "flops_per_step": res["flops_per_step"],
                   "dense_equiv_flops_per_step": dense_equiv_flops(wl.shapes, wl.T),
                   "input_bytes": res["in_bytes"],
                   "l2": "inputs larger than L2 and a 258 MB L2 flush before each step", "note": wl.note},
        "us_per_muon_step": 1e3 * res["ms_per_step"],
        "us_per_muon_step_median": res["us_per_muon_step_median"],
        "us_per_poly_step": res["us_per_poly_step"],
        "wall_s_timed": res["wall_s_timed"],
        "gpu_launches": res["gpu_launches"],
        "e2e": res["e2e"],
        "roofline": res["roofline"],
        "trace": res["trace"],
        "clocks": res["clocks"],
        "cpu_baseline": cpu,
    }
    line.update(extras)
    print(json.dumps(line))
    return 0


if __name__ == "__main__":
    sys.exit(main())
