#!/usr/bin/env python3
"""Benchmark of the Polar Express online stage on GB300.

One "step" is one Muon orthogonalisation step of the workload: every matrix
of the model normalised and taken through T polynomial steps by one
``pe_polar_batched`` call (prepare launch + one persistent grouped tcgen05
launch per polynomial step, replayed from a CUDA graph).

Reported ``value``: algorithmic polar TFLOP/s, sum over matrices of
T (3 s^2 L + s^3) per step (s = min(m, n), L = max(m, n); the Gram and A^2
products are symmetric and counted once), divided by the device time of the
step, with inputs resident in HBM. ``e2e`` repeats the measurement with the
inputs copied from pinned host memory and the factors copied back inside the
timed region. ``roofline`` attributes device time to the dominant kernel
from CUDA events bracketing each launch (library tracing) over the same
steps. ``cpu_baseline`` times the FP64 oracle on the host cores on a bounded
sample.

Launch: ``python bench.py [--gpus N] [--steps K] [--warmup W]``; for N > 1
under torchrun, each rank runs its own copy of the workload (weak scaling)
and rank 0 prints the line. ``--impl reference`` times the FP64 oracle on
the host (the reference arm).
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
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

METRIC = "polar TFLOP/s & µs/Muon-step, BF16 grouped vs FP32 plain at equal max|σ−1|"
L2_BYTES = 129 * 1024 * 1024

WORKLOADS = {
    "gpt2_small": lambda: synth.gpt2_small(),
    "uneven_d1024": lambda: synth.uneven_d1024(),
    "gpt2_heads": lambda: synth.gpt2_heads(),
    "large_dense": lambda: synth.large_dense(),
    "ill_conditioned": lambda: synth.ill_conditioned(),
    "plain_small": lambda: synth.plain_small(),
}


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


def accuracy_sample(wl):
    """Indices of the accuracy sample: the first matrix of each distinct shape (up to 4)."""
    seen = {}
    for i, sh in enumerate(wl.shapes):
        seen.setdefault(sh, i)
    return list(seen.values())[:4]


def cpu_baseline_leg(wl, table, budget_s: float, acc_idx):
    """The leg of this script that runs the FP64 oracle: its timing on the
    host cores (oracle_sample) and the FP64 iterates of the accuracy sample
    (the spectral form where the factors are known, else the iteration on the
    FP32-cast input), with the true polar factors. Returns (timing, refs)."""
    import oracle as O
    refs = {}
    for i in acc_idx:
        sv = wl.svd[i]
        if sv is not None:
            refs[i] = (O.polar_express_spectral(sv.U, sv.s, sv.V, table), sv.U @ sv.V.T)
        else:
            G = wl.matrices[i]
            refs[i] = (O.polar_express(G.astype(np.float32).astype(np.float64), table), O.polar_svd(G))
    return oracle_sample(wl, table, budget_s), refs


def oracle_sample(wl, table, budget_s: float):
    """Time the FP64 oracle iteration over the workload's matrices in order
    until `budget_s` has elapsed (at least one matrix). Returns
    (TFLOP/s, seconds, matrices done)."""
    import oracle as O
    done = 0
    flops = 0.0
    t0 = time.perf_counter()
    for G in wl.matrices:
        # a matrix whose full iteration would overrun the budget (at an
        # assumed 100 GFLOP/s FP64) is sampled with its first step only
        steps = len(table)
        if dense_equiv_flops([G.shape], steps) / 1e11 > max(budget_s, 1.0):
            steps = 1
        O.polar_express(G, table[:steps])
        done += 1
        flops += algorithmic_flops([G.shape], steps)
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    return flops / dt / 1e12, dt, done


# ------------------------------------------------------------------ main

def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_reference(args, wl, world, rank):
    if rank != 0:
        return 0
    import oracle as O
    table, _ = O.optimal_composition(wl.l, wl.T, safety=1.01)
    # each step: one matrix (cycling) through the FP64 iteration
    n = len(wl.matrices)
    for i in range(args.warmup):
        oracle_sample(synth.Workload(wl.name, [wl.matrices[i % n]], [None], wl.l, wl.T, wl.dtype), table, 0.0)
    tot_f, tot_t = 0.0, 0.0
    for i in range(args.steps):
        G = wl.matrices[i % n]
        t0 = time.perf_counter()
        O.polar_express(G, table)
        tot_t += time.perf_counter() - t0
        tot_f += algorithmic_flops([G.shape], wl.T)
    val = tot_f / tot_t / 1e12
    cores = cpu_cores()
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "TFLOP/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name, "T": wl.T, "l": wl.l, "matrices": n,
                   "step": "one matrix of the workload per step, cycling"},
        "cpu_baseline": {"value": val, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
                         "sample": f"FP64 numpy oracle iteration, one matrix of {wl.name} per step, T={wl.T}"},
        "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


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


def roofline_line(trace, shapes, dtype, flops_step, in_bytes, workload, peaks):
    """Roofline of the dominant kernel (largest traced time): algorithmic
    flops (or bytes) per launch over its mean CUDA-event launch time, against
    the measured burst peak (and the sustained one for tensor-bound kernels);
    DRAM traffic from the committed ncu figure while the source matches."""
    dom_name, (dom_n, dom_ms) = max(trace.items(), key=lambda kv: kv[1][1])
    dom_avg_ms = dom_ms / dom_n
    tot_trace_ms = sum(v[1] for v in trace.values())
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
            # FP32 SIMT roof: 152 SMs x 128 FP32 lanes x 2 flop x max SM clock
            peak, unit, bound = 152 * 128 * 2 * peaks["sm_max_mhz"] * 1e6 / 1e12, "TFLOP/s", "alu"
        else:
            peak, unit, bound = peaks["bf16_tflops"], "TFLOP/s", "tensor"
    else:
        achieved = in_bytes * 2 / (dom_avg_ms * 1e-3) / 1e9
        peak, unit, bound = peaks["hbm_gbs"], "GB/s", "hbm"
    roofline = {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit, "frac": achieved / peak,
                "traffic": committed_traffic(workload, dom_name), "kernel": dom_name, "kernel_ms_avg": dom_avg_ms,
                "launches_traced": dom_n, "share_of_step": dom_ms / tot_trace_ms,
                "peak_source": peaks["source"] + " burst",
                "algorithmic_bytes_per_launch_bf16": algorithmic_bytes_bf16(shapes, 1)}
    if bound == "tensor":
        roofline["peak_sustained"] = peaks["bf16_tflops_sustained"]
        roofline["frac_sustained"] = achieved / peaks["bf16_tflops_sustained"]
    return roofline


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="gpt2_small", choices=sorted(WORKLOADS))
    ap.add_argument("--dtype", default=None, choices=["fp32", "bf16", "bf16x3"])
    ap.add_argument("--phased", action="store_true", help="three grouped launches per step")
    ap.add_argument("--no-extras", action="store_true", help="skip the FP32 comparison and accuracy sample")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--no-largest", action="store_true", help="skip the largest-configuration measurement")
    ap.add_argument("--sweep", action="store_true",
                    help="error vs iteration count and vs time for FP32, BF16, BF16x3 and Newton-Schulz "
                         "(ill-conditioned workload)")
    args = ap.parse_args()
    if args.steps < 1:
        ap.error("--steps must be >= 1")
    args.warmup = max(args.warmup, 3)   # at least 3 untimed warm-up steps

    world, rank, local = dist_setup()
    wl = WORKLOADS[args.workload]()
    if args.impl == "reference":
        return run_reference(args, wl, world, rank)

    import torch
    import paper_2505_16932_gb300 as pe
    from paper_2505_16932_gb300 import build as B

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    B.build()
    pe.lib()
    dtype = args.dtype or ("bf16" if wl.dtype != "fp32" else "fp32")
    table = pe.pe_coeffs(5, wl.l, wl.T, 1.01)
    shapes = wl.shapes
    T = wl.T
    flops = algorithmic_flops(shapes, T)
    flops_step = flops / T
    host_in = [torch.from_numpy(G.astype(np.float32)).pin_memory() for G in wl.matrices]
    host_out = [torch.empty_like(h).pin_memory() for h in host_in]
    dev_in = [h.to("cuda") for h in host_in]
    dev_x = [d.clone() for d in dev_in]
    in_bytes = sum(h.numel() * 4 for h in host_in)
    flush = torch.empty(max(2 * L2_BYTES, 256 << 20) // 4, dtype=torch.float32, device="cuda")
    flags = pe.PE_BATCH_PHASED if args.phased else 0
    stream = torch.cuda.current_stream()

    def restore():
        for d, s in zip(dev_x, dev_in):
            d.copy_(s, non_blocking=True)

    def one_step(evs=None):
        restore()
        flush.fill_(1.0)
        if evs:
            evs[0].record(stream)
        pe.pe_polar_batched(dev_x, table, dtype, flags=flags)
        if evs:
            evs[1].record(stream)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x):
        if world == 1:
            return x
        import torch.distributed as dist
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    for _ in range(args.warmup):
        one_step()
    pe.pe_sync_status()

    # ---------------------------------------------------- timed region
    sampler = ClockSampler(local)
    if rank == 0:
        sampler.start()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    l0 = pe.pe_launch_count()
    wall0 = time.perf_counter()
    for k in range(args.steps):
        one_step(evs[k])
    barrier()
    wall = time.perf_counter() - wall0
    launches = pe.pe_launch_count() - l0
    pe.pe_sync_status()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    dev_ms = max_over_ranks(sum(step_ms))
    ms_per_step = dev_ms / args.steps
    value = world * flops * args.steps / (dev_ms * 1e-3) / 1e12

    # ---------------------------------------------- per-kernel trace pass
    pe.pe_trace_enable(True)
    for k in range(args.steps):
        one_step()
    trace = pe.pe_trace_read()
    pe.pe_trace_enable(False)
    pe.pe_sync_status()

    # -------------------------------------------------- end-to-end pass
    e2e_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for _ in range(max(1, args.warmup)):   # builds and tunes the per-group plans outside the timed region
        pe.pe_polar_batched_host(host_in, host_out, table, dtype)
    torch.cuda.synchronize()
    barrier()
    for k in range(args.steps):
        flush.fill_(1.0)
        e2e_ev[k][0].record(stream)
        # the C ABI's host-buffer entry: copies in, grouped compute, copies
        # out, pipelined by the library across groups of matrices
        pe.pe_polar_batched_host(host_in, host_out, table, dtype)
        e2e_ev[k][1].record(stream)
    barrier()
    e2e_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in e2e_ev))
    e2e_value = world * flops * args.steps / (e2e_ms * 1e-3) / 1e12
    clocks = sampler.stop() if rank == 0 else None
    pe.pe_sync_status()

    # ---------------------------------------------------------- roofline
    roofline = roofline_line(trace, shapes, dtype, flops_step, in_bytes, wl.name, measured_peaks())

    # ------------------------------------------ extras (rank 0, N = 1 style)
    extras = {}
    cpu = None
    if rank == 0:
        acc_idx = [] if args.no_extras else accuracy_sample(wl)
        (tf, secs, done), refs = cpu_baseline_leg(wl, table, args.cpu_budget, acc_idx)
        if not args.no_extras:
            extras = accuracy_and_fp32(pe, torch, wl, table, dev_in, dtype, flush, stream, args, refs)
            extras["newton_schulz5"] = newton_schulz_line(pe, torch, wl, dev_in, dtype, flush, stream, refs, args)
            if dtype == "bf16":
                extras["torch_cublas_bf16"] = cublas_listing_line(torch, wl, table, dev_in, flush, stream, refs,
                                                                  ms_per_step, args)
            extras["spectrum_bound"] = spectrum_bound_line(pe, wl, dev_in)
        if args.sweep or wl.name == "ill_conditioned":
            extras["error_vs_T"] = error_sweep(pe, torch, wl, dev_in, flush, stream)
        if not args.no_largest and wl.name != "large_dense" and world == 1:
            extras["largest_config"] = largest_config(pe, torch, flush, stream, min(args.steps, 10))
        cpu = {"value": tf, "unit": "TFLOP/s", "cores": cpu_cores(), "kind": "oracle",
               "sample": f"FP64 numpy oracle iteration of the first {done} of {len(shapes)} matrices, "
                         f"T={T} ({secs:.1f} s)"}
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    if rank != 0:
        return 0
    line = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16" if dtype == "bf16" else dtype, "data": "synthetic",
        "config": {"workload": wl.name, "matrices": len(shapes), "T": T, "l": wl.l, "path": dtype +
                   (" grouped phased" if args.phased else " grouped persistent (one launch per step), CUDA graph"),
                   "flops_per_step": flops, "dense_equiv_flops_per_step": dense_equiv_flops(shapes, T),
                   "input_bytes": in_bytes, "l2": "inputs larger than L2 and a 258 MB L2 flush before each step",
                   "note": wl.note},
        "us_per_muon_step": 1e3 * ms_per_step,
        "us_per_muon_step_median": 1e3 * statistics.median(step_ms),
        "us_per_poly_step": 1e3 * ms_per_step / T,
        "wall_s_timed": wall,
        "gpu_launches": int(launches),
        "e2e": {"value": e2e_value, "unit": "TFLOP/s", "h2d_bytes_per_step": in_bytes, "d2h_bytes_per_step": in_bytes,
                "ms_per_step": e2e_ms / args.steps},
        "roofline": roofline,
        "trace": {k: {"launches": v[0], "ms_total": v[1]} for k, v in trace.items()},
        "clocks": clocks,
        "cpu_baseline": cpu,
    }
    worst = extras.pop("_worst", None)
    line.update(extras)
    if worst is not None:
        w16, w32, ms32 = worst
        # equal max|sigma - 1| at the same T: both paths apply the same table,
        # so the BF16 error must not exceed the FP32 one by more than 5%
        line["speedup_vs_fp32_plain"] = {
            "value": ms32 / ms_per_step, "T_bf16": T, "T_fp32": T, "max_sigma_err_bf16": w16,
            "max_sigma_err_fp32": w32, "equal_error": bool(w16 <= 1.05 * w32 + 1e-4)}
    print(json.dumps(line))
    return 0


def largest_config(pe, torch, flush, stream, steps):
    """The largest configuration (8192 x 8192, 4096 x 14336, 14336 x 4096;
    Haar U, V; s log-uniform in [1e-4, 1]; l = 1e-4, T = 6), generated on the
    GPU with a seeded torch generator (input plumbing only). Times the BF16
    grouped path and the FP32 plain path and compares their max|sigma - 1|
    restricted to sigma_i(G) >= 1e-3 sigma_max (computed on the GPU from the
    known factors: singular values of U1^T X V1)."""
    shapes = [(8192, 8192), (4096, 14336), (14336, 4096)]
    T, l = 6, 1e-4
    gen = torch.Generator(device="cuda")
    gen.manual_seed(3)
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
    table = pe.pe_coeffs(5, l, T, 1.01)
    flops = algorithmic_flops(shapes, T)
    out = {"workload": "large_dense_8192sq_4096x14336_14336x4096", "T": T, "l": l, "flops_per_step": flops}
    xs = [x.clone() for x in mats]

    def timed(path, tab, n):
        for _ in range(2):
            for d, s0 in zip(xs, mats):
                d.copy_(s0)
            pe.pe_polar_batched(xs, tab, path)
        tot = 0.0
        for _ in range(n):
            for d, s0 in zip(xs, mats):
                d.copy_(s0)
            flush.fill_(3.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            pe.pe_polar_batched(xs, tab, path)
            b.record(stream)
            b.synchronize()
            tot += a.elapsed_time(b)
        return tot / n

    def restricted_err():
        worst = 0.0
        for X, (U1, V1) in zip(xs, facs):
            C = U1.T @ X @ V1                  # FP32 (TF32 off)
            sv = torch.linalg.svdvals(C)
            worst = max(worst, float((sv - 1.0).abs().max()))
        return worst

    ms16 = timed("bf16", table, max(3, steps))
    e16 = restricted_err()
    ms32 = timed("fp32", table, 2)
    e32 = restricted_err()
    # smallest BF16 step count whose restricted error matches the FP32 one
    t16, ms16_eq, e16_eq = T, ms16, e16
    while e16_eq > 1.05 * e32 + 1e-4 and t16 < T + 4:
        t16 += 1
        tab16 = pe.pe_coeffs(5, l, t16, 1.01)
        ms16_eq = timed("bf16", tab16, 3)
        e16_eq = restricted_err()
    peaks = measured_peaks()
    out["bf16"] = {"value": flops / (ms16 * 1e-3) / 1e12, "unit": "TFLOP/s", "ms_per_step": ms16,
                   "frac_of_bf16_peak": flops / (ms16 * 1e-3) / 1e12 / peaks["bf16_tflops"],
                   # the call runs for seconds under the power cap: the sustained figure applies too
                   "frac_of_bf16_sustained": flops / (ms16 * 1e-3) / 1e12 / peaks["bf16_tflops_sustained"],
                   "restricted_max_sigma_err": e16}
    out["fp32_plain"] = {"value": flops / (ms32 * 1e-3) / 1e12, "unit": "TFLOP/s", "ms_per_step": ms32,
                         "restricted_max_sigma_err": e32}
    out["speedup_vs_fp32_plain_equal_err"] = {"value": ms32 / ms16_eq, "T_bf16": t16, "T_fp32": T,
                                              "restricted_max_sigma_err_bf16": e16_eq,
                                              "restricted_max_sigma_err_fp32": e32}
    del xs, mats, facs
    torch.cuda.empty_cache()
    return out


NS5_ROW = (15.0 / 8.0, -10.0 / 8.0, 3.0 / 8.0)   # the fixed Newton-Schulz quintic (Sec. 2)


def newton_schulz_line(pe, torch, wl, dev_in, dtype, flush, stream, refs, args):
    """The fixed-coefficient Newton-Schulz quintic, T = the workload's T, run
    through the same kernels (same grouped call and graph): time per step and
    max|sigma - 1| on the accuracy sample."""
    table = np.array([NS5_ROW] * wl.T)
    xs = [d.clone() for d in dev_in]
    for _ in range(2):
        for d, s in zip(xs, dev_in):
            d.copy_(s)
        pe.pe_polar_batched(xs, table, dtype)
    n = max(3, min(20, args.steps // 5))
    tot = 0.0
    for _ in range(n):
        for d, s in zip(xs, dev_in):
            d.copy_(s)
        flush.fill_(3.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        pe.pe_polar_batched(xs, table, dtype)
        b.record(stream)
        b.synchronize()
        tot += a.elapsed_time(b)
    ms = tot / n
    errs = [_max_sigma_err(xs[i].cpu().numpy().astype(np.float64)) for i in sorted(refs)]
    pe_errs = [_max_sigma_err(refs[i][0]) for i in sorted(refs)]
    return {"value": algorithmic_flops(wl.shapes, wl.T) / (ms * 1e-3) / 1e12, "unit": "TFLOP/s", "ms_per_step": ms,
            "T": wl.T, "dtype": dtype, "max_sigma_err_sample": max(errs) if errs else None,
            "polar_express_fp64_max_sigma_err_sample": max(pe_errs) if pe_errs else None}


def cublas_listing_line(torch, wl, table, dev_in, flush, stream, refs, ours_ms, args):
    """The same method written with PyTorch library calls (cuBLAS GEMMs), the
    form of the paper's own online code (App. A): X, A and B stored in BF16,
    one batched GEMM call per product for each stack of same-shape matrices,
    the combinations b A + c A A and a X + B X folded into the GEMM calls
    (baddbmm's beta and alpha), the whole step sequence replayed from a CUDA
    graph. A comparison point for the kernels of this library, which it
    does not call; time per Muon step and relative error on the accuracy
    sample against the FP64 iteration."""
    groups = {}
    for i, sh in enumerate(wl.shapes):
        groups.setdefault(sh, []).append(i)
    stacks = [(sh, idx, torch.stack([dev_in[i] for i in idx])) for sh, idx in groups.items()]
    outs = [torch.empty_like(G) for _, _, G in stacks]
    coef = [tuple(float(v) for v in row) for row in table]

    def step_sequence():
        for (sh, _, G), out in zip(stacks, outs):
            nrm = torch.linalg.vector_norm(G, dim=(1, 2), keepdim=True)
            X = (G / (1.01 * nrm + 1e-7)).to(torch.bfloat16)
            if sh[0] > sh[1]:
                X = X.mT                               # short side first
            for a, b, c in coef:
                A = torch.bmm(X, X.mT)
                B = torch.baddbmm(A, A, A, beta=b, alpha=c)
                X = torch.baddbmm(X, B, X, beta=a, alpha=1.0)
            out.copy_(X.mT if sh[0] > sh[1] else X)

    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        for _ in range(3):
            step_sequence()
    stream.wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step_sequence()
    graph.replay()
    n = max(3, min(20, args.steps // 5))
    tot = 0.0
    for _ in range(n):
        flush.fill_(3.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        graph.replay()
        b.record(stream)
        b.synchronize()
        tot += a.elapsed_time(b)
    ms = tot / n
    errs = []
    for (sh, idx, _), out in zip(stacks, outs):
        for k, i in enumerate(idx):
            if i in refs:
                errs.append(_rel_fro(out[k].cpu().numpy().astype(np.float64), refs[i][0]))
    del graph, stacks, outs
    torch.cuda.empty_cache()
    return {"value": algorithmic_flops(wl.shapes, wl.T) / (ms * 1e-3) / 1e12, "unit": "TFLOP/s", "ms_per_step": ms,
            "T": wl.T, "kind": "torch bmm/baddbmm (cuBLAS) in BF16 per same-shape stack, CUDA graph",
            "rel_fro_vs_fp64_iteration_sample_max": max(errs) if errs else None,
            "speedup_of_this_library": ms / ours_ms}


def spectrum_bound_line(pe, wl, dev_in, iters=10):
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
        pe.pe_spectrum_bound(dev_in[i], v0, iters)
        t0 = time.perf_counter()
        z, f = pe.pe_spectrum_bound(dev_in[i], v0, iters)
        rows.append({"shape": list(sh), "ms": 1e3 * (time.perf_counter() - t0), "z_over_f": z / f if f else None})
    return {"iters": iters, "rows": rows}


def error_sweep(pe, torch, wl, dev_in, flush, stream, Ts=(2, 4, 6, 8, 10, 12), gamma=1e-3):
    """Error against the truth U V^T vs iteration count T and vs time, for the
    Polar Express tables (FP32 plain, BF16, BF16x3) and the Newton-Schulz
    quintic (BF16), on a workload with known factors. Errors per T: the
    largest over the workload's matrices of max|sigma_i - 1| restricted to the
    directions with s_i >= gamma s_max (singular values of U1^T X V1, FP64 on
    the GPU) and of ||X - U V^T||_F / sqrt(n)."""
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
            xs = [d.clone() for d in dev_in]
            pe.pe_polar_batched(xs, table, dt)            # plan, tuning
            ms = 0.0
            for _ in range(3):
                for d, s in zip(xs, dev_in):
                    d.copy_(s)
                flush.fill_(4.0)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                pe.pe_polar_batched(xs, table, dt)
                b.record(stream)
                b.synchronize()
                ms += a.elapsed_time(b) / 3
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


def _rel_fro(X, Y):
    return float(np.linalg.norm(X - Y) / np.linalg.norm(Y))


def _err_fro(X, P):
    return float(np.linalg.norm(X - P) / np.sqrt(min(X.shape)))


def _max_sigma_err(X):
    return float(np.max(np.abs(np.linalg.svd(X, compute_uv=False) - 1.0)))


def accuracy_and_fp32(pe, torch, wl, table, dev_in, dtype, flush, stream, args, refs):
    """FP32 plain path on the same workload (time per step) and errors of the
    accuracy sample against the FP64 iterates ``refs`` that the cpu_baseline
    leg computed."""
    out = {}
    xs = [d.clone() for d in dev_in]
    # FP32 plain timing
    for _ in range(2):
        for d, s in zip(xs, dev_in):
            d.copy_(s)
        pe.pe_polar_batched(xs, table, "fp32")
    n = max(3, min(20, args.steps // 5))
    tot = 0.0
    for _ in range(n):
        for d, s in zip(xs, dev_in):
            d.copy_(s)
        flush.fill_(2.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        pe.pe_polar_batched(xs, table, "fp32")
        b.record(stream)
        b.synchronize()
        tot += a.elapsed_time(b)
    ms32 = tot / n
    flops = algorithmic_flops(wl.shapes, wl.T)
    idx = sorted(refs)
    res = {}
    for path in (dtype, "fp32"):
        xs2 = [dev_in[i].clone() for i in idx]
        pe.pe_polar_batched(xs2, table, path)
        torch.cuda.synchronize()
        errs = []
        for j, i in enumerate(idx):
            got = xs2[j].cpu().numpy().astype(np.float64)
            ref, P = refs[i]
            errs.append({"shape": list(wl.shapes[i]), "rel_fro_vs_fp64_iteration": _rel_fro(got, ref),
                         "err_fro_per_sqrt_n": _err_fro(got, P), "max_sigma_err": _max_sigma_err(got),
                         "fp64_max_sigma_err": _max_sigma_err(ref)})
        res[path] = errs
    worst16 = max(e["max_sigma_err"] for e in res[dtype])
    worst32 = max(e["max_sigma_err"] for e in res["fp32"])
    out["fp32_plain"] = {"value": flops / (ms32 * 1e-3) / 1e12, "unit": "TFLOP/s", "ms_per_step": ms32,
                         "max_sigma_err_sample": worst32, "T": wl.T}
    out["accuracy"] = res
    out["_worst"] = (worst16, worst32, ms32)
    return out


if __name__ == "__main__":
    sys.exit(main())
