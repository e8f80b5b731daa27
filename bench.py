#!/usr/bin/env python3
"""Throughput benchmark: LLG cell-updates per second on one or more GB300s.

Workload (default "batched_heun"): 256 replicas of a Permalloy disk R = 50 nm,
L = 10 nm, a = 2 nm (50 x 50 cells, 1976 in the disk, FFT grid 128 x 128),
T = 300 K, alpha = 0.01, dt = 10 fs, Philox seeds 0..255, FP32 fields -- the
batched Langevin-Heun configuration.  One bench step is CHUNK = 50 stochastic
Heun time steps of every replica (two full field evaluations each) followed
by the per-replica statistics sample (vortex core estimator, FP64 moments and
uint64 histograms of r and V, all on the device).  A cell-update is one time step of one disk cell of one replica.

Other workloads: "large_disk" (8 replicas of R = 500 nm, L = 20 nm, FFT grid
1024 x 1024, Heun at 300 K: the HBM-bound configuration) and "plain" (the
batched workload's disk as a single replica).

The JSON line also carries: the plain single-replica number (batched vs
plain), the roofline of the dominant kernel, the end-to-end number through the
C ABI with host buffers, SM clocks sampled during the timed region, and the
FP64 CPU oracle timed on the host cores.  A default run (batched_heun) also
times the large-disk workload the same way and nests its record, with its own
HBM roofline, e2e, clocks and oracle sample, under "large_disk".  With --impl
reference the oracle alone is timed as the reference arm.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

CHUNK = 50          # Heun steps per bench step
DT = 1e-14          # 10 fs
T_K = 300.0
ALPHA = 0.01

# The headline metric: cell-updates per second of the batched form, reported
# next to the plain single-replica form on the same GPU at the same accuracy,
# and the fraction of the roofline of the dominant kernel.
METRIC = ("LLG cell-updates/sec (batched vs plain, same GPU, rel. field err <=1e-5) "
          "and % HBM roofline")

WORKLOADS = {
    "batched_heun": dict(R=50e-9, L=10e-9, B=256),
    "plain": dict(R=50e-9, L=10e-9, B=1),
    "large_disk": dict(R=500e-9, L=20e-9, B=8),
}


def fft_flops_per_eval(P, C):
    """Algorithmic flops of one field evaluation: 2.5 P^2 log2(P^2) per real 2D
    transform (three forward, three inverse), 14 per spectral point of the
    tensor multiply, 60 per cell for the epilogue."""
    import math
    return 6 * 2.5 * P * P * math.log2(P * P) + 14 * P * (P // 2 + 1) + 60 * C


def fp32_alu_peak_tflops(sms, sm_mhz=2070.0, lanes=128):
    """FP32 FMA peak: SMs x FP32 lanes x 2 flops x clock (the device's SM
    count, 128 FP32 lanes per SM, the maximum SM clock)."""
    return sms * lanes * 2 * sm_mhz * 1e6 / 1e12


def device_sms(device=0):
    import torch
    return torch.cuda.get_device_properties(device).multi_processor_count


# The sources that make up each workload's dominant kernel: its translation
# unit and the device headers it includes (nd_kernels.h holds only host
# declarations and is left out).
KERNEL_SOURCES = {
    "batched_heun": ["nd_fused_f32.cu", "nd_cluster.cuh", "nd_field_impl.cuh", "nd_phases.cuh", "nd_fft.cuh",
                     "nd_common.cuh"],
    "large_disk": ["nd_glob_f32.cu", "nd_field_impl.cuh", "nd_phases.cuh", "nd_fft.cuh", "nd_common.cuh"],
}
KERNEL_SOURCES["plain"] = KERNEL_SOURCES["batched_heun"]


def kernel_sources_sha256(workload="batched_heun"):
    """Hash of the CUDA sources of the workload's dominant kernel (changes
    whenever that kernel changes)."""
    import hashlib
    d = os.path.join(ROOT, "paper_1207_2192_gb300", "csrc")
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[workload]:
        h.update(f.encode())
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()


def profiled_traffic(workload):
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary, or None if that kernel's sources changed since it was captured."""
    p = os.path.join(ROOT, "profiles", "kernel_traffic.json")
    if not os.path.exists(p):
        return None
    e = json.load(open(p)).get("entries", {}).get(workload)
    if e is None or e.get("sources_sha256") != kernel_sources_sha256(workload):
        return None
    return e.get("dram_bytes_per_launch")


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p))
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "fallback": True}


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        # the raw samples go to $ND_CLOCKS_CSV if set, else to a temporary file
        self.path = os.environ.get("ND_CLOCKS_CSV") or os.path.join(
            os.environ.get("TMPDIR", "/tmp"), f"nd_clocks_gpu{gpu_index}_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(self.gpu)], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), smax=float(parts[2]), power=float(parts[3]) if parts[3] not in ("[N/A]", "") else None,
                                 hw=parts[5], hwt=parts[6], swt=parts[7], swp=parts[8]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        reasons = set()
        for r in rows:
            for k, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"), ("swt", "sw_thermal_slowdown"),
                            ("swp", "sw_power_cap")):
                if r[k].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in rows), "sm_max_mhz": max(r["smax"] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows)}


# ------------------------------------------------------------- GPU workload

class Workload:
    def __init__(self, name, device):
        import torch
        import paper_1207_2192_gb300 as nd
        self.nd, self.torch = nd, torch
        w = WORKLOADS[name]
        self.name = name
        self.disk = nd.Disk(w["R"], w["L"], alpha=ALPHA)
        self.B = w["B"]
        self.h = nd.Nanodisk([self.disk], [self.B], nd.ND_FP32)
        # the stepping plan of the size class: the public autotuner times the
        # one-CTA kernel's thread counts, the cluster plan and the global path
        nd.nd_autotune(self.h.h, nd.ND_METHOD_HEUN, DT, CHUNK)
        L0 = self.h.layout[0]
        self.D, self.P, self.C = L0["D"], L0["P"], L0["cells"]
        self.m = self.h.empty_device()
        self.h.init_vortex(self.m, np.zeros((self.B, 2)))
        self.T = np.full(self.B, T_K)
        self.seeds = np.arange(self.B, dtype=np.uint64)
        self.step = 0
        self.stream = torch.cuda.current_stream()
        # r histogram: 0.05 nm bins over 0..15 nm; V histogram: 1 m/s bins over 0..400 m/s
        self.nd.nd_stats_reset(self.h.h, 15e-9, 300, 400.0, 400)

        # the production step as one CUDA graph: CHUNK Heun steps of every
        # replica and one statistics sample; replays advance the noise counter
        self.graph = None

    def make_graph(self):
        self.graph = self.nd.nd_graph_create(self.h.h, self.m, self.nd.ND_METHOD_HEUN, CHUNK, DT, self.T, self.seeds,
                                             step0=self.step, stats_sample=True)
        self.graph_kernels = self.nd.nd_graph_nodes(self.graph)

    def cell_updates_per_step(self):
        return self.B * self.C * CHUNK

    def run_step(self, m=None):
        """One bench step: CHUNK Heun steps, then the core statistics sample
        (core estimator + FP64 moments and uint64 histograms, on the device,
        no host synchronisation).  Returns the number of kernel launches."""
        target = self.m if m is None else m
        self.h.heun(target, CHUNK, DT, self.T, self.seeds, step0=self.step, stream=self.stream)
        self.step += CHUNK
        self.nd.nd_stats_sample(self.h.h, target, CHUNK * DT, self.stream)
        return 3


def max_over_ranks(x, dist, device):
    """Largest value of x over all ranks (the slowest rank sets the time)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, seconds_max):
    """Weak scaling: every rank runs its own replicas; the job's rate is all
    ranks' units over the slowest rank's time."""
    return units_per_rank * world / seconds_max


def l2_flush(torch, buf):
    buf.add_(1.0)   # writes 256 MB > 129 MB L2


def global_path_bytes_per_step(wl):
    """Algorithmic HBM bytes of one Heun step of every replica on the global
    path: per field evaluation the stage state, y_n and the accumulator
    (60 B per cell), four passes over the [3][D][P/2+1] half spectrum, and the
    spectral kernel once per evaluation."""
    kh = wl.P // 2 + 1
    per_eval = wl.B * (60 * wl.C + 4 * 3 * wl.D * kh * 8) + kh * kh * 16
    return 2 * per_eval * CHUNK


def kernel_name(wl):
    """Name of the kernel that steps the workload's size class under the plan
    the handle uses (fused on-chip kernel with its thread count, or the global
    path)."""
    info = wl.nd.nd_plan_info(wl.h.h, 0)
    if info and info["plan_heun"] in (200, 201):
        nc = info["threads_heun"] // (512 if wl.P >= 256 else 256)
        return f"k_cluster<{wl.P},float,HEUN,{nc}> (one replica per {nc}-CTA cluster)"
    if info and info["threads_heun"] > 0:
        return f"k_fused<{wl.P},float,HEUN,{info['threads_heun']}>"
    return "global-path Heun step (k_g_rows, k_g_cols_tile x/y and z, k_g_epi)"


def measure(name, steps, warmup, world, local_rank, dist, flush):
    """Time one workload: graph replays in the device-timed region (L2 flushed
    before each), nd_step_heun alone for the roofline, and nd_step_heun on
    pinned host buffers end to end.  Returns (record or None off rank 0, wl)."""
    import torch
    wl = Workload(name, local_rank)
    for _ in range(warmup):
        wl.run_step()
    wl.make_graph()
    for _ in range(warmup):
        wl.nd.nd_graph_launch(wl.graph, wl.stream)
        wl.step += CHUNK
    torch.cuda.synchronize()

    # ---- device-timed region: graph replays (CHUNK Heun steps + statistics
    # sample), inputs resident in HBM, L2 flushed between steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    launches = 0
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clk:
        for i in range(steps):
            l2_flush(torch, flush)
            ev[i][0].record()
            wl.nd.nd_graph_launch(wl.graph, wl.stream)
            ev[i][1].record()
            wl.step += CHUNK
            launches += wl.graph_kernels
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(sum(step_ms), dist, "cuda")
    # the stepping kernels alone (events around nd_step_heun on the same
    # stream, L2 flushed), for the roofline of the dominant kernel
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(5)]
    for a, b in kev:
        l2_flush(torch, flush)
        a.record()
        wl.h.heun(wl.m, CHUNK, DT, wl.T, wl.seeds, step0=wl.step, stream=wl.stream)
        b.record()
        wl.step += CHUNK
    torch.cuda.synchronize()
    kern_ms = [a.elapsed_time(b) for a, b in kev]
    cu_rank = wl.cell_updates_per_step() * steps
    value = whole_job_rate(cu_rank, world, total_ms / 1e3)

    # ---- end to end through the C ABI with host buffers (pinned), copies timed
    host = torch.empty(wl.h.state_elems, dtype=torch.float32, pin_memory=True)
    host.copy_(wl.m.cpu())
    nbytes = host.numel() * host.element_size()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for i in range(steps):
        wl.nd.nd_step_heun(wl.h.h, host.data_ptr(), CHUNK, DT, wl.T, wl.seeds, wl.step, None)
        wl.step += CHUNK
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    e2e = whole_job_rate(cu_rank, world, e2e_s)
    if os.environ.get("RANK", "0") != "0":
        return None, wl

    peaks = measured_peaks()
    kern_avg_s = statistics.mean(kern_ms) / 1e3
    timing = "CUDA events around nd_step_heun on the bench stream, 5 launches, L2 flushed"
    if wl.P <= 128:
        flop_cu = 2 * fft_flops_per_eval(wl.P, wl.C) / wl.C          # per cell-update (Heun = 2 evaluations)
        achieved = flop_cu * wl.cell_updates_per_step() / kern_avg_s / 1e12
        sms = device_sms(local_rank)
        peak = fp32_alu_peak_tflops(sms)
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": profiled_traffic(name), "kernel": kernel_name(wl), "flops_per_cell_update": flop_cu,
                "units_per_launch": wl.cell_updates_per_step(),
                "peak_note": f"FP32 FMA: {sms} SMs x 128 lanes x 2 x 2070 MHz, derived from unit counts "
                             "(MEASURED_PEAKS.json has no FP32 entry)",
                "timing": timing}
    else:
        nbytes_step = global_path_bytes_per_step(wl)
        achieved = nbytes_step / kern_avg_s / 1e9
        peak = peaks.get("hbm_gbs", 6800.0)
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": profiled_traffic(name), "kernel": kernel_name(wl),
                "bytes_per_cell_update": nbytes_step / wl.cell_updates_per_step(),
                "units_per_launch": wl.cell_updates_per_step(),
                "peak_note": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)" +
                             (" -- fallback value" if peaks.get("fallback") else ""),
                "timing": timing}
    rec = {
        "value": value, "unit": "cell-updates/s", "steps": steps, "ms_per_step": total_ms / steps,
        "config": {"workload": name, "replicas_per_gpu": wl.B, "R_nm": wl.disk.R * 1e9,
                   "L_nm": wl.disk.L * 1e9, "a_nm": wl.disk.a * 1e9, "D": wl.D, "cells": wl.C, "P": wl.P,
                   "T_K": T_K, "alpha": ALPHA, "dt_fs": DT * 1e15, "heun_steps_per_bench_step": CHUNK,
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "l2": "flushed between timed steps (256 MB write)",
                   "launch": "one CUDA graph per bench step (nd_graph_create)"},
        "roofline": roof,
        "kernel_ms_per_step": statistics.mean(kern_ms),
        "e2e": {"value": e2e, "unit": "cell-updates/s", "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes},
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    return rec, wl


def uneven_record(steps, warmup, world, local_rank, dist, flush):
    """The uneven batch: 64 disks with R ~ U(20, 100) nm, L/R ~ U(0.05, 0.2)
    and T ~ U(0, 400) K (ndsynth.uneven_disks, seed 0), the 8 at T = 0 on RK4
    and the rest on Heun, in two handles tuned together (nd_autotune_group);
    their 50-step graphs joined into one graph, one launch per bench step,
    timed the same way as the main workload.  Returns the nested record
    (rank 0)."""
    import torch
    import ndsynth
    import paper_1207_2192_gb300 as nd
    R, L, T = ndsynth.uneven_disks(64, seed=0)
    groups = {"rk4": list(range(8)), "heun": list(range(8, 64))}
    stream = torch.cuda.current_stream()
    hs, ms, gs, args_by = {}, {}, {}, {}
    cells, classes = 0, []
    built = {}
    for name, idx in groups.items():
        built[name] = nd.Nanodisk([nd.Disk(R[i], L[i], alpha=ALPHA) for i in idx], None, nd.ND_FP32)
    # the plans of both handles tuned together, as their joined graph runs them
    nd.nd_autotune_group([built["rk4"].h, built["heun"].h], [nd.ND_METHOD_RK4, nd.ND_METHOD_HEUN], DT, CHUNK)
    for name, idx in groups.items():
        h = built[name]
        method = nd.ND_METHOD_RK4 if name == "rk4" else nd.ND_METHOD_HEUN
        m = h.empty_device()
        h.init_vortex(m, np.stack([0.1 * R[idx], np.zeros(len(idx))], 1))
        Tk = T[idx] if name == "heun" else None
        sd = np.arange(len(idx), dtype=np.uint64) if name == "heun" else None
        gs[name] = nd.nd_graph_create(h.h, m, method, CHUNK, DT, Tk, sd, step0=0)
        hs[name], ms[name], args_by[name] = h, m, (method, Tk, sd)
        cells += sum(h.layout[r]["cells"] for r in range(h.B))
        c = 0
        while True:
            info = nd.nd_plan_info(h.h, c)
            if info is None:
                break
            classes.append({"method": name, "P": info["P"], "replicas": info["replicas"],
                            "plan": info["plan_rk4" if name == "rk4" else "plan_heun"]})
            c += 1
    g = nd.nd_graph_join([gs["rk4"], gs["heun"]])
    launches_per_step = nd.nd_graph_nodes(g)
    for _ in range(warmup):
        nd.nd_graph_launch(g, stream)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    if dist:
        dist.barrier()
    with ClockSampler(local_rank) as clk:
        for i in range(steps):
            l2_flush(torch, flush)
            ev[i][0].record()
            nd.nd_graph_launch(g, stream)
            ev[i][1].record()
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    total_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev), dist, "cuda")
    value = whole_job_rate(cells * CHUNK * steps, world, total_ms / 1e3)
    hosts = {}
    for name in groups:
        hosts[name] = torch.empty(hs[name].state_elems, dtype=torch.float32, pin_memory=True)
        hosts[name].copy_(ms[name].cpu())
    nbytes = sum(x.numel() * x.element_size() for x in hosts.values())
    e2e_steps = max(3, steps // 4)
    # end to end as the joined graph is used: every step both handles' states
    # go in from pinned host memory, one graph launch steps them, and they come
    # back to the host before the next step
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        for name in groups:
            ms[name].copy_(hosts[name], non_blocking=True)
        nd.nd_graph_launch(g, stream)
        for name in groups:
            hosts[name].copy_(ms[name], non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    # the same through the stepping calls on host buffers, one handle after the other
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        nd.nd_step_rk4(hs["rk4"].h, hosts["rk4"].data_ptr(), CHUNK, DT, None)
        _, Tk, sd = args_by["heun"]
        nd.nd_step_heun(hs["heun"].h, hosts["heun"].data_ptr(), CHUNK, DT, Tk, sd, 1000 * CHUNK + i * CHUNK, None)
    calls_s = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    nd.nd_graph_destroy(g)
    for x in gs.values():
        nd.nd_graph_destroy(x)
    if os.environ.get("RANK", "0") != "0":
        return None
    return {
        "value": value, "unit": "cell-updates/s", "steps": steps, "ms_per_step": total_ms / steps,
        "config": {"workload": "uneven batch, 64 disks (R 20-100 nm, L/R 0.05-0.2, T 0-400 K; RK4 at T = 0)",
                   "disks_per_gpu": 64, "cells": cells, "size_classes": classes,
                   "heun_steps_per_bench_step": CHUNK, "dt_fs": DT * 1e15, "alpha": ALPHA,
                   "schedule": "two handles' graphs joined into one graph launch (nd_graph_join); classes side by side; "
                               "plans from nd_autotune_group",
                   "l2": "flushed between timed steps (256 MB write)"},
        "e2e": {"value": whole_job_rate(cells * CHUNK * e2e_steps, world, e2e_s), "unit": "cell-updates/s",
                "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
                "path": "pinned host -> device copies, nd_graph_launch of the joined graph, device -> host copies, "
                        "synchronised every step",
                "step_calls_value": whole_job_rate(cells * CHUNK * e2e_steps, world, calls_s),
                "step_calls_path": "nd_step_rk4 then nd_step_heun on the pinned host buffers (the C ABI stages "
                                   "each handle's copies itself; the handles run one after the other)"},
        "gpu_launches": launches_per_step * steps, "clocks": clk.summary(),
    }


def run_ours(args, rank, world, local_rank):
    import torch
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    flush = torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    rec, wl = measure(args.workload, args.steps, args.warmup, world, local_rank, dist, flush)
    large = uneven = None
    if args.workload == "batched_heun" and args.large_steps > 0:
        # the HBM-bound configuration, timed the same way, nested in the line
        large, _ = measure("large_disk", args.large_steps, args.warmup, world, local_rank, dist, flush)
    if args.workload == "batched_heun" and args.uneven_steps > 0:
        uneven = uneven_record(args.uneven_steps, args.warmup, world, local_rank, dist, flush)
    result = None
    if rank == 0:
        peaks = measured_peaks()
        result = {
            "metric": METRIC, "value": rec["value"], "unit": "cell-updates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": rec["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (analytic centred vortex, Philox thermal noise)",
            "config": rec["config"], "roofline": rec["roofline"], "kernel_ms_per_step": rec["kernel_ms_per_step"],
            "e2e": rec["e2e"], "gpu_launches": rec["gpu_launches"], "clocks": rec["clocks"],
        }
        if "hbm_gbs" in peaks:
            result["hbm_peak_gbs"] = peaks["hbm_gbs"]
        if large is not None:
            result["large_disk"] = large
        if uneven is not None:
            result["uneven_batch"] = uneven
    if dist:
        dist.destroy_process_group()
    return result, wl


def plain_number(args):
    """Batched-vs-plain: the same disk as one replica, same kernels and accuracy."""
    import torch
    wl = Workload("plain", 0)
    for _ in range(3):
        wl.run_step()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n = max(3, args.steps)
    a.record()
    for _ in range(n):
        wl.run_step()
    b.record()
    torch.cuda.synchronize()
    return wl.cell_updates_per_step() * n / (a.elapsed_time(b) / 1e3), kernel_name(wl)


# ---------------------------------------------------------------- oracle

def oracle_rate(workload, budget_s=12.0):
    """FP64 direct-sum oracle, as it stands, on the host cores: Heun steps of
    one replica of the workload's disk.  Returns (cell-updates/s, sample)."""
    import oracle
    w = WORKLOADS[workload]
    model = oracle.Model(w["R"], w["L"], alpha=ALPHA)
    m = model.init_vortex(0.0, 0.0)
    if model.C > 20000:
        # a full step is out of reach (C^2 pair terms per evaluation): time the
        # direct-sum field at sampled cells, in batches of 64 until the budget
        # is spent, and extrapolate (2 evaluations per Heun step)
        inside = np.flatnonzero(model.mask.ravel())
        done, k, t0 = 0, 0, time.perf_counter()
        while True:
            cells = inside[(np.arange(64) * 3067 + 64 * k) % len(inside)]
            model.field_at(m, cells)
            done += len(cells)
            k += 1
            el = time.perf_counter() - t0
            if el >= budget_s:
                break
        rate = done / (2.0 * el)
        return rate, (f"extrapolated: direct-sum field at {done} cells (of {model.C}) of one "
                      f"R={w['R']*1e9:.0f} nm replica in {el:.1f} s, 2 evaluations per Heun step"), oracle.num_threads()
    Ts = oracle.scaled_temperature(T_K, model.A, model.L)
    dtau = model.dtau(DT)
    t0 = time.perf_counter()
    model.heun(m, 1, dtau, Ts, 0, 0)
    one = time.perf_counter() - t0
    n = max(1, min(2000, int(budget_s / max(one, 1e-6))))
    t0 = time.perf_counter()
    model.heun(m, n, dtau, Ts, 0, 1)
    el = time.perf_counter() - t0
    rate = model.C * n / el
    return rate, f"{n} Heun steps of one R={w['R']*1e9:.0f} nm replica ({model.C} cells), {el:.1f} s", oracle.num_threads()


def run_reference(args):
    """The reference arm: the oracle, as it stands, on the host cores.  Each
    step is one bounded sample of the workload (its own Heun steps, or for the
    large disk sampled direct-sum cells); the budget per step keeps the whole
    run near a minute whatever K and W are."""
    rates, times = [], []
    sample = ""
    cores = 1
    budget = min(8.0, max(0.25, 60.0 / max(1, args.steps + args.warmup)))
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        r, sample, cores = oracle_rate(args.workload, budget_s=budget)
        if i >= args.warmup:
            rates.append(r)
            times.append(time.perf_counter() - t0)
    value = statistics.mean(rates)
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "cell-updates/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * statistics.mean(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload},
        "cpu_baseline": {"value": value, "unit": "cell-updates/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)   # about 1 s of timed replays: several clock samples
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batched_heun", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--large-steps", type=int, default=150,
                    help="bench steps of the nested large-disk record (0: skip it)")
    ap.add_argument("--uneven-steps", type=int, default=100,
                    help="bench steps of the nested uneven-batch record (0: skip it)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return
    result, wl = run_ours(args, rank, world, local_rank)
    if rank == 0:
        if not args.no_plain and args.workload == "batched_heun":
            plain, plain_kernel = plain_number(args)
            result["plain"] = {"value": plain, "unit": "cell-updates/s", "replicas": 1, "kernel": plain_kernel,
                               "batched_over_plain": result["value"] / world / plain}
        if not args.no_cpu_baseline:
            rate, sample, cores = oracle_rate(args.workload)
            result["cpu_baseline"] = {"value": rate, "unit": "cell-updates/s", "cores": cores, "kind": "oracle",
                                      "sample": sample}
            if "large_disk" in result:
                rate, sample, cores = oracle_rate("large_disk", budget_s=8.0)
                result["large_disk"]["cpu_baseline"] = {"value": rate, "unit": "cell-updates/s", "cores": cores,
                                                        "kind": "oracle", "sample": sample}
        print(json.dumps(result), flush=True)


if __name__ == "__main__":
    main()
