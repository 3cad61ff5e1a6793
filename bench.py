#!/usr/bin/env python
"""Block Toeplitz matvec benchmark on GB300: split FFT (Algorithm 1) vs the
plain full circulant embedding.

Default workload: d = 3, 256^3 grid, c = 3 dyadic Green blocks
(kh = 2 pi / 20, fully symmetric, mirror-compressed symbol), complex64, one
right-hand side: the largest single-GPU configuration, on which the split
form is compared with the plain 512^3 full embedding (own kernels and
cuFFT).  One step = one btmv_apply (every pass of the path) on
device-resident inputs.  Prints ONE JSON line on rank 0; with the default
workload the line also carries compact figures of the other workloads
(128^3 Green, 256^3 skew, 64^2 complex128, batched64, serving200) under
"secondary" (skip them with --no-secondary).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 (torchrun): every rank runs its own independent instance (weak
scaling, no data-path collective); a barrier brackets the timed region and
the slowest rank's time is used.
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
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

WORKLOAD = "d3_256_c3_green_c64"
PROFILE_EVERY = 10      # applies per event-profiled apply in the timed region
L2_BYTES = 129 * 1024 * 1024


def chunk_steps(steps: int) -> int:
    """Timed-region steps per chunk for the per-step percentiles: at least
    ten chunks whenever there are at least ten steps."""
    return max(1, steps // 10)


def metric_name(cfg) -> str:
    """The headline metric string for the default workload; the same wording
    for the other single-problem workloads, with their own sizes."""
    n = cfg["n"]
    grid = f"{n[0]}^{len(n)}" if len(set(n)) == 1 else "x".join(str(v) for v in n)
    kind = {"green": "Green", "skew": "skew", "random": "random"}.get(cfg["kind"], cfg["kind"])
    prec = "complex64" if cfg["precision"] == "c64" else "complex128"
    return f"block Toeplitz matvecs/s (split FFT, d={len(n)} {grid} c={cfg['c']} {kind}, {prec})"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(W.WORKLOADS) + ["batched64", "serving200", "multirhs", "cpu_fig3",
                                                                  "fused_levels"])
    ap.add_argument("--no-compare", action="store_true", help="skip the full-embedding and cuFFT rows")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle timing")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the compact figures of the other workloads")
    return ap.parse_args()


# ------------------------------------------------------------------ helpers
def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# source files that define each kernel kind bench.py reports on; a recorded
# ncu figure is used only while these files are unchanged
KERNEL_SOURCES = {
    "leaf": ["fast_leaf.cu", "fast_leaf3.cu", "fast.cuh", "kernels.cuh", "fft.cuh"],
    "fwd_split": ["fast_pass.cu", "fast_pass_tma.cu", "fast.cuh", "kernels.cuh", "fft.cuh"],
    "merge": ["fast_pass.cu", "fast_pass_tma.cu", "fast.cuh", "kernels.cuh", "fft.cuh"],
    "fused2": ["fused2.cu", "fast.cuh", "kernels.cuh", "fft.cuh"],
    "small2d": ["small2d.cu", "fast.cuh", "kernels.cuh", "fft.cuh"],
    "fused2c": ["fused2c.cu", "fast.cuh", "kernels.cuh", "fft.cuh"],
}


def source_sha(kernel_kind=None):
    """sha256 (16 hex digits) of the kernel kind's source files, or of every
    file under csrc/ when no kind is given."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2406_17981_gb300", "csrc")
    files = KERNEL_SOURCES.get(kernel_kind) or sorted(os.listdir(d))
    for f in sorted(files):
        with open(os.path.join(d, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_kind: str, workload: str):
    """DRAM bytes per launch recorded by ncu for this kernel (profiles/),
    or None when absent or taken on other sources."""
    path = os.path.join(ROOT, "profiles", f"ncu_{kernel_kind}_{workload}.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m1 = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    m2 = re.search(r"sources_sha256:\s*([0-9a-f]+)", txt)
    if not m1 or not m2 or m2.group(1) != source_sha(kernel_kind):
        return None
    return float(m1.group(1))


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev: int):
        self.dev = dev
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(self.dev)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = []
        for line in out.strip().splitlines():
            f = [v.strip() for v in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append(dict(sm=float(f[1]), smax=float(f[2]), power=float(f[3]),
                                 hw=f[5], hwt=f[6], swt=f[7], swp=f[8]))
            except ValueError:
                continue
        if not rows:
            return None
        load = [r for r in rows if r["power"] > 300] or rows
        reasons = set()
        for r in load:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                              ("swt", "sw_thermal_slowdown"), ("swp", "sw_power_cap")):
                if r[key].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in load),
                "sm_max_mhz": max(r["smax"] for r in rows),
                "samples": len(load), "reasons": sorted(reasons)}


def dist_setup(args):
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v: float, ws: int) -> float:
    """The slowest rank's time (all ranks get it)."""
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(ws: int, units_per_rank: float, ms_max: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time (weak scaling: every rank runs its own instance)."""
    return ws * units_per_rank / (ms_max / 1000.0)


def make_generator(cfg):
    n = cfg["n"]
    if cfg["kind"] == "green":
        t, par = W.green_dyadic_orthant(n, kh=cfg["kh"])
        return t, par, 1 | 2
    if cfg["kind"] == "skew":
        t, par = W.skew_orthant(n, seed=cfg["t_seed"])
        return t, par, 1 | 2
    return W.random_generator(n, cfg["c"], seed=cfg["t_seed"]), None, 0


# ------------------------------------------------------------------ reference arm
def run_reference(args, cfg):
    """The FP64 CPU oracle as it stands, on a bounded sample: each step
    evaluates the direct sum (the definition) at a fixed set of output points,
    all components; the rate is scaled to matvecs/s by points / grid size."""
    from oracle import toeplitz as OT
    n, c = cfg["n"], cfg["c"]
    s = int(np.prod(n))
    t, par, _ = make_generator(cfg)
    tf = W.orthant_to_full(t, par) if par is not None else t
    x = W.random_vector(n, c, seed=cfg["x_seed"])
    rng = np.random.default_rng(17)
    t0 = time.perf_counter()
    OT.direct_points(tf, x, [tuple(int(v) for v in rng.integers(0, n))])
    per_pt = time.perf_counter() - t0
    budget = 150.0 / max(1, args.steps + args.warmup)
    npts = max(1, int(budget / max(per_pt, 1e-6)))
    pts = [tuple(int(v) for v in rng.integers(0, n)) for _ in range(npts)]
    for _ in range(args.warmup):
        OT.direct_points(tf, x, pts)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        OT.direct_points(tf, x, pts)
    el = time.perf_counter() - t0
    value = args.steps * npts / s / el
    cores = len(os.sched_getaffinity(0))
    unit = "matvecs/s"
    line = {"impl": "reference", "metric": metric_name(cfg), "value": value, "unit": unit, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, "d": len(n), "n": list(n), "c": c,
                                            "nrhs": 1, "sample_points_per_step": npts},
            "cpu_baseline": {"value": value, "unit": unit, "cores": cores, "kind": "oracle",
                             "sample": f"direct sum (definition, FP64 NumPy) at {npts} output points x {c} "
                                       f"components per step, scaled by points / {s}"},
            "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ------------------------------------------------------------------ our arm
def main():
    args = parse()
    if args.workload in ("batched64", "serving200", "multirhs", "cpu_fig3", "fused_levels"):
        fn = {"batched64": run_batched, "serving200": run_serving, "multirhs": run_multirhs,
              "cpu_fig3": run_cpu_fig3, "fused_levels": run_fused_levels}[args.workload]
        line = fn(args)
        if line is not None:
            print(json.dumps(line))
        return
    cfg = W.WORKLOADS[args.workload]
    if args.impl == "reference":
        if int(os.environ.get("RANK", "0")) != 0:
            return
        run_reference(args, cfg)
        return

    ws, rank, local = dist_setup(args)
    line = measure_single(args, cfg, ws, rank, local)
    if rank == 0 and args.workload == WORKLOAD and not args.no_secondary:
        line["secondary"] = secondaries(args)
    barrier(ws)
    if rank == 0:
        print(json.dumps(line))


def measure_single(args, cfg, ws, rank, local):
    """The timed split applies of one single-problem workload, with its
    roofline, end-to-end, CPU-oracle and full-embedding figures; returns the
    JSON line (rank 0) or None."""
    import torch

    from paper_2406_17981_gb300 import analysis as A
    from paper_2406_17981_gb300 import btmv as bt

    n, c = cfg["n"], cfg["c"]
    prec = bt.BTMV_C64 if cfg["precision"] == "c64" else bt.BTMV_C128
    cdt = torch.complex64 if prec == bt.BTMV_C64 else torch.complex128
    esz = 8 if prec == bt.BTMV_C64 else 16
    t, par, sflags = make_generator(cfg)
    x_host = W.random_vector(n, c, seed=cfg["x_seed"])
    xc = x_host.astype(np.complex64 if prec == bt.BTMV_C64 else np.complex128)

    # kernel durations come from CUDA events recorded live in the timed
    # region around the launches of one apply in every PROFILE_EVERY (events
    # separate launches, so recording every apply would slow the step)
    V = int(np.prod(n)) * c * esz
    # rotate over a pool of inputs/outputs so that no step finds its x in L2
    npool = max(2, math.ceil(2 * L2_BYTES / (2 * V)) + 1)
    xs = [torch.from_numpy(xc).to("cuda") for _ in range(npool)]
    ys = [torch.empty_like(xs[0]) for _ in range(npool)]
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    os.environ["BTMV_PROFILE_EVERY"] = str(PROFILE_EVERY)
    plan = bt.Plan(n, c, prec, bt.BTMV_ALGO_SPLIT, max_rhs=1, flags=bt.BTMV_FLAG_PROFILE)
    del os.environ["BTMV_PROFILE_EVERY"]
    plan.set_kernel(t, sflags, par)
    info = plan.info
    assert V == info["vector_bytes"]
    for i in range(args.warmup):
        plan.apply(xs[i % npool], ys[i % npool], 1)
    torch.cuda.synchronize()
    # device memory the plan holds (symbol, tables, workspace), measured
    plan_resident = free0 - torch.cuda.mem_get_info()[0]
    CHUNK = chunk_steps(args.steps)
    bt.btmv_profile_read(plan.handle)
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    barrier(ws)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    marks = [(0, e0)]                        # an event every CHUNK steps: per-step time spread
    e0.record()
    for i in range(args.steps):
        if i and i % CHUNK == 0:
            ev = torch.cuda.Event(enable_timing=True)
            ev.record()
            marks.append((i, ev))
        plan.apply(xs[i % npool], ys[i % npool], 1)
    e1.record()
    marks.append((args.steps, e1))
    torch.cuda.synchronize()
    barrier(ws)
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    chunk_ms = [a[1].elapsed_time(b[1]) / (b[0] - a[0]) for a, b in zip(marks, marks[1:]) if b[0] > a[0]]
    spread = [float(v) for v in np.percentile(chunk_ms, [10, 50, 90])] if len(chunk_ms) >= 3 else None
    ms_max = max_over_ranks(ms, ws)
    prof = bt.btmv_profile_read(plan.handle)
    sampled = (args.steps + PROFILE_EVERY - 1) // PROFILE_EVERY   # applies 0, k, 2k, .. after the read
    value = job_rate(ws, args.steps, ms_max)
    launches = info["launches_per_apply"] * args.steps

    # dominant kernel and its roofline (algorithmic bytes per launch / event time)
    sym_b = info["symbol_bytes"]
    pb = A.apply_kind_bytes(n, c, 1, esz, sym_b, one_kernel=len(n) == 2 and info["launches_per_apply"] == 1)
    kind_bytes = {k: v for k, v in pb.items() if k not in ("total", "V")}
    dom = max((k for k in kind_bytes if prof[k][1] > 0), key=lambda k: prof[k][0])
    per_apply_launches = prof[dom][1] / sampled
    bytes_per_launch = kind_bytes[dom] / per_apply_launches
    avg_launch_s = prof[dom][0] / prof[dom][1] / 1000.0
    peaks, peak_src = measured_peaks()
    peak = float(peaks["hbm_gbs"])
    achieved = bytes_per_launch / avg_launch_s / 1e9
    kernels = {k: {"launches_per_step": prof[k][1] / sampled, "avg_us": 1000 * prof[k][0] / prof[k][1],
                   "share": prof[k][0] / max(1e-12, sum(v[0] for v in prof.values())),
                   "algo_GBps": (kind_bytes[k] / (prof[k][1] / sampled)) / (prof[k][0] / prof[k][1] / 1000) / 1e9}
               for k in kind_bytes if prof[k][1] > 0}
    whole_GBps = pb["total"] * args.steps / (ms / 1000.0) / 1e9

    # end to end: host buffers through the public call (H2D + compute + D2H)
    e2e = None
    if True:
        # pinned host buffers; every step copies its x in and its y out
        xh = [torch.from_numpy(xc).pin_memory() for _ in range(3)]
        yh = [torch.empty_like(xh[0]).pin_memory() for _ in range(3)]
        ne = max(3, min(args.steps, 200))
        for i in range(2):
            bt.btmv_apply(plan.handle, xh[i], yh[i], 1)
        barrier(ws)
        t0 = time.perf_counter()
        for i in range(ne):
            bt.btmv_apply(plan.handle, xh[i % 3], yh[i % 3], 1)   # synchronous with host pointers
        el_sync = max_over_ranks(time.perf_counter() - t0, ws)
        for i in range(3):
            bt.btmv_apply_host_async(plan.handle, xh[i], yh[i], 1)
        bt.btmv_host_wait(plan.handle)
        barrier(ws)
        t0 = time.perf_counter()
        for i in range(ne):                     # pipelined: copies of one step overlap the apply of the next
            bt.btmv_apply_host_async(plan.handle, xh[i % 3], yh[i % 3], 1)
        bt.btmv_host_wait(plan.handle)
        el = max_over_ranks(time.perf_counter() - t0, ws)
        e2e = {"value": ws * ne / el, "unit": "matvecs/s", "h2d_bytes_per_step": V, "d2h_bytes_per_step": V,
               "steps": ne, "call": "btmv_apply_host_async, two staging slots, pinned host buffers",
               "synchronous_btmv_apply_value": ws * ne / el_sync}

    extra = {}
    cpu = None
    if rank == 0:
        y_gpu = ys[(args.steps - 1) % npool].cpu().numpy().astype(np.complex128)
        if not args.no_cpu:
            tf = W.orthant_to_full(t, par) if par is not None else t
            cores = len(os.sched_getaffinity(0))
            if int(np.prod(n)) <= 128 ** 3:
                from oracle import embed as OE
                t0 = time.perf_counter()
                ref = OE.embed_matvec(tf, xc.astype(np.complex128), workers=cores)
                el = time.perf_counter() - t0
                cpu = {"value": 1.0 / el, "unit": "matvecs/s", "cores": cores, "kind": "oracle",
                       "sample": f"one full matvec of the {args.workload} workload by the FP64 oracle "
                                 f"(circulant embedding, scipy.fft, {cores} workers), {el:.1f} s"}
                extra["rel_l2_vs_fp64_oracle"] = float(np.linalg.norm(y_gpu - ref) / np.linalg.norm(ref))
            else:
                # bounded sample: the direct sum (definition) at a few output points
                from oracle import toeplitz as OT
                rng = np.random.default_rng(23)
                pts = [tuple(int(v) for v in rng.integers(0, n)) for _ in range(8)]
                t0 = time.perf_counter()
                vals = OT.direct_points(tf, xc.astype(np.complex128), pts)
                el = time.perf_counter() - t0
                s_pts = int(np.prod(n))
                cpu = {"value": len(pts) / s_pts / el, "unit": "matvecs/s", "cores": 1, "kind": "oracle",
                       "sample": f"direct sum (FP64 NumPy) at {len(pts)} output points x {c} components, "
                                 f"{el:.1f} s, scaled by points / {s_pts}"}
                got = np.stack([y_gpu[(0, slice(None)) + p] for p in pts])
                extra["rel_l2_vs_fp64_oracle_sampled"] = float(np.linalg.norm(got - vals[:, 0]) /
                                                                np.linalg.norm(vals[:, 0]))
        # peak HBM of one apply: what the plan holds (measured by the drop in
        # free device memory) plus the caller's x and y
        extra["peak_hbm_split_bytes"] = plan_resident + 2 * V
        extra["peak_hbm_split_model_bytes"] = (info["symbol_bytes"] + info["workspace_bytes"] +
                                               info["table_bytes"] + 2 * V)
        if not args.no_compare:
            extra["two_stream_variant"] = time_two_streams(args, cfg, t, par, sflags, xc, prec, V)
            extra.update(compare_full(args, cfg, t, par, sflags, xc, prec, cdt, V, esz, info))
            full = extra["full_embedding_own"]
            extra["speedup_split_vs_full_own"] = full["ms_per_step"] / (ms_max / args.steps)
            algo_full = full["algo_bytes_per_step"]
            extra["byte_ratio_full_own_over_split"] = algo_full / pb["total"]
            extra["peak_hbm_ratio_full_over_split"] = full["peak_hbm_bytes"] / extra["peak_hbm_split_bytes"]
            extra["peak_hbm_like_for_like"] = like_for_like_memory(args, cfg, t, par, sflags, prec, V, n, c,
                                                                   extra["peak_hbm_split_bytes"],
                                                                   full["peak_hbm_bytes"])
            cf = extra.get("full_embedding_cufft", {})
            if "ms_per_step" in cf:
                extra["speedup_split_vs_cufft_full"] = cf["ms_per_step"] / (ms_max / args.steps)
    del plan
    barrier(ws)
    if rank != 0:
        return None
    line = {
        "metric": metric_name(cfg), "value": value, "unit": "matvecs/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
        "ms_per_step_p10_p50_p90": spread, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec == bt.BTMV_C64 else "f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "d": len(n), "n": list(n), "c": c, "nrhs": 1,
                   "precision": cfg["precision"], "algo": "split (Algorithm 1, depth-first)",
                   "symbol": "compressed parity + block symmetric" if sflags == 3 else "full",
                   "l2": f"inputs rotated over {npool} x/y pairs ({npool * 2 * V / 2**20:.0f} MiB) "
                         f"+ {info['workspace_bytes'] / 2**20:.0f} MiB workspace + "
                         f"{info['symbol_bytes'] / 2**20:.0f} MiB symbol, larger than the 129 MB L2",
                   "parallelism": f"{ws} independent instance(s), one per GPU"},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_source": f"{peak_src} hbm_gbs",
                     "traffic": ncu_traffic("small2d" if dom == "fused_levels" and len(n) == 2 else dom,
                                            args.workload),
                     "algorithmic_bytes_per_launch": bytes_per_launch},
        "whole_step_algo_GBps": whole_GBps,
        "kernels": kernels,
        "gpu_launches": launches,
        "e2e": e2e,
        "cpu_baseline": cpu,
        "clocks": clocks,
    }
    line.update(extra)
    return line


def compact_single(args, workload, steps):
    """One single-problem workload in brief: split matvecs/s over `steps`
    applies (inputs rotated past L2), the dominant kernel's roofline, the
    two-stream traversal's rate for d >= 3, and the error against the FP64
    oracle (the full circulant embedding up to 128^3, the direct sum at 8
    sampled points above, the dense direct sum for the 64^2 complex128
    configuration)."""
    import torch

    from paper_2406_17981_gb300 import analysis as A
    from paper_2406_17981_gb300 import btmv as bt
    cfg = W.WORKLOADS[workload]
    n, c = cfg["n"], cfg["c"]
    prec = bt.BTMV_C64 if cfg["precision"] == "c64" else bt.BTMV_C128
    esz = 8 if prec == bt.BTMV_C64 else 16
    t, par, sflags = make_generator(cfg)
    xc = W.random_vector(n, c, seed=cfg["x_seed"]).astype(np.complex64 if esz == 8 else np.complex128)
    V = int(np.prod(n)) * c * esz
    npool = max(2, math.ceil(2 * L2_BYTES / (2 * V)) + 1)
    xs = [torch.from_numpy(xc).cuda() for _ in range(npool)]
    ys = [torch.empty_like(xs[0]) for _ in range(npool)]
    os.environ["BTMV_PROFILE_EVERY"] = "5"
    plan = bt.Plan(n, c, prec, bt.BTMV_ALGO_SPLIT, max_rhs=1, flags=bt.BTMV_FLAG_PROFILE)
    del os.environ["BTMV_PROFILE_EVERY"]
    plan.set_kernel(t, sflags, par)
    info = plan.info
    for i in range(5):
        plan.apply(xs[i % npool], ys[i % npool], 1)
    torch.cuda.synchronize()
    bt.btmv_profile_read(plan.handle)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for i in range(steps):
        plan.apply(xs[i % npool], ys[i % npool], 1)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    prof = bt.btmv_profile_read(plan.handle)
    sampled = (steps + 4) // 5
    pb = A.apply_kind_bytes(n, c, 1, esz, info["symbol_bytes"],
                            one_kernel=len(n) == 2 and info["launches_per_apply"] == 1)
    kind_bytes = {k: v for k, v in pb.items() if k not in ("total", "V")}
    peak = float(measured_peaks()[0]["hbm_gbs"])
    kernels = {}
    for k, b in kind_bytes.items():
        if prof[k][1] > 0:
            per = b / (prof[k][1] / sampled)
            us = 1000 * prof[k][0] / prof[k][1]
            kernels[k] = {"avg_us": us, "algo_GBps": per / us / 1e3, "frac": per / us / 1e3 / peak,
                          "share": prof[k][0] / max(1e-12, sum(v[0] for v in prof.values()))}
    out = {"matvecs_per_s": 1000.0 / ms, "ms_per_step": ms, "steps": steps,
           "whole_step_algo_GBps": pb["total"] / ms / 1e6, "whole_step_frac": pb["total"] / ms / 1e6 / peak,
           "kernels": kernels, "launches_per_step": info["launches_per_apply"]}
    y = ys[(steps - 1) % npool].cpu().numpy().astype(np.complex128)
    plan.close()
    if len(n) >= 3:
        # the same apply with the two top-level subtrees on two streams
        out["two_stream_variant"] = time_two_streams(args, cfg, t, par, sflags, xc, prec, V)
    if not args.no_cpu:
        tf = W.orthant_to_full(t, par) if par is not None else t
        x128 = xc.astype(np.complex128)
        if int(np.prod(n)) <= 64 * 64:
            from oracle import toeplitz as OT
            ref = OT.direct_matvec(tf, x128)
            out["rel_l2_vs_fp64_direct_sum"] = float(np.linalg.norm(y - ref) / np.linalg.norm(ref))
        elif int(np.prod(n)) <= 128 ** 3:
            from oracle import embed as OE
            ref = OE.embed_matvec(tf, x128, workers=len(os.sched_getaffinity(0)))
            out["rel_l2_vs_fp64_oracle"] = float(np.linalg.norm(y - ref) / np.linalg.norm(ref))
        else:
            from oracle import toeplitz as OT
            rng = np.random.default_rng(29)
            pts = [tuple(int(v) for v in rng.integers(0, n)) for _ in range(8)]
            vals = OT.direct_points(tf, x128, pts)
            got = np.stack([y[(0, slice(None)) + q] for q in pts])
            out["rel_l2_vs_fp64_oracle_sampled"] = float(np.linalg.norm(got - vals[:, 0]) /
                                                         np.linalg.norm(vals[:, 0]))
    return out


def secondaries(args):
    """Compact figures of the other configurations, measured after the
    headline's timed region (each in its own try: a failure is reported, the
    headline line still prints)."""
    import torch

    from paper_2406_17981_gb300 import btmv as bt
    out = {}
    steps = max(20, min(args.steps, 200))
    for wl in ("d3_128_c3_green_c64", "d3_256_c3_skew_c64", "d2_64_c1_random_c128"):
        t0 = time.perf_counter()
        try:
            out[wl] = compact_single(args, wl, steps)
        except Exception as ex:
            out[wl] = {"error": str(ex)[:300]}
        out[wl]["wall_s"] = time.perf_counter() - t0
        torch.cuda.synchronize()
    t0 = time.perf_counter()
    try:
        sub = argparse.Namespace(**vars(args))
        sub.steps, sub.warmup = max(10, min(args.steps, 50)), 3
        b = run_batched(sub, dist=False)
        out["batched64"] = {k: b[k] for k in ("value", "unit", "ms_per_step")}
        out["batched64"].update({"mode": b["config"]["launch"], "roofline_frac_whole_step": b["roofline"]["frac"],
                                 "persistent_kernel_mode": b["persistent_kernel_mode"],
                                 "sequential_btmv_apply": b["sequential_btmv_apply"]})
    except Exception as ex:
        out["batched64"] = {"error": str(ex)[:300]}
    out["batched64"]["wall_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    try:
        sv = run_serving(argparse.Namespace(**vars(args)), dist=False)
        out["serving200"] = {"matvecs_per_s": sv["value"], "p50_ms": sv["p50_ms"], "p99_ms": sv["p99_ms"],
                             "speedup_vs_one_at_a_time_full": sv["speedup_vs_one_at_a_time_full"],
                             "matvecs": sv["steps"]}
    except Exception as ex:
        out["serving200"] = {"error": str(ex)[:300]}
    out["serving200"]["wall_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    try:
        out["fused_levels"] = run_fused_levels(argparse.Namespace(**vars(args)), dist=False)
    except Exception as ex:
        out["fused_levels"] = {"error": str(ex)[:300]}
    out["fused_levels"]["wall_s"] = time.perf_counter() - t0
    del bt
    return out


def run_batched(args, dist=True):
    """64 uneven d=3 Green instances (each dim from {24..96}, 1..16 rhs,
    complex64) through btmv_apply_batched: one graph replay per step (a
    persistent kernel or parallel per-instance branches, as tuned).  Rate
    counts (instance, rhs) pairs.  Returns the JSON line (rank 0)."""
    import torch

    from paper_2406_17981_gb300 import analysis as A
    from paper_2406_17981_gb300 import btmv as bt
    ws, rank, local = dist_setup(args) if dist else (1, 0, torch.cuda.current_device())
    insts = W.batched_instances()
    plans, xs, ys = [], [], []
    tot_bytes = 0
    for it in insts:
        n, r = it["n"], it["nrhs"]
        t_orth, par = W.green_dyadic_orthant(n, kh=it["kh"])
        p = bt.Plan(n, 3, bt.BTMV_C64, bt.BTMV_ALGO_SPLIT, max_rhs=r)
        p.set_kernel(t_orth, 3, par)
        x = torch.from_numpy(W.random_vector(n, 3, seed=it["x_seed"], nrhs=r).astype(np.complex64)).cuda()
        plans.append(p)
        xs.append(x)
        ys.append(torch.empty_like(x))
        tot_bytes += A.split_pass_bytes(n, 3, r, 8, p.info["symbol_bytes"])["total"]
    handles = [p.handle for p in plans]
    nr = [it["nrhs"] for it in insts]
    pairs = sum(nr)
    t_tune = time.perf_counter()
    bt.btmv_apply_batched(handles, xs, ys, nr)          # first call: autotune + capture
    torch.cuda.synchronize()
    t_tune = time.perf_counter() - t_tune
    tuning = bt.btmv_batch_tuning(handles, xs, ys, nr)
    for _ in range(args.warmup):
        bt.btmv_apply_batched(handles, xs, ys, nr)
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    barrier(ws)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        bt.btmv_apply_batched(handles, xs, ys, nr)
    e1.record()
    torch.cuda.synchronize()
    barrier(ws)
    clocks = sampler.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), ws)
    value = ws * args.steps * pairs / (ms / 1000.0)
    # the same work as one btmv_apply per instance (register kernels where they apply)
    seq_steps = max(3, min(args.steps, 50))
    e0.record()
    for _ in range(seq_steps):
        for p, x, y, r in zip(plans, xs, ys, nr):
            bt.btmv_apply(p.handle, x, y, r)
    e1.record()
    torch.cuda.synchronize()
    seq_ms = e0.elapsed_time(e1) / seq_steps
    # the same batch forced into the one-persistent-kernel mode (a new argument
    # set: fresh outputs), for comparison with the tuner's choice
    os.environ["BTMV_NO_AUTOTUNE"] = "1"
    os.environ["BTMV_BATCH_MODE"] = "0"
    ys0 = [torch.empty_like(x) for x in xs]
    try:
        bt.btmv_apply_batched(handles, xs, ys0, nr)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(seq_steps):
            bt.btmv_apply_batched(handles, xs, ys0, nr)
        e1.record()
        torch.cuda.synchronize()
        pers_ms = e0.elapsed_time(e1) / seq_steps
        pers_stages = bt.btmv_batch_tuning(handles, xs, ys0, nr)["stages"]
    finally:
        del os.environ["BTMV_NO_AUTOTUNE"]
        del os.environ["BTMV_BATCH_MODE"]
    peaks, peak_src = measured_peaks()
    achieved = tot_bytes / (ms / args.steps / 1000.0) / 1e9
    for p in plans:
        p.close()
    if rank != 0:
        return None
    line = {"metric": "batched block Toeplitz matvecs/s ((instance, rhs) pairs, 64 uneven d=3 c=3 Green, complex64)",
            "value": value, "unit": "matvecs/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batched64", "instances": len(insts), "rhs_total": pairs,
                       "dims": list(W.BATCH_DIMS),
                       "launch": ("one persistent kernel per step, captured CUDA graph" if tuning["mode"] == 0 else
                                  "one captured CUDA graph per step whose parallel branches run each "
                                  "instance's own kernels (autotuner's choice)"),
                       "tuning": tuning, "autotune_and_capture_s": t_tune,
                       "l2": "64 instances' vectors, workspaces and symbols are far larger than L2"},
            "roofline": {"bound": "hbm", "kernel": "whole step", "achieved": achieved,
                         "peak": float(peaks["hbm_gbs"]), "unit": "GB/s",
                         "frac": achieved / float(peaks["hbm_gbs"]), "peak_source": f"{peak_src} hbm_gbs",
                         "traffic": None, "algorithmic_bytes_per_step": tot_bytes},
            "sequential_btmv_apply": {"ms_per_step": seq_ms, "matvecs_per_s": pairs / (seq_ms / 1000.0)},
            "persistent_kernel_mode": {"ms_per_step": pers_ms, "matvecs_per_s": pairs / (pers_ms / 1000.0),
                                       "stages": pers_stages},
            "gpu_launches": args.steps * (1 if tuning["mode"] == 0 else tuning["stages"]), "clocks": clocks}
    return line


def run_multirhs(args):
    """16 right-hand sides sharing one Green operator (d = 3, c = 3,
    complex64): the default leaf (register kernels, one rhs per line group),
    the shared-symbol CUDA-core contraction, and the tensor-core contraction.
    Rates count rhs-matvecs per second."""
    import torch

    from paper_2406_17981_gb300 import btmv as bt
    ws, rank, local = dist_setup(args)
    out = {}
    steps = max(5, min(args.steps, 200))
    for n in ((64, 64, 64), (128, 128, 128)):
        r = 16
        t_orth, par = W.green_dyadic_orthant(n, kh=W.KH_GREEN)
        x = torch.from_numpy(W.random_vector(n, 3, seed=31, nrhs=r).astype(np.complex64)).cuda()
        ys = {}
        for name, fl in (("register", 0), ("shared_rhs_cuda_core", bt.BTMV_FLAG_SHARED_RHS),
                         ("tensor_core", bt.BTMV_FLAG_TENSOR_CORE)):
            p = bt.Plan(n, 3, bt.BTMV_C64, bt.BTMV_ALGO_SPLIT, max_rhs=r, flags=fl | bt.BTMV_FLAG_PROFILE)
            p.set_kernel(t_orth, 3, par)
            y = torch.empty_like(x)
            for _ in range(3):
                p.apply(x, y, r)
            torch.cuda.synchronize()
            bt.btmv_profile_read(p.handle)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(steps):
                p.apply(x, y, r)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / steps
            prof = bt.btmv_profile_read(p.handle)
            leaf_us = 1000 * prof["leaf"][0] / max(1, prof["leaf"][1])
            ys[name] = y.cpu().numpy().astype(np.complex128)
            out[f"{n[0]}^3 r{r} {name}"] = {"rhs_matvecs_per_s": r * 1000.0 / ms, "ms_per_step": ms,
                                            "leaf_us_per_launch": leaf_us}
            p.close()
        ref = ys["register"]
        for name in ("shared_rhs_cuda_core", "tensor_core"):
            out[f"{n[0]}^3 r16 {name}"]["rel_diff_vs_register"] = float(
                np.linalg.norm(ys[name] - ref) / np.linalg.norm(ref))
    if rank != 0:
        return None
    best = max(v["rhs_matvecs_per_s"] for k, v in out.items() if k.startswith("128"))
    line = {"metric": "multi-rhs block Toeplitz rhs-matvecs/s (d=3 c=3 Green, 16 rhs, complex64)",
            "value": best, "unit": "matvecs/s", "n_gpus": ws, "steps": steps, "warmup": 3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": {"workload": "multirhs", "nrhs": 16}, "variants": out}
    return line


FUSED_N, FUSED_RHS = (512, 64, 64), 8


def run_fused_levels(args, dist=True):
    """The d = 3 split apply with its last two levels fused into one kernel
    per level-1 node (BTMV_FLAG_FUSED_LEVELS) against the unfused schedule,
    each with one and two streams: n = 512 x 64 x 64, c = 3 Green, complex64,
    8 right-hand sides (each vector 403 MB, past L2).  Rates count
    right-hand-side matvecs per second; the fused kernel's launch time comes
    from the plan's profile events and its algorithmic bytes from
    analysis.fused_pass_bytes (node read and written, symbol once per apply,
    so half of it per launch)."""
    import torch

    from paper_2406_17981_gb300 import analysis as A
    from paper_2406_17981_gb300 import btmv as bt
    ws, rank, local = dist_setup(args) if dist else (1, 0, 0)
    n, r = FUSED_N, FUSED_RHS
    steps = max(5, min(args.steps, 100))
    t_orth, par = W.green_dyadic_orthant(n, kh=W.KH_GREEN)
    xc = W.random_vector(n, 3, seed=37, nrhs=r).astype(np.complex64)
    x = torch.from_numpy(xc).cuda()
    out, ys = {}, {}
    for name, fl in (("unfused", 0), ("fused", bt.BTMV_FLAG_FUSED_LEVELS),
                     ("unfused_two_streams", bt.BTMV_FLAG_TWO_STREAMS),
                     ("fused_two_streams", bt.BTMV_FLAG_FUSED_LEVELS | bt.BTMV_FLAG_TWO_STREAMS)):
        p = bt.Plan(n, 3, bt.BTMV_C64, bt.BTMV_ALGO_SPLIT, max_rhs=r, flags=fl)
        p.set_kernel(t_orth, bt.BTMV_SYM_BLOCK | bt.BTMV_SYM_PARITY, par)
        y = torch.empty_like(x)
        ms = time_plan_apply_rhs(p, x, y, r, steps)
        ys[name] = y
        out[name] = {"rhs_matvecs_per_s": r * 1000.0 / ms, "ms_per_step": ms,
                     "launches_per_apply": p.info["launches_per_apply"]}
        sym_bytes = p.info["symbol_bytes"]
        p.close()
    # the fused kernel alone: profile events around each launch
    p = bt.Plan(n, 3, bt.BTMV_C64, bt.BTMV_ALGO_SPLIT, max_rhs=r,
                flags=bt.BTMV_FLAG_FUSED_LEVELS | bt.BTMV_FLAG_PROFILE)
    p.set_kernel(t_orth, bt.BTMV_SYM_BLOCK | bt.BTMV_SYM_PARITY, par)
    y = torch.empty_like(x)
    time_plan_apply_rhs(p, x, y, r, 1)
    bt.btmv_profile_read(p.handle)
    for _ in range(5):
        p.apply(x, y, r)
    prof = bt.btmv_profile_read(p.handle)
    p.close()
    fb = A.fused_pass_bytes(n, 3, r, 8, sym_bytes)
    per_launch = fb["fused_levels"] / 2
    us = 1000 * prof["fused_levels"][0] / max(1, prof["fused_levels"][1])
    peak = float(measured_peaks()[0]["hbm_gbs"])
    out["fused_kernel"] = {"avg_us": us, "launches": prof["fused_levels"][1], "algo_bytes_per_launch": per_launch,
                           "algo_GBps": per_launch / us / 1e3, "frac_of_measured_hbm": per_launch / us / 1e3 / peak,
                           "share_of_apply": prof["fused_levels"][0] / max(1e-12, sum(v[0] for v in prof.values())),
                           "traffic": ncu_traffic("fused2", "d3_512x64x64_c3_green_c64")}
    out["speedup_fused_vs_unfused"] = out["unfused"]["ms_per_step"] / out["fused"]["ms_per_step"]
    out["speedup_fused_vs_unfused_two_streams"] = (out["unfused_two_streams"]["ms_per_step"] /
                                                   out["fused_two_streams"]["ms_per_step"])
    yf = ys["fused"].cpu().numpy().astype(np.complex128)
    yu = ys["unfused"].cpu().numpy().astype(np.complex128)
    out["rel_l2_fused_vs_unfused"] = float(np.linalg.norm(yf - yu) / np.linalg.norm(yu))
    if not args.no_cpu:
        from oracle import toeplitz as OT
        rng = np.random.default_rng(41)
        pts = [tuple(int(v) for v in rng.integers(0, n)) for _ in range(6)]
        vals = OT.direct_points(W.orthant_to_full(t_orth, par), xc[:1].astype(np.complex128), pts)
        got = np.stack([yf[(0, slice(None)) + q] for q in pts])
        out["rel_l2_vs_fp64_direct_sum_sampled"] = float(np.linalg.norm(got - vals[:, 0]) /
                                                         np.linalg.norm(vals[:, 0]))
    if rank != 0 or not dist:
        return out
    return {"metric": "block Toeplitz rhs-matvecs/s, last two levels fused (d=3 c=3 Green 512x64x64, 8 rhs, complex64)",
            "value": out["fused"]["rhs_matvecs_per_s"], "unit": "matvecs/s", "n_gpus": ws, "steps": steps,
            "warmup": 3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": {"workload": "fused_levels", "n": list(n), "nrhs": r,
                                            "l2": "inputs larger than L2"},
            "variants": out}


def time_plan_apply_rhs(plan, x, y, nrhs, steps):
    """Mean ms of `steps` applies with nrhs right-hand sides (after 3 warm-up applies)."""
    import torch
    for _ in range(3):
        plan.apply(x, y, nrhs)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        plan.apply(x, y, nrhs)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def run_cpu_fig3(args):
    """The paper's wall-clock study (Sec. III, Fig. 3) on the host cores:
    split vs full circulant embedding, d = 1..4, power-of-two sizes, scalar
    random complex generators, scipy.fft on every core this process may use.
    No GPU.  The operation-count ratio R_c (Eq. CompRatio) is printed beside
    each measured ratio."""
    from paper_2406_17981_gb300 import analysis as A
    from paper_2406_17981_gb300 import cpu_study as CS
    if int(os.environ.get("RANK", "0")) != 0:
        return None
    t0 = time.perf_counter()
    rows = CS.study(repeats=3)
    for r in rows:
        r["model_R_c"] = A.ratio_complexity(r["d"], r["n"])
    el = time.perf_counter() - t0
    best = max(r["ratio_embed_over_split"] for r in rows)
    return {"metric": "wall-clock ratio full embedding / split on the host cores (Sec. III study)",
            "value": best, "unit": "ratio", "n_gpus": 0, "steps": len(rows), "warmup": 1,
            "ms_per_step": 1000.0 * el / max(1, len(rows)), "higher_is_better": True, "scaling": "none",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "cpu_fig3", "cores": CS.cores(), "fft": "scipy.fft",
                       "sizes": {str(k): v for k, v in CS.DEFAULT_SIZES.items()}},
            "rows": rows}


def serving_specs(count=200, seed=7):
    """Config: 200 solves, half d=2 c=1 scalar Green on 256^2..1024^2, half
    d=3 c=3 dyadic Green on 32^3..192^3 (7-smooth sizes), BiCGSTAB on
    I - alpha T with ||alpha T|| <= 0.9, tolerance 1e-6, <= 60 matvecs each, Poisson arrivals
    (mean gap 5 ms) so that nearly all solves are in flight together."""
    from paper_2406_17981_gb300 import btmv as bt
    from paper_2406_17981_gb300 import serve
    rng = np.random.default_rng(seed)
    d2 = [256, 320, 384, 512, 640, 768, 1024]
    d3 = [32, 48, 64, 96, 128, 160, 192]
    gens, alphas = {}, {}
    specs = []
    tarr = 0.0
    for k in range(count):
        if k % 2 == 0:
            m = int(rng.choice(d2))
            n, c = (m, m), 1
        else:
            m = int(rng.choice(d3))
            n, c = (m, m, m), 3
        if n not in gens:
            gens[n] = W.green_scalar_orthant(n, W.KH_GREEN) if c == 1 else W.green_dyadic_orthant(n, W.KH_GREEN)
        t, par = gens[n]
        flags = (bt.BTMV_SYM_BLOCK if c == 3 else 0) | bt.BTMV_SYM_PARITY
        if n not in alphas:
            alphas[n] = serve.scaled_alpha(t, par, flags, n, c, target=0.9)
        tarr += float(rng.exponential(0.005))
        specs.append(serve.SolveSpec(n, c, t, par, flags, alphas[n], b_seed=1000 + k, max_matvecs=60,
                                     tol=1e-6, arrival=tarr, name=f"solve{k}"))
    return specs


def run_serving(args, dist=True):
    """Serving: continuous batching of the matvecs of 200 concurrent solves
    (80 GB HBM budget), against the same solves one matvec at a time with
    the plain full embedding.  Returns the JSON line (rank 0)."""
    import torch

    from paper_2406_17981_gb300 import btmv as bt
    from paper_2406_17981_gb300 import serve
    ws, rank, local = dist_setup(args) if dist else (1, 0, torch.cuda.current_device())
    t0 = time.perf_counter()
    specs = serving_specs()
    t_setup = time.perf_counter() - t0
    # untimed warm-up on a few short solves: the first use of each library and
    # torch kernel in a fresh process loads its module
    warm = [serve.SolveSpec(s.n, s.c, s.t, s.parity, s.sym_flags, s.alpha, s.b_seed, 4, s.tol, 0.0, s.name)
            for s in specs[:8]]
    serve.Server(budget_bytes=80 * 10 ** 9, max_inflight=2).run(warm)
    serve.Server(budget_bytes=80 * 10 ** 9, max_inflight=1, algo=bt.BTMV_ALGO_FULL, batched=False).run(warm)
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    res = serve.Server(budget_bytes=80 * 10 ** 9, max_inflight=2).run(specs)
    clocks = sampler.stop()
    base = serve.Server(budget_bytes=80 * 10 ** 9, max_inflight=1, algo=bt.BTMV_ALGO_FULL,
                        batched=False).run(specs)
    if rank != 0:
        return None
    strip = lambda r: {k: v for k, v in r.items() if k not in ("solutions", "rhs")}  # noqa: E731
    line = {"metric": "served block Toeplitz matvecs/s (200 concurrent BiCGSTAB solves, complex64)",
            "value": res["matvecs_per_s"], "unit": "matvecs/s", "n_gpus": ws, "steps": res["matvecs"],
            "warmup": 0, "ms_per_step": 1000.0 * res["wall_s"] / max(1, res["matvecs"]),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "serving200", "solves": len(specs), "budget_bytes": 80 * 10 ** 9,
                       "generator_and_alpha_setup_s": t_setup},
            "serving_split_batched": strip(res),
            "one_at_a_time_full_embedding": strip(base),
            "p50_ms": res["p50_ms"], "p99_ms": res["p99_ms"],
            "speedup_vs_one_at_a_time_full": res["matvecs_per_s"] / base["matvecs_per_s"],
            "clocks": clocks}
    return line


def time_two_streams(args, cfg, t, par, sflags, xc, prec, V):
    """The same split apply with the two top-level subtrees on two streams
    (BTMV_FLAG_TWO_STREAMS): faster when passes and leaves overlap, at the
    cost of d-2 more workspace vectors."""
    import torch

    from paper_2406_17981_gb300 import btmv as bt
    n, c = cfg["n"], cfg["c"]
    if len(n) < 3:
        return None
    p = bt.Plan(n, c, prec, bt.BTMV_ALGO_SPLIT, max_rhs=1, flags=bt.BTMV_FLAG_TWO_STREAMS)
    p.set_kernel(t, sflags, par)
    info = p.info
    npool = max(2, math.ceil(2 * L2_BYTES / (2 * V)) + 1)
    xs = [torch.from_numpy(xc).cuda() for _ in range(npool)]
    ys = [torch.empty_like(xs[0]) for _ in range(npool)]
    steps = max(10, min(args.steps, 500))
    for i in range(5):
        p.apply(xs[i % npool], ys[i % npool], 1)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for i in range(steps):
        p.apply(xs[i % npool], ys[i % npool], 1)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    p.close()
    return {"matvecs_per_s": 1000.0 / ms, "ms_per_step": ms,
            "peak_hbm_bytes": info["symbol_bytes"] + info["workspace_bytes"] + info["table_bytes"] + 2 * V}


def time_plan_apply(plan, x, y, steps):
    """Mean ms of `steps` applies on device buffers (after 3 warm-up applies)."""
    import torch
    for _ in range(3):
        plan.apply(x, y, 1)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        plan.apply(x, y, 1)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def compare_full(args, cfg, t, par, sflags, xc, prec, cdt, V, esz, info_split):
    """The plain full embedding (Sec. I) on the same symbol store as the split
    plan: with the library's own kernels, and with cuFFT transforms
    (BTMV_ALGO_FULL_CUFFT: cuFFT plus the library's pad, multiply and
    projection kernels).  Peak HBM = device memory the plan holds (measured
    as the drop in free memory, cuFFT's work area included) + x and y."""
    import torch

    from paper_2406_17981_gb300 import analysis as A
    from paper_2406_17981_gb300 import btmv as bt
    n, c = cfg["n"], cfg["c"]
    out = {}
    steps = max(10, min(args.steps, 200))
    x = torch.from_numpy(xc).cuda()
    y = torch.empty_like(x)
    for key, algo in (("full_embedding_own", bt.BTMV_ALGO_FULL), ("full_embedding_cufft", bt.BTMV_ALGO_FULL_CUFFT)):
        try:
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
            fp = bt.Plan(n, c, prec, algo, max_rhs=1)
            fp.set_kernel(t, sflags, par)
            finfo = fp.info
            ms = time_plan_apply(fp, x, y, steps)
            resident = free0 - torch.cuda.mem_get_info()[0]
            fb = A.full_pass_bytes(n, c, 1, esz, finfo["symbol_bytes"])
            out[key] = {"matvecs_per_s": 1000.0 / ms, "ms_per_step": ms,
                        "symbol": "compressed" if finfo["compressed"] else "full",
                        "algo_bytes_per_step": fb["total"], "algo_GBps": fb["total"] / (ms / 1000) / 1e9,
                        "peak_hbm_bytes": resident + 2 * V,
                        "peak_hbm_model_bytes": (finfo["symbol_bytes"] + finfo["workspace_bytes"] +
                                                 finfo["table_bytes"] + 2 * V)}
            if algo == bt.BTMV_ALGO_FULL_CUFFT:
                out[key]["kernels"] = "cuFFT C2C (cufftPlanMany, c batched) + own pad / multiply / projection"
            fp.close()
            del fp
        except Exception as ex:  # report, never fail the bench line
            out[key] = {"error": str(ex)[:200]}
    return out


def like_for_like_memory(args, cfg, t, par, sflags, prec, V, n, c, split_peak, full_peak):
    """Peak-HBM ratio full embedding / split with the same symbol storage on
    both sides, measured (both on the mirror-compressed store when the
    workload has parity symmetry), beside the model of Eq. MemRatio /
    MemRatioSym extended to c x c blocks: symbol S in units of s elements,
    vectors c per unit; the paper's accounting (embedding in place, split
    holding x) and this library's (x and y both held by the caller)."""
    from paper_2406_17981_gb300 import analysis as A
    d = len(n)
    s = int(np.prod(n))
    bsym = bool(sflags & 1)
    S_comp = A.symbol_bytes(n, c, 1, bsym, True) / s
    S_full = A.symbol_bytes(n, c, 1, bsym, False) / s
    out = {"measured_same_store": full_peak / split_peak,
           "store": "compressed" if sflags & 2 else "full"}
    for name, S in (("compressed", S_comp), ("full", S_full)):
        out[f"model_paper_accounting_{name}"] = A.ratio_memory_blocks(d, c, S, S)
        out[f"model_x_and_y_held_{name}"] = (2 ** d * c + 2 * c + S) / ((d + 1) * c + S)
    return out


if __name__ == "__main__":
    main()
