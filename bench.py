"""Benchmark: grid cells/s of the thin-disk forces F_r + F_phi on one GB300.

Workload: the 2048 x 4096 log-polar disk (r in [0.01, 100]; sigma =
exp(0.5 g) e^{-r/3}, g a seeded unit-variance k^-3 Gaussian field), FP32, with
kernel spectra built once in FP64 before timing.  A timed step is one forward
evaluation (sg_forces: rows -> columns -> inverse rows) of the whole grid;
the adjoint (sg_forces_backward) and the FP64 path are timed the same way and
reported beside it.  The L2 (126 MB) is flushed before every timed step,
outside the step's event pair, by a 256 MB write followed by a 256 MB read:
the step starts on a cold L2 that holds no dirty line of the flush.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank solves its own disk (replicas: the path
does not shard); the timed region is bracketed by barriers and the max over
ranks is used.  --impl reference times the FP64 CPU oracle (direct O(N^2)
sum over oracle-built kernels) on the host cores, on bounded samples of
target cells, rank 0 only.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "grid cells/s of F_r+F_phi (FP32 vs FP64, 1 GB300) at stated rel-L2; % HBM roofline"
WORKLOAD = "lognormal-grf-2048x4096"
NU, NPHI, R_IN, R_OUT, SEED = 2048, 4096, 0.01, 100.0, 1509
# algorithmic bytes per cell of the three forward passes in FP32 (reads and
# writes of the minimal data each pass must move, symmetry-reduced spectra)
BYTES_PER_CELL = {"rows": 8.0, "cols": 20.0, "inv_rows": 16.0}
# DRAM bytes (read + write) of one launch of the dominant pass at 2048 x 4096
# FP32, from one ncu capture of the bench command itself, valid only for the
# kernel sources it was taken on (kernel_sources_sha below).
# dense TF32 tensor rate per dense BF16 rate (nominal 1.1 / 2.25 PFLOP/s on GB300)
TF32_PER_BF16 = 1.1 / 2.25

PASS_TRAFFIC = {"pass": "cols", "sources_sha256": "71d599da13166125", "bytes_per_launch": 100.792320e6 + 7.000576e6}


def kernel_sources_sha(texts=None) -> str:
    """Hash of the pass kernels' sources (fftconv.cu, sg_common.cuh) with
    comments and white space removed: the recorded DRAM traffic stays valid
    through edits that leave the code itself unchanged."""
    import hashlib
    import re

    if texts is None:
        texts = []
        for f in ("fftconv.cu", "sg_common.cuh"):
            with open(os.path.join(ROOT, "paper_1509_01450_gb300", "csrc", f)) as fh:
                texts.append(fh.read())
    h = hashlib.sha256()
    for text in texts:
        text = re.sub(r"/\*.*?\*/", "", re.sub(r"//[^\n]*", "", text), flags=re.S)
        h.update("".join(text.split()).encode())
    return h.hexdigest()[:16]


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, device=None) -> float:
    """Largest x over the ranks of the default process group (x itself when
    there is no group or it has one rank).  Every rank must call it."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(world_size: int, cells_per_rank: int, ms_max: float) -> float:
    """cells/s of the whole job: every rank processes its own disk of
    cells_per_rank cells per step; the slowest rank's step time counts."""
    return world_size * cells_per_rank / (ms_max * 1e-3)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.rows = []
        if self.proc is None:
            return
        time.sleep(0.2)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        for line in out.splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def summary(self):
        rows = getattr(self, "rows", [])
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def cpu_baseline(n_targets: int = 2048, seed: int = 0):
    """FP64 oracle (direct sum over oracle-built kernels) on the host cores,
    on n_targets sampled cells of the same 2048 x 4096 workload."""
    import numpy as np

    import oracle
    import workloads

    u_min, du = workloads.grid_params(NU, R_IN, R_OUT)
    r, phi = workloads.centres(NU, NPHI, u_min, du)
    sigma = workloads.lognormal_disk(r, phi, SEED)
    t0 = time.time()
    Kr, Kp = oracle.kernels(NU, NPHI, du)
    t_table = time.time() - t0
    tg = np.random.default_rng(seed).choice(NU * NPHI, n_targets, replace=False)
    t0 = time.time()
    oracle.direct_sum(sigma, Kr, Kp, targets=tg)
    dt = time.time() - t0
    # the oracle's FFT evaluation of the same convolution (numpy's FFT as a
    # library step): the whole grid, a second and faster CPU figure
    t0 = time.time()
    oracle.fft_conv(sigma, Kr, Kp)
    dt_fft = time.time() - t0
    return {"value": n_targets / dt, "unit": "cells/s", "cores": oracle.max_threads(), "kind": "oracle",
            "sample": f"{n_targets} target cells of the {NU}x{NPHI} grid, FP64 direct sum over all "
                      f"{NU * NPHI} source cells; oracle kernel table built once beforehand ({t_table:.1f} s)",
            "fft": {"value": NU * NPHI / dt_fft, "unit": "cells/s", "ms_per_step": 1e3 * dt_fft,
                    "sample": "the whole grid by the oracle's numpy FFT convolution (FP64, one thread)"}}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np

    import oracle
    import workloads

    u_min, du = workloads.grid_params(NU, R_IN, R_OUT)
    r, phi = workloads.centres(NU, NPHI, u_min, du)
    sigma = workloads.lognormal_disk(r, phi, SEED)
    Kr, Kp = oracle.kernels(NU, NPHI, du)
    per_step = max(8, 4096 // max(args.steps, 1))
    rng = np.random.default_rng(0)
    for _ in range(args.warmup):
        oracle.direct_sum(sigma, Kr, Kp, targets=rng.choice(NU * NPHI, per_step, replace=False))
    t0 = time.time()
    for _ in range(args.steps):
        oracle.direct_sum(sigma, Kr, Kp, targets=rng.choice(NU * NPHI, per_step, replace=False))
    dt = time.time() - t0
    value = per_step * args.steps / dt
    line = {"metric": METRIC, "impl": "reference", "value": value, "unit": "cells/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "nu": NU, "nphi": NPHI, "r_in": R_IN, "r_out": R_OUT, "seed": SEED},
            "cpu_baseline": {"value": value, "unit": "cells/s", "cores": oracle.max_threads(), "kind": "oracle",
                             "sample": f"{per_step} sampled target cells per step, FP64 direct sum"},
            "e2e": {"value": value, "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def host_link(torch, dev, h2d_bytes: int, d2h_bytes: int, reps: int = 20):
    """The host link's own ceiling for the end-to-end step's traffic: plain
    pinned copies (cudaMemcpyAsync through torch) of h2d_bytes in and
    d2h_bytes out, each alone and both at once on two streams, timed with
    CUDA events (GB/s per direction)."""
    hi = torch.empty(h2d_bytes // 4, dtype=torch.float32).pin_memory()
    ho = torch.empty(d2h_bytes // 4, dtype=torch.float32).pin_memory()
    di = torch.empty(h2d_bytes // 4, dtype=torch.float32, device=dev)
    do = torch.empty(d2h_bytes // 4, dtype=torch.float32, device=dev)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()

    def run(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    def both():
        with torch.cuda.stream(s1):
            di.copy_(hi, non_blocking=True)
        with torch.cuda.stream(s2):
            ho.copy_(do, non_blocking=True)
        torch.cuda.current_stream().wait_stream(s1)
        torch.cuda.current_stream().wait_stream(s2)

    t_in = run(lambda: di.copy_(hi, non_blocking=True))
    t_out = run(lambda: ho.copy_(do, non_blocking=True))
    t_both = run(both)
    # one call reads all of sigma before its column pass and writes F only
    # after it: its copies follow one another (serial_ms); the two
    # directions overlap only across consecutive calls (concurrent_ms)
    return {"h2d_gbs": h2d_bytes / (t_in * 1e-3) / 1e9, "d2h_gbs": d2h_bytes / (t_out * 1e-3) / 1e9,
            "h2d_ms": t_in, "d2h_ms": t_out, "serial_ms": t_in + t_out, "concurrent_ms": t_both,
            "bound_ms_per_step": t_in + t_out,
            "how": f"pinned cudaMemcpyAsync of {h2d_bytes} B host-to-device and {d2h_bytes} B device-to-host, "
                   "alone and concurrently on two streams"}


class L2Flush:
    """Empties L2 between timed steps: a 256 MB write (the flush), then a
    256 MB read, so that the step starts on a cold L2 holding no dirty lines
    of the flush (whose write-back would otherwise fall into the step)."""

    def __init__(self, torch, dev, mb: int = 256):
        n = mb * 1024 * 1024 // 4
        self.w = torch.empty(n, dtype=torch.float32, device=dev)
        self.r = torch.ones(n, dtype=torch.float32, device=dev)
        self.torch = torch

    def __call__(self):
        self.w.zero_()
        self.torch.sum(self.r)


def batch_throughput(torch, dev, flush, peak_gbs, n_disks: int = 256, seed: int = 1450, reps: int = 10):
    """cells/s of the batching form: n_disks exponential disks with spirals,
    N_u in {128..1024} and N_phi in {256..2048} drawn per disk, one plan per
    distinct size, all enqueued by one sg_forces_batched call; timed eagerly
    and as a replayed CUDA graph of that call (L2 flushed before each)."""
    import tempfile

    import workloads
    from paper_1509_01450_gb300 import Plan, SgError, batch_prepare, batch_tune, forces_batched

    disks = workloads.batch_disks(n_disks, seed)
    plans = {}
    for d in disks:
        if (d.nu, d.nphi) not in plans:
            plans[(d.nu, d.nphi)] = Plan(d.nu, d.nphi, d.u_min, d.du, 1.0, "float32").build()
    sig = [torch.tensor(d.sigma(), dtype=torch.float32, device=dev) for d in disks]
    outs = [(torch.empty_like(s), torch.empty_like(s)) for s in sig]
    items = [(plans[(d.nu, d.nphi)], s, a, b) for d, s, (a, b) in zip(disks, sig, outs)]
    cells = sum(d.nu * d.nphi for d in disks)
    stream = torch.cuda.current_stream()

    def timed(fn):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for a, b in ev:
            flush()
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize()
        return statistics.mean(a.elapsed_time(b) for a, b in ev)

    # the persistent path's schedule, tuned for these sizes once per machine
    # (the file keeps it for later runs)
    cache = os.path.join(tempfile.gettempdir(), "sg_batch_schedules.txt")
    try:
        tune_ms = batch_tune(items, cache)
        persistent = True
    except SgError:
        tune_ms, persistent = None, False
    for _ in range(3):
        forces_batched(items, stream=stream)
    eager_ms = timed(lambda: forces_batched(items, stream=stream))
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        forces_batched(items, stream=side)
    stream.wait_stream(side)
    torch.cuda.synchronize()
    with torch.cuda.graph(g):
        forces_batched(items, stream=torch.cuda.current_stream())
    g.replay()
    torch.cuda.synchronize()
    graph_ms = timed(g.replay)
    # the same batch with its N_phi = 256 disks on short_dft plans (their rows
    # as tensor-core DFT products, two batched launches beside the persistent
    # kernels), replayed from a CUDA graph
    tcp = {}
    for d in disks:
        if d.nphi == 256 and (d.nu, d.nphi) not in tcp:
            tcp[(d.nu, d.nphi)] = Plan(d.nu, d.nphi, d.u_min, d.du, 1.0, "float32").build(short_dft=1)
    items_tc = [(tcp.get((d.nu, d.nphi), plans[(d.nu, d.nphi)]), s, a, b) for d, s, (a, b) in zip(disks, sig, outs)]
    tc_ms = None
    try:
        batch_prepare(items_tc)
        forces_batched(items_tc, stream=stream)
        g2 = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g2):
            forces_batched(items_tc, stream=torch.cuda.current_stream())
        g2.replay()
        torch.cuda.synchronize()
        tc_ms = timed(g2.replay)
    except SgError:
        pass
    # the three passes' algorithmic bytes over all disks, against the copy peak
    bytes_ = sum(BYTES_PER_CELL.values()) * cells
    return {"workload": f"{n_disks} disks, seed {seed}, {len(plans)} sizes, {cells} cells", "unit": "cells/s",
            "value": cells / (eager_ms * 1e-3), "ms": eager_ms,
            "graph_value": cells / (graph_ms * 1e-3), "graph_ms": graph_ms,
            "short_dft_rows_256": None if tc_ms is None else {
                "graph_ms": tc_ms, "graph_value": cells / (tc_ms * 1e-3), "launches": 5,
                "disks": sum(1 for d in disks if d.nphi == 256)},
            "persistent": persistent, "launches": 3 if persistent else 3 * n_disks,
            "tune_ms": {"default": tune_ms[0], "tuned": tune_ms[1]} if tune_ms else None,
            "graph_path_roofline_frac": bytes_ / (graph_ms * 1e-3) / 1e9 / peak_gbs}


def short_dft_measure(torch, dev, timed, n, nu: int = 4096, nphi: int = 256):
    """The short_dft option (the row transforms as split-TF32 DFT-matrix
    products on tcgen05) beside the FFT rows on an nu x nphi lognormal disk:
    forward and adjoint step times (L2 flushed before each), the row passes'
    CUDA-event times, their tensor throughput, and the two forms' agreement."""
    import workloads
    from paper_1509_01450_gb300 import Plan

    u_min, du = workloads.grid_params(nu, R_IN, R_OUT)
    r, phi = workloads.centres(nu, nphi, u_min, du)
    s = torch.tensor(workloads.lognormal_disk(r, phi, SEED), dtype=torch.float32, device=dev)
    gr, gp = torch.randn_like(s), torch.randn_like(s)
    out = {"workload": f"lognormal-grf-{nu}x{nphi}", "unit": "cells/s"}
    res = {}
    for tag, opt in (("tensor_cores", 1), ("fft", 0)):
        plan = Plan(nu, nphi, u_min, du, 1.0, "float32").build(short_dft=opt)
        Fr, Fp, gs = torch.empty_like(s), torch.empty_like(s), torch.empty_like(s)
        for _ in range(3):
            plan.forces(s, Fr, Fp)
            plan.backward(gr, gp, gs)
        fwd = timed(lambda: plan.forces(s, Fr, Fp), n)
        bwd = timed(lambda: plan.backward(gr, gp, gs), n)
        passes = [plan.forces_timed(s, Fr, Fp) for _ in range(n)]
        plan.check()
        res[tag] = (Fr.double(), Fp.double())
        out[tag] = {"value": nu * nphi / (fwd * 1e-3), "ms_per_step": fwd, "backward_ms_per_step": bwd,
                    "rows_ms": statistics.mean(p[0] for p in passes), "inv_rows_ms": statistics.mean(p[2] for p in passes)}
    (a, b), (c, d) = res["tensor_cores"], res["fft"]
    out["rel_l2_tensor_cores_vs_fft"] = math.sqrt(float(((a - c) ** 2).sum() + ((b - d) ** 2).sum()) /
                                                  float((c ** 2).sum() + (d ** 2).sum()))
    # tensor work per forward step: the DFT products (2 nu N^2 flops each; P1
    # one, P3 two), each executed as three TF32 products (hi hi, hi lo, lo hi)
    tc = out["tensor_cores"]
    flops = {"rows": 2.0 * nu * nphi * nphi, "inv_rows": 2 * 2.0 * nu * nphi * nphi}
    peaks, kind = measured_peaks()
    tf32_peak = float(peaks.get("bf16_tflops", 1900.0)) * TF32_PER_BF16
    for k in ("rows", "inv_rows"):
        t = tc[k + "_ms"] * 1e-3
        tc[k + "_tflops_executed"] = 3 * flops[k] / t / 1e12
        tc[k + "_frac_of_tf32_peak"] = 3 * flops[k] / t / 1e12 / tf32_peak
    out["tf32_peak_tflops"] = {"value": tf32_peak, "from": f"bf16 {kind} x {TF32_PER_BF16:.3f} (nominal TF32 / BF16)"}
    return out


def run_passes_only(args):
    """The forward and adjoint passes of the bench workload alone, for an
    external profiler: one plan, W + K forward steps, then W + K adjoint
    steps (same density, L2 flushed before each), the plan's error flag
    checked at the end.  Prints one JSON line of mean step times; it is not
    a bench line."""
    import torch

    import workloads
    from paper_1509_01450_gb300 import Plan, build as cuda_build

    cuda_build.build()
    dev = torch.device("cuda", 0)
    u_min, du = workloads.grid_params(NU, R_IN, R_OUT)
    r, phi = workloads.centres(NU, NPHI, u_min, du)
    plan = Plan(NU, NPHI, u_min, du, 1.0, "float32").build(short_dft=1 if args.short_dft else 0)
    sigma = torch.tensor(workloads.lognormal_disk(r, phi, SEED), dtype=torch.float32, device=dev)
    Fr, Fp = torch.empty_like(sigma), torch.empty_like(sigma)
    gs = torch.empty_like(sigma)
    flush = L2Flush(torch, dev)
    out = {"workload": WORKLOAD, "mode": "passes only", "short_dft": bool(args.short_dft)}
    for name, fn in (("forward_ms", lambda: plan.forces(sigma, Fr, Fp)), ("backward_ms", lambda: plan.backward(Fr, Fp, gs))):
        for _ in range(args.warmup):
            flush()
            fn()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for a, b in ev:
            flush()
            a.record()
            fn()
            b.record()
        torch.cuda.synchronize()
        out[name] = statistics.mean(a.elapsed_time(b) for a, b in ev)
    plan.check()
    print(json.dumps(out), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)

    import workloads
    from paper_1509_01450_gb300 import Plan, build as cuda_build

    cuda_build.build()
    u_min, du = workloads.grid_params(NU, R_IN, R_OUT)
    r, phi = workloads.centres(NU, NPHI, u_min, du)
    sigma_np = workloads.lognormal_disk(r, phi, SEED + rank)
    t0 = time.time()
    plan = Plan(NU, NPHI, u_min, du, 1.0, "float32").build()
    torch.cuda.synchronize()
    build_s = time.time() - t0
    sigma = torch.tensor(sigma_np, dtype=torch.float32, device=dev)
    Fr = torch.empty_like(sigma)
    Fp = torch.empty_like(sigma)
    flush = L2Flush(torch, dev)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    for _ in range(args.warmup):
        plan.forces(sigma, Fr, Fp)
    torch.cuda.synchronize()
    # the step's three launches captured once in a CUDA graph, so that no
    # host-side delay between them falls inside a timed step
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        plan.forces(sigma, Fr, Fp)
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize()

    # ---- timed region: K forward steps, each bracketed by its own events --
    stream = torch.cuda.current_stream()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    with ClockSampler(dev.index) as clk:
        barrier()
        torch.cuda.synchronize()
        w0 = time.time()
        for k in range(args.steps):
            flush()
            starts[k].record(stream)
            graph.replay()
            ends[k].record(stream)
        torch.cuda.synchronize()
        barrier()
        wall = time.time() - w0
    plan.check()  # no pass of the timed steps gave up waiting for its copies
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    ms = max_over_ranks(sum(step_ms) / len(step_ms), dev)
    cells = NU * NPHI
    value = whole_job_value(ws, cells, ms)

    # ---- per-pass durations (roofline of the dominant kernel) -------------
    passes = []
    for _ in range(max(20, min(args.steps, 200))):
        flush()
        passes.append(plan.forces_timed(sigma, Fr, Fp))
    p_rows = statistics.mean(p[0] for p in passes)
    p_cols = statistics.mean(p[1] for p in passes)
    p_inv = statistics.mean(p[2] for p in passes)
    peaks, peak_kind = measured_peaks()
    peak = float(peaks.get("hbm_gbs", 6800.0))
    dom_name, dom_ms = max((("cols", p_cols), ("rows", p_rows), ("inv_rows", p_inv)), key=lambda x: x[1])
    achieved = BYTES_PER_CELL[dom_name] * cells / (dom_ms * 1e-3) / 1e9
    total_bytes = sum(BYTES_PER_CELL.values()) * cells
    traffic = None
    if (dom_name == PASS_TRAFFIC["pass"] and (NU, NPHI) == (2048, 4096)
            and kernel_sources_sha() == PASS_TRAFFIC["sources_sha256"]):
        traffic = PASS_TRAFFIC["bytes_per_launch"]

    # ---- adjoint and FP64, same protocol ----------------------------------
    def timed(fn, n):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
        for s, e in ev:
            flush()
            s.record()
            fn()
            e.record()
        torch.cuda.synchronize()
        return statistics.mean(s.elapsed_time(e) for s, e in ev)

    gr = torch.randn_like(sigma)
    gp = torch.randn_like(sigma)
    gs = torch.empty_like(sigma)
    for _ in range(3):
        plan.backward(gr, gp, gs)
    bwd_ms = timed(lambda: plan.backward(gr, gp, gs), max(20, min(args.steps, 200)))
    bpasses = []
    for _ in range(max(20, min(args.steps, 200))):
        flush()
        bpasses.append(plan.backward_timed(gr, gp, gs))
    bwd_pass_ms = {k: statistics.mean(b[i] for b in bpasses) for i, k in enumerate(("rows", "cols", "inv_rows"))}
    plan64 = Plan(NU, min(NPHI, 4096), u_min, du, 1.0, "float64").build()
    s64 = sigma.double()
    f64r, f64p = torch.empty_like(s64), torch.empty_like(s64)
    for _ in range(3):
        plan64.forces(s64, f64r, f64p)
    fp64_ms = timed(lambda: plan64.forces(s64, f64r, f64p), 20)
    # FP32 accuracy against the FP64 GPU path on the same input
    plan.forces(sigma, Fr, Fp)
    plan64.forces(s64, f64r, f64p)
    torch.cuda.synchronize()
    num = float(((Fr.double() - f64r) ** 2).sum() + ((Fp.double() - f64p) ** 2).sum())
    den = float((f64r ** 2).sum() + (f64p ** 2).sum())
    rel_fp32_vs_fp64 = math.sqrt(num / den)
    # the compensated FP32 plan (double-float passes; FP64 fields): its cost
    # beside the FP32 and FP64 steps, and its accuracy against FP64
    planc = Plan(NU, min(NPHI, 4096), u_min, du, 1.0, "float32x2").build()
    fcr, fcp = torch.empty_like(s64), torch.empty_like(s64)
    for _ in range(3):
        planc.forces(s64, fcr, fcp)
    comp_ms = timed(lambda: planc.forces(s64, fcr, fcp), 20)
    gcs, gr64, gp64 = torch.empty_like(s64), gr.double(), gp.double()
    for _ in range(3):
        planc.backward(gr64, gp64, gcs)
    comp_bwd_ms = timed(lambda: planc.backward(gr64, gp64, gcs), 20)
    planc.forces(s64, fcr, fcp)
    torch.cuda.synchronize()
    num = float(((fcr - f64r) ** 2).sum() + ((fcp - f64p) ** 2).sum())
    rel_comp_vs_fp64 = math.sqrt(num / den)
    del planc, fcr, fcp, gcs, gr64, gp64
    # the same with the kernels stored at weighting p = 2 (the e^{2u} form)
    plan_p2 = Plan(NU, NPHI, u_min, du, 1.0, "float32").build(weight_p=2)
    plan_p2.forces(sigma, Fr, Fp)
    torch.cuda.synchronize()
    num = float(((Fr.double() - f64r) ** 2).sum() + ((Fp.double() - f64p) ** 2).sum())
    rel_fp32_p2 = math.sqrt(num / den)
    del plan64, plan_p2, s64, f64r, f64p

    # ---- build options: one-sided edge slopes and the origin wedge (one more
    # kernel per step each), the potential and the Cartesian scheme (the same
    # passes on other tables), and the kernel variants (only the one-time
    # build differs) -----------------------------------------------------------
    variants = {}
    sigma_w = torch.full((NPHI,), float(sigma_np[0].mean()), dtype=torch.float32, device=dev)
    gsw = torch.empty_like(sigma_w)
    sigma_cart = torch.zeros_like(sigma)  # N_x x 2 N_y with the y-padding zero
    sigma_cart[:, : NPHI // 2] = sigma[:, : NPHI // 2]
    for name, kw in (("sim_ntpz19", {"n_tpz": 19}), ("particle", {"kind": "particle"}),
                     ("particle_plus", {"kind": "particle+"}),
                     ("softened", {"kind": "softened", "soften": 0.015 * 64 / NU}),
                     ("radial_edges_onesided", {"radial_edges": 1}),
                     ("origin_wedge", {"radial_edges": 1, "wedge": 1}),
                     ("potential", {"kind": "potential", "weight_p": 1}),
                     ("cartesian", {"kind": "cartesian"})):
        t0 = time.time()
        h = 2.0 / NU if name == "cartesian" else du  # Cartesian: [-1, 1] in x, square cells
        pv = Plan(NU, NPHI, u_min, h, 1.0, "float32").build(**kw)
        torch.cuda.synchronize()
        entry = {"build_s": time.time() - t0}
        if name in ("radial_edges_onesided", "origin_wedge", "potential", "cartesian"):
            if name == "origin_wedge":
                fwd = lambda: pv.forces_wedge(sigma, sigma_w, Fr, Fp)
                bwd = lambda: pv.backward_wedge(gr, gp, gs, gsw)
            else:
                s_in = sigma_cart if name == "cartesian" else sigma
                fwd = lambda: pv.forces(s_in, Fr, Fp)
                bwd = lambda: pv.backward(gr, gp, gs)
            for _ in range(3):
                fwd()
            ems = timed(fwd, max(20, min(args.steps, 200)))
            for _ in range(3):
                bwd()
            ebms = timed(bwd, max(20, min(args.steps, 200)))
            # the Cartesian plan's cells are N_x x N_y: half the plan's columns
            ccells = cells // 2 if name == "cartesian" else cells
            entry.update({"value": ws * ccells / (ems * 1e-3), "unit": "cells/s", "ms_per_step": ems,
                          "extra_ms_vs_default": ems - ms, "backward_ms_per_step": ebms,
                          "backward_extra_ms_vs_default": ebms - bwd_ms})
            if name == "cartesian":
                entry["grid"] = f"{NU} x {NPHI // 2} square cells (plan {NU} x {NPHI}, y zero-padded)"
        variants[name] = entry
        del pv

    # ---- short azimuthal transforms on the tensor cores (build option
    # short_dft) beside the FFT rows, on the largest N_phi = 256 grid ---------
    short = short_dft_measure(torch, dev, timed, max(20, min(args.steps, 200)))

    # ---- end to end through the C ABI with host buffers --------------------
    sig_h = torch.tensor(sigma_np, dtype=torch.float32).pin_memory()
    fr_h = torch.empty_like(sig_h).pin_memory()
    fp_h = torch.empty_like(sig_h).pin_memory()
    for _ in range(3):
        plan.forces_host(sig_h, fr_h, fp_h)
    n_e2e = max(10, min(args.steps, 100))
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(n_e2e):
        plan.forces_host(sig_h, fr_h, fp_h)
    e1.record()
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / n_e2e
    e2e_value = ws * cells / (e2e_ms * 1e-3)
    link = host_link(torch, dev, cells * 4, 2 * cells * 4)

    # ---- batching form: 256 uneven disks through sg_forces_batched ----------
    batch = None if args.no_batch else batch_throughput(torch, dev, flush, peak)

    if rank == 0:
        clocks = clk.summary()
        line = {
            "metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "nu": NU, "nphi": NPHI, "r_in": R_IN, "r_out": R_OUT, "seed": SEED,
                       "kernel_weight_p": 0, "l2": "flushed by a 256 MB write, then a 256 MB read, before every timed step (cold, clean L2)",
                       "step": "one sg_forces (three kernels) replayed from a CUDA graph",
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
            "roofline": {"bound": "hbm", "kernel": f"forward {dom_name} pass", "achieved": achieved, "peak": peak,
                         "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                         "algorithmic_bytes_per_cell": BYTES_PER_CELL[dom_name]},
            "path_roofline": {"bytes_per_cell": sum(BYTES_PER_CELL.values()),
                              "achieved_gbs": total_bytes / (ms * 1e-3) / 1e9,
                              "frac": total_bytes / (ms * 1e-3) / 1e9 / peak},
            "pass_ms": {"rows": p_rows, "cols": p_cols, "inv_rows": p_inv},
            "backward": {"value": ws * cells / (bwd_ms * 1e-3), "unit": "cells/s", "ms_per_step": bwd_ms,
                         "pass_ms": bwd_pass_ms,
                         "path_roofline_frac": total_bytes / (bwd_ms * 1e-3) / 1e9 / peak},
            "fp64": {"value": ws * cells / (fp64_ms * 1e-3), "unit": "cells/s", "ms_per_step": fp64_ms,
                     "fp32_speedup": fp64_ms / ms},
            "compensated_fp32": {"value": ws * cells / (comp_ms * 1e-3), "unit": "cells/s", "ms_per_step": comp_ms,
                                 "backward_ms_per_step": comp_bwd_ms, "cost_vs_fp32": comp_ms / ms,
                                 "speedup_vs_fp64": fp64_ms / comp_ms, "vs_fp64_gpu_rel_l2": rel_comp_vs_fp64},
            "accuracy": {"fp32_vs_fp64_gpu_rel_l2": rel_fp32_vs_fp64, "fp32_weight_p2_vs_fp64_gpu_rel_l2": rel_fp32_p2,
                         "compensated_vs_fp64_gpu_rel_l2": rel_comp_vs_fp64},
            "build_s": build_s,
            "build_options": variants,
            "batched": batch,
            "short_dft": short,
            "e2e": {"value": e2e_value, "unit": "cells/s", "ms_per_step": e2e_ms,
                    "h2d_bytes_per_step": cells * 4, "d2h_bytes_per_step": 2 * cells * 4,
                    "host_link": link, "frac_of_link_bound": link["bound_ms_per_step"] / e2e_ms},
            "gpu_launches": 3 * args.steps,
            "clocks": clocks,
            "wall_s_timed_region": wall,
        }
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(args.cpu_targets)
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--cpu-targets", type=int, default=2048)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 256-disk batching measurement")
    ap.add_argument("--size", default=None, help="NUxNPHI override (profiling runs only; not a bench line)")
    ap.add_argument("--passes-only", action="store_true",
                    help="time only the forward and adjoint passes (for profiler captures; not a bench line)")
    ap.add_argument("--short-dft", action="store_true",
                    help="with --passes-only: the plan's row transforms on the tensor cores (N_phi <= 256)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.size:
        global NU, NPHI, WORKLOAD
        NU, NPHI = (int(x) for x in args.size.lower().split("x"))
        WORKLOAD = f"lognormal-grf-{NU}x{NPHI} (profiling size)"
    if args.impl == "reference":
        return run_reference(args)
    if args.passes_only:
        return run_passes_only(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
