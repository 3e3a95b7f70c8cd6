"""Benchmark: D3Q19 + immersed-boundary MLUPS on one GB300.

One step = one full immersed-boundary cycle of the method (per-cell area and
volume, membrane forces + spreading, fused stream-collide with force,
interpolation + advance) over the 256x128x64 micropost-filter workload
(62 cells, 120 bead spheres), FP32 populations.  Inputs are resident in HBM;
the populations (2 x 159 MB) are larger than the 126 MB L2.

After W warm-up steps the state is saved and K steps are timed twice from it:
first as CUDA-graph replays (the reported `value`), then with CUDA events
around every kernel launch (per-kernel durations and the roofline of the
stream-collide kernel).  `cycle_frac` is the whole cycle's MLUPS at 152 bytes
per node against the measured HBM copy bandwidth.

The same line carries short fixed windows of the other single-GPU workloads
(`workloads`): the 512x256x128 filter with FP32, FP16 and BF16 population
storage (cycle MLUPS, stream-collide fraction of the HBM bandwidth at 152 or
76 bytes per fluid node, 16-bit over FP32 ratios) and the batched 24-channel
gap sweep; the oracle's single-thread figure sits beside the all-core one.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]

Multi-GPU: the path is run as independent replicas (one per rank, no
collective in the data path); `value` is the total over ranks.
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

BYTES_PER_NODE = {"f32": 152, "f16": 76, "bf16": 76}   # 19 reads + 19 writes per fluid node update
METRIC = "D3Q19+IBM MLUPS on 1 GB300 (% HBM roofline); adjoint/forward step ratio"


def make_workload(name: str):
    """The channels of a workload (one, or the batched sweep's 24)."""
    from paper_1110_0995_gb300 import scene

    if name == "micropost_filter_256x128x64":
        return [scene.micropost_filter(seed=11)]
    if name == "micropost_filter_512x256x128":
        return [scene.micropost_filter_large(seed=31)]
    if name == "channel_32x16x64_1rbc":
        return [scene.channel_plain(seed=1)]
    if name == "gap_sweep_24ch":
        return scene.gap_sweep(seed=21)
    raise ValueError(name)


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        time.sleep(0.2)
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]
        else:
            self.lines = []

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            parts = [p.strip() for p in l.split(",")]
            if len(parts) < 6:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[2:6]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        # samples taken while the GPU was busy (the sampler starts slightly before the region)
        busy = sorted(sm)[len(sm) // 4:] or sm
        return {"sm_mhz": statistics.median(busy), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_sample_scene(budget_nodes: int):
    """A smaller instance of the filter workload (same post geometry family,
    cell density, force) for the CPU oracle, about `budget_nodes` lattice nodes."""
    from paper_1110_0995_gb300 import scene

    for dims, cols, rows, nr, nc in [((256, 128, 64), 4, 3, 60, 2), ((128, 64, 64), 2, 2, 15, 1),
                                     ((64, 64, 64), 1, 2, 8, 0), ((64, 32, 32), 1, 1, 2, 0),
                                     ((32, 32, 16), 1, 1, 1, 0)]:
        n = dims[0] * dims[1] * dims[2]
        if n <= budget_nodes:
            return scene.micropost_filter(seed=11, dims=dims, cols=cols, rows=rows, n_rbc=nr, n_ctc=nc), n
    return scene.micropost_filter(seed=11, dims=(32, 32, 16), cols=1, rows=1, n_rbc=1, n_ctc=0), 32 * 32 * 16


def time_oracle(sc, steps: int, warmup: int = 1):
    import oracle

    s = oracle.System.from_scene(sc)
    s.step(warmup)
    t0 = time.perf_counter()
    s.step(steps)
    return time.perf_counter() - t0


def profiled_traffic(workload: str, storage: str, variant):
    """DRAM bytes per stream-collide launch from the committed ncu summary of
    this workload, or None when there is none, it is for another variant, or
    the kernel sources changed since the counters were taken."""
    import hashlib
    import re

    path = os.path.join(ROOT, "profiles", f"k_stream_collide_{workload}_{storage}.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(r"^dram_bytes_per_launch: (\d+)$", text, re.M)
    h = re.search(r"^kernel_source_sha256: (.*)$", text, re.M)
    # the captured variant: explicit "variant: npt bs" line, else the name of a
    # one-kernel-per-variant template k_stream_collide<S, NPT, BS>
    v = re.search(r"^variant: (-?\d+) (\d+)$", text, re.M) or re.search(r"k_stream_collide<\w+, (-?\d+), (\d+)>", text)
    if not (m and h and v) or (int(v.group(1)), int(v.group(2))) != (variant["npt"], variant["bs"]):
        return None
    pf = re.search(r"^l2_prefetch_nodes: (\d+)$", text, re.M)
    if pf and int(pf.group(1)) != variant.get("pf", 0):
        return None
    parts = h.group(1).split()
    for name, digest in zip(parts[0::2], parts[1::2]):
        src = os.path.join(ROOT, "paper_1110_0995_gb300", "csrc", name)
        if not os.path.exists(src) or hashlib.sha256(open(src, "rb").read()).hexdigest() != digest:
            return None
    return int(m.group(1))


def cpu_threads() -> int:
    v = os.environ.get("OMP_NUM_THREADS")
    return int(v) if v else (os.cpu_count() or 1)


def cpu_baseline_line(target_seconds: float = 15.0):
    """The oracle as it stands, on this host's cores, on a bounded sample of the workload."""
    sc, n = oracle_sample_scene(256 * 128 * 64)
    t1 = time_oracle(sc, 1, warmup=1)
    steps = max(1, min(200, int(target_seconds / max(t1, 1e-3))))
    dt = time_oracle(sc, steps, warmup=0)
    return {"value": n * steps / dt / 1e6, "unit": "MLUPS", "cores": cpu_threads(), "kind": "oracle",
            "sample": f"{steps} steps of the full {sc.dims[0]}x{sc.dims[1]}x{sc.dims[2]} filter "
                      f"({len(sc.meshes)} cells), FP64 oracle, {cpu_threads()} OpenMP threads"}


def cpu_baseline_single_thread(target_seconds: float = 10.0):
    """The same oracle timing with one OpenMP thread, in a fresh interpreter
    (the thread count of an OpenMP runtime is fixed at its first use)."""
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-baseline-only",
                            "--cpu-seconds", str(target_seconds)], env=env, capture_output=True, text=True,
                           timeout=300)
        return json.loads(r.stdout.strip().splitlines()[-1])
    except (subprocess.SubprocessError, ValueError, IndexError) as e:
        return {"unavailable": f"single-thread oracle run failed: {type(e).__name__}"}


def adjoint_ratio(steps: int = 400, ckpt_every: int = 50):
    """Cost of the discrete adjoint on the 128x64x64 channel with 12 Brinkman
    beads and 9 cells: forward cycles alone vs lb_adjoint (forward with
    checkpoints + recompute + reverse sweep), CUDA events on the stream."""
    import dataclasses

    import torch

    from paper_1110_0995_gb300 import lbibm, scene

    sc = scene.adjoint_channel()
    bare = dataclasses.replace(sc, spheres=np.zeros((0, 4), np.float32))
    stream = torch.cuda.Stream()
    sim = lbibm.Simulation.from_scene(bare, stream=stream.cuda_stream)
    sim.set_brinkman(np.asarray(sc.spheres, np.float64))
    sim.step(5)
    sim.adjoint(steps, ckpt_every)                 # workspace and graphs outside the timed calls

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), out

    t_fwd, _ = timed(lambda: sim.step(steps))
    t_adj, res = timed(lambda: sim.adjoint(steps, ckpt_every))
    sim.close()
    return {"workload": "adjoint_channel_128x64x64 (12 Brinkman beads, 1 tumor + 8 red cells)", "steps": steps,
            "ckpt_every": ckpt_every, "forward_us_per_step": 1e3 * t_fwd / steps,
            "adjoint_us_per_step": 1e3 * (t_adj - t_fwd) / steps, "adjoint_over_forward": (t_adj - t_fwd) / t_fwd,
            "J": res["J"], "note": "adjoint step = recompute share + reverse sweep; gradients checked against the "
                                   "FP64 oracle's dual numbers in tests/test_gpu_adjoint.py"}


def time_cycles(sim, stream, steps: int, warmup: int = 5):
    """Mean CUDA-graph cycle time (ms) over `steps` cycles after `warmup`, and
    the mean stream-collide launch time (ms) over a second, event-timed pass."""
    import torch

    sim.step(warmup)
    sim.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        sim.step(steps)
        e1.record(stream)
    torch.cuda.synchronize()
    cyc = e0.elapsed_time(e1) / steps
    sim.set_timing(4)
    sim.kernel_times()
    sim.step(steps)
    sim.synchronize()
    kms, kn = sim.kernel_times()
    sim.set_timing(0)
    return cyc, kms[2] / max(1, kn[2])


def extra_workloads(stream, device_name: str, steps: int = 30):
    """Short fixed windows of the other single-GPU workloads: the 512x256x128
    filter (the largest, 16.8 M nodes, 404 cells) with FP32, FP16 and BF16
    population storage, and the batched 24-channel gap sweep (FP32).  MLUPS
    over all nodes from graph replays; the stream-collide's fraction of the
    measured HBM copy bandwidth at its algorithmic bytes per fluid node."""
    from paper_1110_0995_gb300 import autotune, lbibm

    peak, _ = measured_peak()
    out = {}
    big = make_workload("micropost_filter_512x256x128")
    n_nodes = big[0].n_nodes
    res = {}
    n_fluid = None
    for st in ("f32", "f16", "bf16"):
        sim = lbibm.Simulation.from_scenes(big, storage=st, stream=stream.cuda_stream)
        tuned = autotune.tune(sim, device_name, st)
        if n_fluid is None:
            n_fluid = int((sim.solid_mask() == 0).sum())
        cyc, k3 = time_cycles(sim, stream, steps)
        fin = bool(sim.diagnostics()[4] == 0)
        sim.close()
        ach = BYTES_PER_NODE[st] * n_fluid / (k3 * 1e-3) / 1e9
        res[st] = {"mlups": n_nodes / (cyc * 1e-3) / 1e6, "ms_per_step": cyc, "stream_collide_ms": k3,
                   "stream_collide_frac": ach / peak, "cycle_frac": n_nodes / (cyc * 1e-3) * BYTES_PER_NODE[st] / (peak * 1e9),
                   "variant": [tuned["npt"], tuned["bs"], tuned.get("pf", 0)], "finite": fin}
    res["f16_over_f32_cycle"] = res["f16"]["mlups"] / res["f32"]["mlups"]
    res["bf16_over_f32_cycle"] = res["bf16"]["mlups"] / res["f32"]["mlups"]
    res["f16_over_f32_stream_collide"] = res["f32"]["stream_collide_ms"] / res["f16"]["stream_collide_ms"]
    out["micropost_filter_512x256x128"] = dict(res, fluid_nodes=n_fluid, steps=steps)
    sweep = make_workload("gap_sweep_24ch")
    sim = lbibm.Simulation.from_scenes(sweep, storage="f32", stream=stream.cuda_stream)
    tuned = autotune.tune(sim, device_name, "f32")
    nodes = sum(sc.n_nodes for sc in sweep)
    cyc, k3 = time_cycles(sim, stream, steps)
    sim.close()
    out["gap_sweep_24ch"] = {"mlups": nodes / (cyc * 1e-3) / 1e6, "ms_per_step": cyc, "stream_collide_ms": k3,
                             "nodes": nodes, "channels": len(sweep), "cells": sum(len(sc.meshes) for sc in sweep),
                             "variant": [tuned["npt"], tuned["bs"], tuned.get("pf", 0)], "steps": steps,
                             "storage": "f32"}
    return out


def max_over_ranks(values, device="cuda"):
    """The element-wise maximum of a list of floats over all ranks (the job's
    time is its slowest replica's)."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def job_mlups(world: int, nodes_per_replica: int, steps: int, ms: float) -> float:
    """Whole-job MLUPS of `world` replicas that each advance `nodes_per_replica`
    nodes `steps` times, timed at `ms` milliseconds (the slowest replica)."""
    return world * nodes_per_replica * steps / (ms * 1e-3) / 1e6


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return 0
    # calibrate: one oracle step of a small sample, then size the per-step sample
    cal, ncal = oracle_sample_scene(64 * 32 * 32)
    tcal = time_oracle(cal, 2, warmup=1) / 2
    rate = ncal / tcal                              # node updates per second
    budget = 150.0                                  # seconds for warm-up + timed steps
    per_step_nodes = int(rate * budget / max(1, args.steps + args.warmup))
    sc, n = oracle_sample_scene(per_step_nodes)
    import oracle

    s = oracle.System.from_scene(sc)
    s.step(args.warmup)
    t0 = time.perf_counter()
    s.step(args.steps)
    dt = time.perf_counter() - t0
    v = n * args.steps / dt / 1e6
    sample = (f"each step one oracle cycle of the {sc.dims[0]}x{sc.dims[1]}x{sc.dims[2]} filter sample "
              f"({len(sc.meshes)} cells)")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, "storage": "f64 oracle"},
            "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": cpu_threads(), "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch

    rank, local_rank, world = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local_rank)
    from paper_1110_0995_gb300 import _build, lbibm

    _build.build()
    scenes = make_workload(args.workload)
    stream = torch.cuda.Stream()
    sim = lbibm.Simulation.from_scenes(scenes, storage=args.storage, stream=stream.cuda_stream)
    from paper_1110_0995_gb300 import autotune

    if args.variant:
        vals = [int(v) for v in args.variant.split(",")]
        npt, bs, pf = vals[0], vals[1], (vals[2] if len(vals) > 2 else 0)
        sim.set_kernel_config(npt, bs)
        sim.set_prefetch(pf)
        tuned = {"npt": npt, "bs": bs, "pf": pf}
    else:
        tuned = autotune.tune(sim, torch.cuda.get_device_name(local_rank), args.storage)
    n_nodes = sum(s.n_nodes for s in scenes)
    n_fluid = 0
    for k in range(len(scenes)):
        sim.select(k)
        n_fluid += int((sim.solid_mask() == 0).sum())
    sim.select(0)
    n_cells = sum(len(s.meshes) for s in scenes)
    n_ib = sum(s.n_ib_nodes for s in scenes)
    sim.step(args.warmup)
    sim.synchronize()
    state = sim.save_state()                        # both timed passes start from this state

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()

    def timed_pass(kernel_mask):
        """K steps from the saved state; kernel_mask 0 = CUDA-graph replay (the
        product path), else per-launch CUDA events around the masked kernels."""
        sim.load_state(state)
        sim.set_timing(kernel_mask)
        sim.step(1)                                 # graph rebuild / first launch outside the region
        sim.load_state(state)
        sim.synchronize()
        sim.kernel_times()
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local_rank) as clk, torch.cuda.stream(stream):
            e0.record(stream)
            sim.step(args.steps)
            e1.record(stream)
            torch.cuda.synchronize()
        barrier()
        kms, kn = sim.kernel_times()
        diag = np.zeros(6)                          # FP64 sums over the final state, all channels
        for k in range(len(scenes)):
            sim.select(k)
            d = sim.diagnostics()
            diag[:5] += d[:5]
            diag[5] = max(diag[5], d[5])
        sim.select(0)
        return e0.elapsed_time(e1), kms, kn, diag, clk

    # pass 1: the number reported (graph replay, no instrumentation)
    ms, _, kn, diag, clk = timed_pass(0)
    finite = bool(diag[4] == 0)
    # pass 2: the same K steps again with CUDA events around every launch, for
    # the per-kernel durations (events add a few microseconds per launch)
    ms_ev, kms, _, diag_ev, clk_ev = timed_pass(15)
    if world > 1:
        ms, ms_ev = max_over_ranks([ms, ms_ev])
    value = job_mlups(world, n_nodes, args.steps, ms)

    # roofline of the dominant kernel (fused stream-collide)
    k3_ms = kms[2] / max(1, kn[2])             # kn: launches per class (same in both passes)
    peak, peak_kind = measured_peak()
    alg_bytes = BYTES_PER_NODE[args.storage] * n_fluid
    achieved = alg_bytes / (k3_ms * 1e-3) / 1e9
    traffic = profiled_traffic(args.workload, args.storage, tuned)

    # end to end through the C ABI with host buffers: scene upload from host,
    # steps, node positions of every cell read back every 10 steps, final fields
    e2e = None
    if not args.no_e2e:
        e2e_steps = args.steps
        # the caller's page-locked output buffers, allocated before the timed
        # region: two slots of node positions (the readback of one chunk runs
        # behind the next chunk's steps, the host waits for it one chunk
        # later) and the final fields of every channel
        bufs = [[torch.empty((sum(m.n_nodes for m in s.meshes), 3), dtype=torch.float64, pin_memory=True).numpy()
                 for s in scenes] for _ in range(2)]
        fbufs = [(torch.empty(int(np.prod(s.dims)), dtype=torch.float32, pin_memory=True).numpy(),
                  torch.empty(3 * int(np.prod(s.dims)), dtype=torch.float32, pin_memory=True).numpy()) for s in scenes]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s2 = lbibm.Simulation.from_scenes(scenes, storage=args.storage, stream=stream.cuda_stream)
        s2.set_kernel_config(tuned["npt"], tuned["bs"])
        s2.set_prefetch(tuned.get("pf", 0))
        s2.synchronize()
        t_setup = time.perf_counter() - t0
        h2d = sum(m.rest.nbytes + m.tris.nbytes for s in scenes for m in s.meshes) + sum(s.spheres.nbytes for s in scenes)
        d2h = 0
        done = 0
        chunk = 0
        while done < e2e_steps:
            k = min(10, e2e_steps - done)
            s2.step(k)
            done += k
            slot = chunk & 1
            if chunk >= 2:
                s2.wait_readback(slot)   # the host takes the positions of chunk - 2
            for c, b in enumerate(bufs[slot]):
                s2.select(c)
                s2.all_nodes_into_async(b, slot)
                d2h += b.nbytes
            chunk += 1
        for slot in range(2):
            s2.wait_readback(slot)
        for c in range(len(scenes)):
            s2.select(c)
            rho, u = fbufs[c]
            s2.fields_into(rho, u)
            d2h += rho.nbytes + u.nbytes
        s2.synchronize()
        dt = time.perf_counter() - t0
        s2.close()
        e2e = {"value": world * n_nodes * e2e_steps / dt / 1e6, "unit": "MLUPS",
               "h2d_bytes_per_step": h2d / e2e_steps, "d2h_bytes_per_step": d2h / e2e_steps,
               "setup_ms": 1e3 * t_setup,
               "steady_value": world * n_nodes * e2e_steps / (dt - t_setup) / 1e6,
               "includes": "context creation, scene upload, node positions read back every 10 steps "
                           "(asynchronous, two page-locked slots), final fields (into page-locked buffers; "
                           "the caller's output buffers are allocated before the timed region); steady_value "
                           "leaves out the setup (context creation and scene upload, setup_ms)"}

    if rank == 0:
        cpu = None if (args.no_cpu_baseline or world > 1 or len(scenes) > 1) else cpu_baseline_line()
        if cpu is not None:
            cpu["single_thread"] = cpu_baseline_single_thread()
        adj = None if (args.no_adjoint or world > 1) else adjoint_ratio()
        extra = None if (args.no_extra or world > 1) else extra_workloads(stream, torch.cuda.get_device_name(local_rank))
        line = {
            "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.storage, "data": "synthetic",
            "config": {"workload": args.workload,
                       "lattice": list(scenes[0].dims) if len(scenes) == 1 else [list(s.dims) for s in scenes],
                       "cells": n_cells, "ib_nodes": n_ib, "spheres": int(sum(len(s.spheres) for s in scenes)),
                       "fluid_nodes": n_fluid,
                       "storage": args.storage, "l2": "populations 2x%.0f MB > 126 MB L2" % (
                           19 * BYTES_PER_NODE[args.storage] / 38 * n_nodes / 1e6),
                       "parallelism": "replicas" if world > 1 else "single",
                       "stream_collide_variant": {"nodes_per_thread": tuned["npt"], "block": tuned["bs"],
                                                  "l2_prefetch_nodes": tuned.get("pf", 0)}},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                         "kernel": "k_stream_collide", "alg_bytes_per_launch": alg_bytes,
                         "avg_launch_ms": k3_ms},
            "cycle_frac": value * 1e6 * BYTES_PER_NODE[args.storage] / (peak * 1e9) / world,
            "cycle_frac_how": "value x algorithmic bytes per node / measured HBM copy bandwidth (per GPU)",
            "kernel_ms_per_step": {"elements": kms[0] / max(1, kn[0]), "forces_spread": kms[1] / max(1, kn[1]),
                                   "stream_collide": k3_ms, "interp_advance": kms[3] / max(1, kn[3])},
            "ib_node_updates_per_s": world * n_ib * args.steps / (ms * 1e-3),
            "mlups_fluid_nodes": value * n_fluid / n_nodes,
            "gpu_launches": int(sum(kn)),
            "kernel_timing": {"ms_per_step_with_events": ms_ev / args.steps, "clocks": clk_ev.summary(),
                              "how": "second pass over the same K steps from the same saved state, "
                                     "CUDA events on the simulation stream around every launch"},
            "state_after_timed_steps": {"finite": finite and bool(diag_ev[4] == 0),
                                        "mass_per_fluid_node": diag[0] / n_fluid, "max_u": diag[5]},
            "clocks": clk.summary(),
            "cpu_baseline": cpu,
            "adjoint": adj,
            "workloads": extra,
            "e2e": e2e,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="micropost_filter_256x128x64")
    ap.add_argument("--storage", default="f32", choices=["f32", "f16", "bf16"])
    ap.add_argument("--variant", default="",
                    help="stream-collide variant 'npt,bs[,l2_prefetch_nodes]' instead of the autotuner")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint / forward cost measurement")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the 512x256x128 storage comparison and the gap sweep")
    ap.add_argument("--cpu-baseline-only", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help=argparse.SUPPRESS)
    args = ap.parse_args(argv)
    if args.cpu_baseline_only:
        print(json.dumps(cpu_baseline_line(args.cpu_seconds)), flush=True)
        return 0
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
