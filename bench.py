"""Benchmark: coupled-lattice MLUPS of the double-MRT phase-change LBM on GB300.

One step = one full time step of the method on the 2048^2 heterogeneous
porous cavity (Ra = 1e6, mean Da = 1e-4, porosity recipe seed 3), started
part-way through melting (left 7/8 liquid): the fused D2Q9 + D2Q5 stream-
collide over every node, the phase-change screen, and the enthalpy solve +
latent source on the marked tiles.  MLUPS counts every node (walls included)
per step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Timing: W untimed steps, then K steps between CUDA events on the context
stream, bracketed by a barrier and a device synchronisation; max over ranks.
The state (14 population planes + 3 scalar planes, ~520 MB at 2048^2) is far
larger than the 129 MB L2, so no flush is needed between steps.

Multi-GPU: the path has no exchange step at one cavity per GPU, so N ranks run
N independent replicas (weak scaling, no collective on the data path).

--impl reference times the FP64 CPU oracle on the host cores instead (each
step one oracle time step of the same recipe on a 128^2 lattice).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "coupled-lattice MLUPS (D2Q9 flow + D2Q5 thermal + enthalpy update), 1 GB300"
UNIT = "MLUPS"
FALLBACK_HBM_GBS = 6800.0
# algorithmic bytes per node and step of the fused kernel (FP32):
# flow node: f 9 read + 9 write, g 5 + 5, f_l, phi, K reads = 31 x 4 B
# solid node: g 5 + 5, f_l read = 11 x 4 B; wall node: nothing
BYTES_FLOW_NODE = 124
BYTES_SOLID_NODE = 44
# with 16-bit population storage: f 18 x 2 B, g 10 x 2 B + f_l, phi, K; solid g 10 x 2 + f_l
BYTES_FLOW_NODE_16 = 68
BYTES_SOLID_NODE_16 = 24
KERNEL_SOURCES = ("paper_1503_08406_gb300/csrc/lbm_fused.cuh",
                  "paper_1503_08406_gb300/csrc/lbm_fused_f32.cu",
                  "paper_1503_08406_gb300/csrc/lbm_internal.cuh")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "fused_tma_traffic_heterogeneous_cavity_2048.json")


def kernel_hash() -> str:
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, p), "rb").read())
    return h.hexdigest()[:16]


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--warmup", type=int, default=500)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--n", type=int, default=2048, help="lattice edge (default 2048)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--storage", choices=("fp32", "fp16", "bf16"), default="fp32",
                    help="population storage (arithmetic is FP32 in every case)")
    ap.add_argument("--workload", choices=("cavity", "batched", "adjoint", "adjoint_coupled",
                                           "convection"),
                    default="cavity",
                    help="cavity: the 2048^2 heterogeneous cavity (default); batched: 64 "
                         "uneven cavities advanced together through one CUDA graph; adjoint: "
                         "melted fraction and its gradients on an n x ny conduction slab, "
                         "timed against the forward run alone; adjoint_coupled: the same "
                         "with the flow lattice on, the n^2 inverse-problem cavity; "
                         "convection: the uniform n^2 convection-melting cavity, its "
                         "melted fraction, Nusselt number and f_l = 0.5 contour")
    ap.add_argument("--ny", type=int, default=512, help="adjoint workload: slab height")
    ap.add_argument("--objective", choices=("melt", "nusselt"), default="melt",
                    help="adjoint workload: melted fraction at the end, or the left-wall "
                         "Nusselt number averaged over the steps")
    ap.add_argument("--trace", type=int, default=0,
                    help="cavity workload: after the measurements, step this many more steps "
                         "with the kernel trace on and print each launch's start, end and CTA "
                         "count (a timeline of the overlapped graph replay)")
    ap.add_argument("--checkpoint", type=int, default=0,
                    help="adjoint workloads: keep the whole state every K steps (0: every "
                         "state when it fits in half the free memory, else sqrt(steps))")
    ap.add_argument("--autotune", action="store_true",
                    help="batched workload: tune each cavity's stream-collide kernel first")
    return ap.parse_args(argv)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def init_dist(world: int, backend: str):
    if world <= 1:
        return None
    import torch.distributed as dist
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    os.environ.setdefault("MASTER_PORT", "29511")
    dist.init_process_group(backend)
    return dist


def aggregate(ms_local: float, cells: int, steps: int, world: int, dist=None, device=None):
    """Whole-job throughput of independent replicas: every rank did cells*steps
    updates; the job time is the slowest rank's."""
    ms = ms_local
    if dist is not None:
        import torch
        t = torch.tensor([ms_local], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = world * cells * steps / (ms / 1e3) / 1e6
    return value, ms


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            for k in ("hbm_gbs", "hbm_GBs", "hbm"):
                if k in d:
                    v = d[k]
                    if isinstance(v, dict):
                        v = v.get("value", v.get("burst"))
                    return float(v), "measured"
        except (ValueError, TypeError):
            pass
    return FALLBACK_HBM_GBS, "fallback"


def traffic_per_launch(n: int):
    """DRAM bytes per fused launch from the committed ncu summary, scaled to
    this lattice by node count; None if the kernel changed since the capture."""
    if not os.path.exists(TRAFFIC_FILE):
        return None
    try:
        d = json.load(open(TRAFFIC_FILE))
    except ValueError:
        return None
    if d.get("kernel_hash") != kernel_hash():
        return None
    return d["dram_bytes_per_launch"] * (n * n) / float(d["nodes"])


def cpu_baseline(n_bench: int):
    """The FP64 oracle, as it stands, on the host cores: a bounded sample of the
    benchmark workload (a few steps of the same 2048^2 state)."""
    import oracle
    import lbm_workloads as W
    oracle.build()
    w = W.bench_cavity(n_bench)
    o = oracle.Oracle(w.nx, w.ny, **w.params)
    o.set_fields(w.phi, w.K, w.T0, w.fl0)
    o.step(1)
    steps = 4
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    cores = os.cpu_count()
    return {"value": w.cells * steps / dt / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{steps} oracle steps of the {w.nx}x{w.ny} benchmark state "
                      f"(FP64, OpenMP over rows, {cores} threads), after 1 untimed step"}


def reference_arm(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    import lbm_workloads as W
    oracle.build()
    n = 128
    w = W.bench_cavity(n)
    o = oracle.Oracle(w.nx, w.ny, **w.params)
    o.set_fields(w.phi, w.K, w.T0, w.fl0)
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    value = w.cells * args.steps / dt / 1e6
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / max(args.steps, 1) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": W.bench_cavity(args.n).name, "lattice": [args.n, args.n],
                   "reference_sample": f"same recipe on a {n}x{n} lattice, one oracle step per step"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} timed oracle steps on the {n}x{n} sample "
                                   f"after {args.warmup} untimed"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def batched(args, torch):
    """64 uneven cavities (sides 64..512, Ra 1e4..1e7, seed 4): the same steps
    run one cavity after another (each through its own CUDA graphs) and all
    together through one batch graph; one JSON line, value = the batched
    whole-job MLUPS."""
    import lbm_workloads as W
    from paper_1503_08406_gb300 import Batch, Lattice
    ws = W.batched_cavities(64, seed=4)
    cells = sum(w.cells for w in ws)
    stream = torch.cuda.current_stream()
    lats = []
    for w in ws:
        lat = Lattice(w.nx, w.ny, stream=stream, **{**w.params, "storage": args.storage})
        lat.set_fields(w.phi, w.K, w.T0, w.fl0)
        lats.append(lat)
    tuned = []
    if args.autotune:
        for lat in lats:
            tuned.append(lat.autotune(16))
        for lat in lats:   # same step count everywhere again
            lat.step(max(x.steps_done() for x in lats) - lat.steps_done())
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # one after another: every cavity's steps on the same stream
    for lat in lats:
        lat.step(args.warmup)
    torch.cuda.synchronize()
    e0.record(stream)
    for lat in lats:
        lat.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_seq = e0.elapsed_time(e1)
    b = Batch(lats)
    mode = b.mode()
    b.step(args.warmup)
    torch.cuda.synchronize()
    launches0 = sum(lat.kernel_launches() for lat in lats)
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    with ClockSampler(vis.split(",")[0] if vis else "0") as clk:
        torch.cuda.synchronize()
        e0.record(b.stream)
        b.step(args.steps)
        e1.record(b.stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    launches = sum(lat.kernel_launches() for lat in lats) - launches0
    status = max((lat.status() for lat in lats), key=abs)
    # algorithmic bytes of the stream-collide passes of all cavities per step
    bf, bs = ((BYTES_FLOW_NODE, BYTES_SOLID_NODE) if args.storage == "fp32"
              else (BYTES_FLOW_NODE_16, BYTES_SOLID_NODE_16))
    nbytes = 0
    for lat in lats:
        fl = lat.macros()["fl"][1:-1, 1:-1]
        nf = int((fl >= 1e-3).sum())
        nbytes += bf * nf + bs * (fl.size - nf)
    peak, peak_kind = measured_peak()
    achieved = nbytes / (ms / args.steps * 1e-3) / 1e9
    value = cells * args.steps / (ms * 1e-3) / 1e6
    line = {
        "metric": METRIC + ", 64 batched cavities", "value": value, "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "batched_cavities_64_seed4", "cells": cells,
                   "sides": sorted({w.nx for w in ws}), "population_storage": args.storage,
                   "graph": "one CUDA graph per 32 steps, " + (
                       "each pass of a step one launch over all cavities" if mode == 1
                       else "one branch per cavity"),
                   "autotuned": tuned if args.autotune else None,
                   "l2": "state ~%d MB > 129 MB L2; no flush" % (
                       (14 * (4 if args.storage == "fp32" else 2) + 12) * cells // 2**20)},
        "sequential": {"value": cells * args.steps / (ms_seq * 1e-3) / 1e6, "unit": UNIT,
                       "ms_per_step": ms_seq / args.steps,
                       "note": "the same steps, one cavity after another on one stream"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None, "peak_kind": peak_kind,
                     "kernel": "whole batched step (stream-collide bytes / step time)",
                     "algorithmic_bytes_per_step": nbytes},
        "gpu_launches": launches, "status": status, "clocks": clk.summary(),
        "e2e": None, "cpu_baseline": None,
    }
    print(json.dumps(line), flush=True)
    b.close()
    return 0


def adjoint(args, torch):
    """The conduction slab (lbm_workloads.adjoint_slab, n x ny): `steps` steps
    forward alone, then the same steps with the adjoint (lbm_adjoint:
    forward, reverse sweep, gradients back on the host), both from the same
    state; one JSON line, value = adjoint time / forward time."""
    import lbm_workloads as W
    from paper_1503_08406_gb300 import Lattice
    w = W.adjoint_slab(args.n, args.ny)
    stream = torch.cuda.current_stream()
    lat = Lattice(w.nx, w.ny, stream=stream, **w.params)

    def reset():
        lat.set_fields(w.phi, w.K, w.T0, w.fl0, w.wall_T_left)
        torch.cuda.synchronize()

    reset()
    lat.step(args.warmup)                       # graphs captured, clocks up
    reset()
    lat.adjoint(max(args.warmup, 2), args.objective)   # allocations and kernels warmed
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reset()
    e0.record(stream)
    lat.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_fwd = e0.elapsed_time(e1)
    reset()
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    with ClockSampler(vis.split(",")[0] if vis else "0") as clk:
        t0 = time.perf_counter()
        J, dphi, dtw = lat.adjoint(args.steps, args.objective)
        ms_adj = (time.perf_counter() - t0) * 1e3
    line = {
        "metric": "adjoint time / forward time, %s and its gradients" % (
            "melted fraction" if args.objective == "melt" else "time-averaged hot-wall Nusselt"),
        "value": ms_adj / ms_fwd, "unit": "x", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_adj / args.steps, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w.name, "lattice": [w.nx, w.ny],
                   "memory": "f_l of every step kept (%.2f GB)" % (
                       (args.steps + 1) * w.cells * 4 / 1e9)},
        "forward": {"ms": ms_fwd, "MLUPS": w.cells * args.steps / (ms_fwd * 1e-3) / 1e6,
                    "timing": "CUDA events on the lattice's stream"},
        "adjoint": {"ms": ms_adj, "timing": "host wall clock around lbm_adjoint_melt "
                    "(forward run, reverse sweep, gradients copied to the host)",
                    "J": J, "dJ_dTw_max": float(abs(dtw).max()),
                    "dJ_dphi_max": float(abs(dphi).max())},
        "status": lat.status(), "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    return 0


def adjoint_coupled(args, torch):
    """The inverse-problem cavity (lbm_workloads.adjoint_cavity, n^2, Ra = 1e6,
    smooth ln K field, heterogeneous porosity, mushy band [0, 0.05]): `steps`
    steps forward alone, then the same steps with the coupled adjoint
    (lbm_adjoint_coupled: forward run, reverse sweep with every state kept or
    sqrt(N) checkpoints and recomputation, gradients back on the host);
    value = adjoint time / forward time."""
    import numpy as np
    import lbm_workloads as W
    from paper_1503_08406_gb300 import Lattice
    w = W.adjoint_cavity(args.n)
    stream = torch.cuda.current_stream()
    lat = Lattice(w.nx, w.ny, stream=stream, **w.params)

    def reset():
        lat.set_fields(w.phi, w.K, w.T0, w.fl0, w.wall_T_left)
        torch.cuda.synchronize()

    reset()
    lat.step(args.warmup)
    reset()
    lat.adjoint_coupled(max(args.warmup, 2), args.objective, args.checkpoint)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reset()
    lat.prepare(args.steps)
    e0.record(stream)
    lat.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_fwd = e0.elapsed_time(e1)
    melt = lat.reduce()["melt_frac"]
    reset()
    n = w.cells
    st_bytes = 60 * n
    free, _ = torch.cuda.mem_get_info()
    keep_all = args.checkpoint == 0 and (args.steps + 1) * st_bytes <= 0.5 * free
    K = args.steps if keep_all else (args.checkpoint or int(np.ceil(np.sqrt(args.steps))))
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    with ClockSampler(vis.split(",")[0] if vis else "0") as clk:
        t0 = time.perf_counter()
        J, dphi, dlnK, dtw = lat.adjoint_coupled(args.steps, args.objective, args.checkpoint)
        ms_adj = (time.perf_counter() - t0) * 1e3
    ph_fwd, ph_rev = lat.adjoint_timing()
    if keep_all:
        memory = "every state kept (%.2f GB)" % ((args.steps + 1) * st_bytes / 1e9)
    else:
        memory = ("whole state every %d steps (%d checkpoints, %.2f GB) plus two segments' "
                  "states (%.2f GB: one recomputed beside the reversal of the other)" % (
                      K, args.steps // K + 1, (args.steps // K + 1) * st_bytes / 1e9,
                      2 * (K + 1) * st_bytes / 1e9))
    line = {
        "metric": "coupled adjoint time / forward time, %s and its gradients" % args.objective,
        "value": ms_adj / ms_fwd, "unit": "x", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_adj / args.steps, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w.name, "lattice": [w.nx, w.ny], "memory": memory,
                   "melted_fraction_after": melt},
        "forward": {"ms": ms_fwd, "MLUPS": n * args.steps / (ms_fwd * 1e-3) / 1e6,
                    "timing": "CUDA events on the lattice's stream (CUDA graphs)"},
        "adjoint": {"ms": ms_adj, "timing": "host wall clock around lbm_adjoint_coupled",
                    "device_ms_forward_run": ph_fwd, "device_ms_reverse_sweep": ph_rev,
                    "reverse_over_forward": ph_rev / ms_fwd,
                    "J": J, "dJ_dlnK_max": float(abs(dlnK).max()),
                    "dJ_dphi_max": float(abs(dphi).max()),
                    "dJ_dTw_max": float(abs(dtw).max())},
        "status": lat.status(), "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    return 0


def convection(args, torch):
    """Convection melting in the uniform porous cavity (lbm_workloads.convection_cavity,
    n^2, phi = 0.4, Da = 1e-4, Ra = 1e5): `steps` steps from the solid start;
    the line reports MLUPS and the outputs the workload asks for: melted
    fraction, hot-wall Nusselt number (every `steps / 50` steps and their
    mean) and the f_l = 0.5 contour (its x position, interpolated, on every
    16th row)."""
    import numpy as np
    import lbm_workloads as W
    from paper_1503_08406_gb300 import Lattice
    w = W.convection_cavity(args.n)
    stream = torch.cuda.current_stream()
    lat = Lattice(w.nx, w.ny, stream=stream, **w.params)
    lat.set_fields(w.phi, w.K, w.T0, w.fl0)
    every = max(args.steps // 50, 1)
    lat.prepare(every)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    nus, done, ms = [], 0, 0.0
    while done < args.steps:
        k = min(every, args.steps - done)
        e0.record(stream)
        lat.step(k)
        e1.record(stream)
        torch.cuda.synchronize()
        ms += e0.elapsed_time(e1)
        done += k
        nus.append(lat.reduce()["nu_hot"])
    r = lat.reduce()
    fl = lat.macros()["fl"]
    contour = []
    for y in range(1, w.ny - 1, 16):
        row = fl[y]
        xs = np.flatnonzero((row[:-1] >= 0.5) & (row[1:] < 0.5))
        if xs.size:
            x0 = int(xs[-1])
            t = (row[x0] - 0.5) / (row[x0] - row[x0 + 1])
            contour.append([y, round(float(x0 + t), 3)])
    line = {
        "metric": "convection melting in the porous cavity: outputs after %d steps" % args.steps,
        "value": w.cells * args.steps / (ms * 1e-3) / 1e6, "unit": "MLUPS", "n_gpus": 1,
        "steps": args.steps, "warmup": 0, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": {"workload": w.name, "lattice": [w.nx, w.ny]},
        "melted_fraction": r["melt_frac"], "nu_hot": r["nu_hot"],
        "nu_hot_mean_over_run": float(np.mean(nus)), "nu_hot_samples_every": every,
        "front_fl05_x_by_row": contour, "status": lat.status(),
    }
    print(json.dumps(line), flush=True)
    return 0


def main(argv=None):
    args = parse(argv)
    if args.impl == "reference":
        return reference_arm(args)
    rank, world, local = dist_env()
    import torch
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (there is no CPU path)")
    torch.cuda.set_device(local)
    if args.workload in ("batched", "adjoint", "adjoint_coupled", "convection"):
        if world > 1:
            raise SystemExit("the %s workload runs on one GPU" % args.workload)
        import __graft_entry__
        __graft_entry__.build()
        run = {"batched": batched, "adjoint": adjoint, "adjoint_coupled": adjoint_coupled,
               "convection": convection}
        return run[args.workload](args, torch)
    dist = init_dist(world, "nccl")
    device = torch.device("cuda", local)
    if local == 0:
        import __graft_entry__
        __graft_entry__.build()
    if dist is not None:
        dist.barrier()
    import lbm_workloads as W
    from paper_1503_08406_gb300 import Lattice

    w = W.bench_cavity(args.n)
    cells = w.cells
    lat = Lattice(w.nx, w.ny, **{**w.params, "storage": args.storage})
    lat.set_fields(w.phi, w.K, w.T0, w.fl0)
    stream = lat.stream
    lat.step(args.warmup)
    torch.cuda.synchronize()
    m0 = lat.macros()
    interior = slice(1, -1)
    fl_in = m0["fl"][interior, interior]
    n_flow = int((fl_in >= 1e-3).sum())
    n_solid = int(fl_in.size - n_flow)
    if args.storage == "fp32":
        bytes_step = BYTES_FLOW_NODE * n_flow + BYTES_SOLID_NODE * n_solid
    else:
        bytes_step = BYTES_FLOW_NODE_16 * n_flow + BYTES_SOLID_NODE_16 * n_solid

    # ---- headline: K steps, CUDA events on the context stream --------------
    # the CUDA graphs lbm_step will replay are captured before the timed region
    lat.prepare(args.steps)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    smi_index = vis.split(",")[local] if vis and len(vis.split(",")) > local else str(local)
    with ClockSampler(smi_index) as clk:
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        launches0 = lat.kernel_launches()
        e0.record(stream)
        lat.step(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
    ms_local = e0.elapsed_time(e1)
    launches = lat.kernel_launches() - launches0
    value, ms = aggregate(ms_local, cells, args.steps, world, dist, device)
    rc = lat.status()

    # ---- roofline of the fused kernel: per-kernel events, same stream ------
    k_roof = args.steps
    lat.timing(True)
    lat.step(k_roof)
    tr = lat.timing_read()
    lat.timing(False)
    nt = max(tr["steps"], 1)
    fused_us = tr["fused_ms"] / nt * 1e3
    solve_us = tr["solve_ms"] / nt * 1e3
    commit_us = tr["commit_ms"] / nt * 1e3
    peak, peak_kind = measured_peak()
    achieved = bytes_step / (fused_us * 1e-6) / 1e9
    # the committed record covers the TMA-staged kernel only
    traffic = (traffic_per_launch(args.n)
               if lat.kernel_variant() == 2 and args.storage == "fp32" else None)

    # ---- end to end through the C ABI with pinned host buffers --------------
    e2e = None
    if not args.no_e2e:
        import numpy as np
        host_in = [torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).pin_memory()
                   for a in (w.phi, w.K, w.T0, w.fl0)]
        host_out = [torch.empty((w.ny, w.nx), dtype=torch.float32).pin_memory() for _ in range(5)]
        lat2 = Lattice(w.nx, w.ny, **{**w.params, "storage": args.storage})

        def e2e_run():
            rc_in = lat2.lib.lbm_set_fields(lat2._h, *[t.data_ptr() for t in host_in], None, 0)
            lat2.step(args.steps)
            rc_out = lat2.lib.lbm_get_macros(lat2._h, *[t.data_ptr() for t in host_out], 0)
            assert rc_in == 0 and rc_out == 0, (rc_in, rc_out)

        e2e_run()            # untimed: the context's graphs are captured, copies warmed
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_run()
        dt = time.perf_counter() - t0
        h2d = sum(t.numel() * 4 for t in host_in)
        d2h = sum(t.numel() * 4 for t in host_out)
        e2e_val, _ = aggregate(dt * 1e3, cells, args.steps, world, dist, device)
        e2e = {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d / args.steps,
               "d2h_bytes_per_step": d2h / args.steps,
               "note": "set_fields from pinned host + K steps + get_macros to pinned host, "
                       "host wall clock, second run on the same context (graphs captured)"}
        lat2.close()

    base = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        base = cpu_baseline(args.n)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "lattice": [w.nx, w.ny], "Ra": 1e6, "Da_mean": 1e-4,
                       "porosity": "clip(0.45+0.15 g, 0.3, 0.6), g smoothed (16 cells), seed 3",
                       "flow_nodes": n_flow, "solid_nodes": n_solid,
                       "population_storage": args.storage,
                       "parallelism": f"replicas x{world}",
                       # state per node: 14 populations + f_l, phi, K (FP32)
                       "l2": "state ~%d MB > 129 MB L2; no flush" % (
                           (14 * (4 if args.storage == "fp32" else 2) + 12) * cells // 2**20)},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                         "kernel": ("fused_tma_kernel" if lat.kernel_variant() == 2
                                    else "fused_step_kernel") + "<%s>" % args.storage,
                         "algorithmic_bytes_per_launch": bytes_step,
                         "fused_us_per_launch": fused_us,
                         "solve_us_per_step": solve_us,
                         "commit_us_per_step": commit_us,
                         "tiles_solved_per_step": tr["tiles_solved"] / nt,
                         "max_inner_sweeps": tr["max_sweeps"]},
            "gpu_launches": launches,
            "status": rc,
        }
        clocks = clk.summary()
        line["clocks"] = clocks
        line["e2e"] = e2e
        line["cpu_baseline"] = base
        print(json.dumps(line), flush=True)
    if args.trace > 0 and rank == 0:
        from paper_1503_08406_gb300.lbm import trace_launches
        lat.trace(1 << 22)
        lat.prepare(args.trace)
        lat.step(args.trace)
        recs = lat.trace_read()
        lat.trace(0)
        print("# kernel trace: %d steps, %d CTA records (times in us)" % (args.trace, len(recs)))
        for r in trace_launches(recs):
            print("%9.1f %9.1f %8.1f  ctas %5d  median CTA %6.1f  step %d  parity %d  %s" % (
                r["start_us"], r["end_us"], r["end_us"] - r["start_us"], r["ctas"],
                r["median_cta_us"], r["step"], r["parity"], r["what"]))
    lat.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
