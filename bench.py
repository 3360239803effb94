"""Benchmark of the fused phase-field LB step on GB300.

Workload: FP32 sessile droplet on a curved wall -- a 128^3 periodic box with a
voxelised solid sphere of radius 30 centred on the bottom plane, solid planes
at z = 0 and z = 127, a droplet of radius 20 (tanh profile, W = 4) tangent to
the sphere's top, input contact angle 60 deg, density ratio 1000,
sigma = 0.005, tau = 0.8, M = 0.02, optimised model (tanh F, free-slip band,
blend 0.95).  Synthetic geometry.

One bench step = one time step of the whole path in one fused kernel launch:
phi recompute, wall ghosts, stencils, macros, h and g collisions and
streaming, and the diagnostics reduction (mass, pressure jump, contact-line
band, max |u|).  The state (3 x 19 FP32 population arrays, ~480 MB) is
larger than L2, so no L2 flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank advances its own replica (independent lattices,
no data-path exchange: weak scaling).  --impl reference times the FP64 CPU
oracle on this workload on the host cores.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
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

METRIC = "fused AC+NS LB step MLUPS"
# Algorithmic bytes per fluid-cell update at FP32 storage: 2 population sets
# x 19 x (read + write) x 4 B, plus the 1-byte cell flag.
ALGO_BYTES_FP32 = 2 * 19 * 2 * 4 + 1
THETA = 60.0
N_BOX = 128
CLOCK_WINDOW_S = 1.0  # untimed load before the timed region, for the clock record
KERNEL_SOURCES = ("pflb_kernels.cuh", "pflb_model.cuh", "pflb_launch.cuh", "pflb_pipe.cuh",
                  "pflb_f32.cu")
KERNEL_NAMES = {0: "k_fused", 1: "k_phi + k_cell", 2: "k_fused_async", 3: "k_pipe"}
KERNEL_TEXT = {0: "fused z-marching, direct loads", 1: "phi pass + per-cell pass",
               2: "fused z-marching, h staged by TMA",
               3: "fused z-marching, populations staged one plane ahead by cp.async, "
                  "each block's wall nodes after its march"}
ORACLE_KEYS = ("sigma", "W", "M", "rho_H", "rho_L", "nu_H", "nu_L", "theta_deg", "Fex", "blend",
               "F_mode", "mobility_corr", "free_slip")


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_2512_01032_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


BATCH_SOURCES = ("pflb_batch.cuh", "pflb_kernels.cuh", "pflb_model.cuh", "pflb_launch.cuh",
                 "pflb_bf16.cu")


def batch_source_hash() -> str:
    h = hashlib.sha256()
    for f in BATCH_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_2512_01032_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def recorded_batch_traffic(storage, fluid):
    """DRAM bytes per launch of the batch kernel, from the committed ncu
    summary of a smaller case scaled by fluid cells, if it was taken on the
    current sources at this storage."""
    try:
        d = json.load(open(os.path.join(ROOT, "profiles", "k_batch_channels8_bf16_traffic.json")))
    except Exception:
        return None
    if d.get("batch_source_hash") != batch_source_hash() or d.get("storage") != storage:
        return None
    return d["dram_bytes_per_fluid_cell"] * fluid


def hbm_peak():
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def recorded_traffic(kernel="k_pipe"):
    """DRAM bytes per launch of the step kernel from the committed ncu
    summary, if it was taken on the current kernel sources."""
    try:
        d = json.load(open(os.path.join(ROOT, "profiles", f"{kernel}_sessile128_traffic.json")))
    except Exception:
        return None
    if d.get("kernel_source_hash") != kernel_source_hash():
        return None
    return d.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clock and throttle-reason sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.out = None
        self.path = os.path.join(os.environ.get("PFLB_CLOCKS_DIR", tempfile.gettempdir()),
                                 f"pflb_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}", "--format=csv",
                 "-lms", "100"], stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            if self.out is not None:
                self.out.close()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.close()
        sm, smax, reasons = [], [], set()
        try:
            for ln in open(self.path).read().strip().splitlines()[1:]:
                f = [x.strip() for x in ln.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1].split()[0]))
                    smax.append(float(f[2].split()[0]))
                except ValueError:
                    continue
                for k, nm in enumerate(self.NAMES):
                    if f[5 + k].lower().startswith("active"):
                        reasons.add(nm)
        except Exception:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def workload(n=N_BOX):
    return synth.sessile_sphere(n, THETA)


def config_of(g, fluid, kind=3):
    return {"workload": f"FP32 sessile droplet on a curved wall, {g.nx}x{g.ny}x{g.nz} D3Q19, "
                        f"solid sphere R=30, drop R=20, theta={THETA:g} deg, density ratio 1000",
            "lattice": [g.nx, g.ny, g.nz], "fluid_cells": int(fluid), "storage": "fp32",
            "kernel": KERNEL_TEXT.get(kind, str(kind)) + " (one launch per step, diagnostics on)",
            "l2": "inputs larger than L2 (no flush)"}


def oracle_lattice(g, p, drop, nthreads):
    import oracle as O
    op = {k: v for k, v in p.items() if k in ORACLE_KEYS}
    L = O.OracleLattice(g.nx, g.ny, g.nz, solid=g.solid, wall_normal=g.normals(),
                        theta_cells=g.theta(), nthreads=nthreads, **op)
    phi0 = O.tanh_phi(0, (g.nx, g.ny, g.nz), drop["center"], drop["R"], p["W"]) * (1 - g.solid)
    L.init_phi(phi0)
    return L


def slab(g, z0, nz_s):
    """The z-planes [z0, z0 + nz_s) of a geometry as a periodic lattice."""
    s = synth.Geometry(g.nx, g.ny, nz_s)
    s.solid3 = g.solid3[z0:z0 + nz_s].copy()
    s.theta3 = g.theta3[z0:z0 + nz_s].copy()
    nrm = g.normals().reshape(g.nz, g.ny, g.nx, 3)[z0:z0 + nz_s].copy()
    s.normals = lambda: nrm.reshape(-1)
    return s


def cpu_baseline(g, p, drop, budget_s=15.0):
    """The oracle as it stands, all host cores, on the same lattice for a
    bounded number of steps (about budget_s of CPU time)."""
    nthreads = os.cpu_count() or 1
    L = oracle_lattice(g, p, drop, nthreads)
    t0 = time.perf_counter()
    L.step(1)
    per = max(time.perf_counter() - t0, 1e-6)
    k = max(1, min(200, int(budget_s / per)))
    t0 = time.perf_counter()
    L.step(k)
    dt = time.perf_counter() - t0
    fluid = int(g.N - g.solid.sum())
    # one thread, on the same lattice, about a third of the budget
    L.set_nthreads(1)
    t0 = time.perf_counter()
    L.step(1)
    k1 = 1
    while time.perf_counter() - t0 < budget_s / 3.0 and k1 < 50:
        L.step(1)
        k1 += 1
    dt1 = time.perf_counter() - t0
    return {"value": fluid * k / dt / 1e6, "unit": "MLUPS", "cores": nthreads, "kind": "oracle",
            "single_thread_value": fluid * k1 / dt1 / 1e6, "cpu_model": cpu_model(),
            "sample": f"{k} FP64 oracle steps of the full {g.nx}x{g.ny}x{g.nz} lattice "
                      f"({dt:.1f} s on {nthreads} threads); {k1} steps on one thread "
                      f"({dt1:.1f} s)"}


ARM_PARTS = {"0xd0c": "Arm Neoverse-N1", "0xd40": "Arm Neoverse-V1", "0xd49": "Arm Neoverse-N2",
             "0xd4f": "Arm Neoverse-V2"}


def cpu_model() -> str:
    """Host CPU model name from /proc/cpuinfo (Arm: the part number, named
    where known), or the platform."""
    try:
        for line in open("/proc/cpuinfo"):
            k, _, v = line.partition(":")
            k, v = k.strip(), v.strip()
            if k in ("model name", "Model") and v:
                return v
            if k == "CPU part" and v:
                return f"{ARM_PARTS.get(v, 'Arm')} (CPU part {v})"
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def main_reference(args):
    """Reference arm: the FP64 oracle timed on the host cores.  Each bench
    step is one oracle step of a z-slab of the workload lattice (around the
    droplet), the slab height chosen so the whole run takes about two
    minutes."""
    if int(os.environ.get("RANK", "0")) != 0:
        return 0
    g, p, drop = workload()
    nthreads = os.cpu_count() or 1
    cal = oracle_lattice(slab(g, 40, 8), p, dict(drop, center=(drop["center"][0],
                                                                drop["center"][1], 10.0)),
                         nthreads)
    t0 = time.perf_counter()
    cal.step(2)
    rate = 2 * g.nx * g.ny * 8 / max(time.perf_counter() - t0, 1e-6)
    per_step_cells = rate * 110.0 / max(1, args.steps + args.warmup)
    nz_s = int(max(4, min(g.nz, per_step_cells // (g.nx * g.ny))))
    z0 = max(0, min(g.nz - nz_s, 50 - nz_s // 2))
    sg = slab(g, z0, nz_s)
    sd = dict(drop, center=(drop["center"][0], drop["center"][1], drop["center"][2] - z0))
    L = oracle_lattice(sg, p, sd, nthreads)
    for _ in range(args.warmup):
        L.step(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        L.step(1)
    dt = time.perf_counter() - t0
    fluid = int(sg.N - sg.solid.sum())
    v = fluid * args.steps / dt / 1e6
    sample = (f"each step: one FP64 oracle step of planes z={z0}..{z0 + nz_s - 1} "
              f"({sg.nx}x{sg.ny}x{nz_s}, {fluid} fluid cells) of the workload lattice")
    line = {"metric": METRIC, "value": v, "unit": "MLUPS", "impl": "reference",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(g, int(g.N - g.solid.sum())),
            "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": nthreads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


ALGO_BYTES = {"fp32": ALGO_BYTES_FP32, "fp64": 2 * 19 * 2 * 8 + 1,
              # 16-bit: 2 sets x 19 x (read + write) x 2 B, the rest population's
              # low half (read + write), the flag
              "fp16": 2 * 19 * 2 * 2 + 2 * 2 + 1, "bf16": 2 * 19 * 2 * 2 + 2 * 2 + 1}


def init_ranks():
    """(world, rank) from the torchrun environment; joins the NCCL process
    group when world > 1 and selects this rank's GPU."""
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    if world > 1 and not dist.is_initialized():
        dist.init_process_group("nccl")
    return world, rank


def main_channels(args):
    """Many uneven lattices at once: the 64 droplet-in-square-channel
    lattices of synth.channel_batch_specs advanced by one persistent kernel
    per step (pflb_batch), launch shape chosen by the batch autotuner, steps
    replayed from a captured CUDA graph.  Also timed: the same lattices
    stepped one launch each per step (the per-lattice loop)."""
    import torch
    from paper_2512_01032_gb300 import pflb, shard
    world, rank = init_ranks()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    stream = torch.cuda.Stream(device=dev)
    storage = args.storage
    specs = synth.channel_batch_specs(args.count)
    # each rank advances its own share of the lattices (no data exchange)
    mine = shard.my_items([sp["nx"] * sp["ny"] * sp["nz"] for sp in specs], rank, world)
    lats, fluid, cells = [], 0, 0
    for sp in (specs[i] for i in mine):
        g, p, init = synth.channel_lattice(sp)
        L = pflb.Lattice(g.nx, g.ny, g.nz, solid=g.solid, wall_normal=g.normals(),
                         theta_cells=g.theta(), stream=stream, storage=storage, **p)
        L.init_tanh(0, init["center"], init["R"])
        lats.append(L)
        fluid += int(g.N - g.solid.sum())
        cells += g.N
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    # per-lattice loop: one fused launch per lattice per step
    for L in lats:
        L.step(args.warmup)
    a, b = ev(), ev()
    torch.cuda.synchronize(dev)
    a.record(stream)
    for _ in range(args.steps):
        for L in lats:
            L.step(1)
    b.record(stream)
    b.synchronize()
    loop_ms, = shard.reduce_max([a.elapsed_time(b)], device=dev)

    B = pflb.Batch(lats, stream=stream)
    best = B.tune(trial_steps=4)
    B.step(args.warmup)
    torch.cuda.synchronize(dev)
    clk = ClockSampler(dev.index)
    clk.start()
    a, b = ev(), ev()
    a.record(stream)
    B.step(args.steps - 1)
    B.step(1, diag_last=True)
    b.record(stream)
    b.synchronize()
    clocks = clk.stop()
    ms, = shard.reduce_max([a.elapsed_time(b)], device=dev)
    nonfinite = sum(L.last_diag(allow_nan=True)["nonfinite"] for L in lats)
    fluid, cells, nonfinite = (int(v) for v in shard.reduce_sum([fluid, cells, nonfinite],
                                                                 device=dev))
    ms_step = ms / args.steps
    value = fluid * args.steps / (ms * 1e-3) / 1e6
    launch = L.get_kernel()
    peak, peak_kind = hbm_peak()
    achieved = fluid * ALGO_BYTES[storage] / (ms_step * 1e-3) / 1e9
    line = {"metric": "batched AC+NS LB step MLUPS (many lattices)", "value": value,
            "unit": "MLUPS", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_step, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f32" if storage != "fp64" else "f64",
            "data": "synthetic",
            "config": {"workload": f"{args.count} droplet-in-square-channel lattices "
                                   f"(Ny=Nz in 32..96, Nx in 96..384, seeded), {storage} storage",
                       "cells": cells, "fluid_cells": fluid, "storage": storage,
                       "kernel": "k_batch persistent work list, graph-replayed",
                       "tuned_launch": {"bx": best[0], "by": best[1], "lz": best[2],
                                        "blocks_per_sm": best[3]},
                       "l2": "inputs larger than L2 (no flush)"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak,
                         "traffic": recorded_batch_traffic(storage, fluid),
                         "traffic_note": "ncu capture of 8 of the lattices, scaled by fluid cells",
                         "peak_kind": f"{peak_kind} copy bandwidth (MEASURED_PEAKS hbm_gbs)",
                         "algorithmic_bytes_per_cell": ALGO_BYTES[storage],
                         "kernel": "k_batch"},
            "per_lattice_loop": {"value": fluid * args.steps / (loop_ms * 1e-3) / 1e6,
                                 "unit": "MLUPS", "launches_per_step": len(lats)},
            "gpu_launches": 2 * args.steps, "clocks": clocks, "nonfinite": nonfinite}
    if rank == 0:
        print(json.dumps(line), flush=True)
    B.close()
    for L in lats:
        L.close()
    return 0


def serve_trace(server, prepared, trace):
    """Replay a request trace in real time: each request is submitted once
    the wall clock passes its arrival time, the server ticking in between."""
    t0 = time.perf_counter()
    tickets, k = [], 0
    while True:
        now = time.perf_counter() - t0
        while k < len(trace) and trace[k]["t_arrival"] <= now:
            g, p, spec = prepared[k]
            tickets.append(server.submit(g["nx"], g["ny"], g["nz"], spec, solid=g["solid"],
                                         wall_normal=g["normals"], theta_cells=g["theta"],
                                         **p))
            k += 1
        n = server.tick()
        if k == len(trace) and n == 0 and server.stats()["queued"] == 0:
            break
        if n == 0 and k < len(trace):
            time.sleep(max(0.0, min(0.01, trace[k]["t_arrival"] - now)))
    return tickets, time.perf_counter() - t0


def main_serve(args):
    """Critical-pressure solves served from a Poisson trace: continuous
    batching (one persistent batch kernel per step over all resident
    requests, admission by HBM budget) against the plain server (one request
    at a time, FP32, one fused launch per step) on the same trace."""
    import torch
    from paper_2512_01032_gb300 import pflb, shard
    world, rank = init_ranks()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    trace = synth.serving_trace(args.count)
    # each rank serves its own share of the requests, keeping arrival times
    mine = shard.my_items([4 * r["w"] * (r["w"] + 2) ** 2 for r in trace], rank, world)
    trace = [trace[i] for i in mine]
    prepared = []
    for req in trace:
        r = synth.constriction_request(req, ramp_every=args.ramp_every,
                                       max_steps=13 * args.ramp_every)
        g = r["geometry"]
        # the client's geometry (mask, normals, angles) is ready before the trace starts
        geo = dict(nx=g.nx, ny=g.ny, nz=g.nz, solid=g.solid, normals=g.normals(),
                   theta=g.theta())
        prepared.append((geo, r["params"], synth.constriction_spec(r, drive=args.drive)))
    out = {}
    modes = [("batched", dict(storage="fp32", batched=True,
                              max_active_cells=args.max_cells)),
             ("plain", dict(storage="fp32", batched=False, max_active=1))]
    if args.storage != "fp32":
        modes.insert(1, (f"batched_{args.storage}", dict(storage=args.storage, batched=True,
                                                         max_active_cells=args.max_cells)))
    for name, cfg in modes:
        S = pflb.Server(hbm_budget_bytes=int(args.budget_gb * (1 << 30)),
                        steps_per_tick=args.ramp_every // 2, **cfg)
        clk = ClockSampler(dev.index)
        clk.start()
        tickets, wall = serve_trace(S, prepared, trace)
        clocks = clk.stop()
        st = S.stats()
        res = [S.poll(t) for t in tickets]
        S.close()
        # over ranks: latencies and step counts gathered, makespan max, counters summed
        lat = shard.merged_sorted(q["latency_s"] for q in res if q["state"] == pflb.REQ_DONE)
        steps = [x for r in shard.gather([q["steps"] for q in res]) for x in r]
        makespan, = shard.reduce_max([st["makespan_s"]], device=dev)
        tot = shard.reduce_sum([st["completed"], st["failed"], st["rejected"],
                                st["cell_updates"],
                                sum(q["broke_through"] for q in res)], device=dev)
        out[name] = dict(solves_per_s=tot[0] / max(makespan, 1e-9),
                         p50_s=shard.nearest_rank(lat, 0.5), p99_s=shard.nearest_rank(lat, 0.99),
                         mean_s=sum(lat) / max(len(lat), 1),
                         makespan_s=makespan, completed=int(tot[0]), failed=int(tot[1]),
                         rejected=int(tot[2]), peak_gb=st["peak_bytes"] / 2 ** 30,
                         mlups=tot[3] / max(makespan, 1e-9) / 1e6,
                         broke_through=int(tot[4]),
                         host_s={k: st[k] for k in ("admit_s", "wait_s", "retire_s")},
                         wall_s=wall, steps=steps, clocks=clocks)
    same = out["batched"]["steps"] == out["plain"]["steps"]
    for v in out.values():
        v.pop("steps")
    extra = {k: v for k, v in out.items() if k not in ("batched", "plain")}
    b = out["batched"]
    line = {"metric": "served critical-pressure solves/s", "value": b["solves_per_s"],
            "unit": "solves/s", "n_gpus": world, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "p50_s": b["p50_s"], "p99_s": b["p99_s"],
            "config": {"workload": f"first {args.count} requests of the seeded Poisson trace "
                                   f"(20/s): square constriction channels 4w x w x w, "
                                   f"w in 48..96, beta ramp 0.7..1.3 every {args.ramp_every} "
                                   f"steps, at most {13 * args.ramp_every} steps",
                       "storage": "fp32", "budget_gb": args.budget_gb,
                       "max_active_cells": args.max_cells, "drive": args.drive,
                       "steps_per_tick": args.ramp_every // 2},
            "batched": out["batched"], "plain_sequential_fp32": out["plain"], **extra,
            "same_step_counts": same}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def batch_compare(dev, steps=100, warmup=5):
    """Compact batching figure for the default line: eight serving-trace
    lattices (square ducts with a central constriction, w = 48 .. 96, liquid
    slug, body-force drive) advanced as one batch at BF16 storage and, beside
    it, the same lattices at FP32 storage stepped one lattice at a time (the
    per-lattice loop of plain serving).  Device time of `steps` steps each
    (CUDA events on the lattices' stream), a few seconds in all."""
    import torch
    from paper_2512_01032_gb300 import pflb
    stream = torch.cuda.Stream(device=dev)
    out = {"workload": "8 serving-trace lattices (w = 48, 52, .., 96 ducts with a central "
                       "constriction), BF16 batch vs per-lattice FP32 loop", "steps": steps}
    for storage, batched in (("bf16", True), ("fp32", False)):
        lats, fluid = [], 0
        for w in (48, 52, 56, 64, 72, 80, 88, 96):
            r = synth.constriction_request(dict(w=w, ratio=0.5, theta=120.0))
            g, i = r["geometry"], r["init"]
            L = pflb.Lattice(g.nx, g.ny, g.nz, solid=g.solid, wall_normal=g.normals(),
                             theta_cells=g.theta(), stream=stream, storage=storage,
                             **r["params"])
            L.init_tanh(i["shape"], i["center"], i["R"], i["normal"])
            L.set_force((r["beta0"] * r["p_crit"] / r["length"], 0.0, 0.0))
            lats.append(L)
            fluid += int(g.N - g.solid.sum())
        B = pflb.Batch(lats, stream=stream) if batched else None
        run = (lambda n: B.step(n)) if batched else (
            lambda n: [L.step(1) for _ in range(n) for L in lats])
        run(warmup)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        a.record(stream)
        run(steps)
        b.record(stream)
        b.synchronize()
        ms = a.elapsed_time(b)
        key = "batched_bf16" if batched else "per_lattice_fp32"
        out[key] = {"value": fluid * steps / (ms * 1e-3) / 1e6, "unit": "MLUPS",
                    "fluid_cells": fluid, "ms_per_step": ms / steps,
                    "kernels": sorted({KERNEL_NAMES.get(L.get_kernel()["kind"], "?")
                                       for L in lats})}
        if B is not None:
            B.close()
        for L in lats:
            L.close()
    out["ratio"] = out["batched_bf16"]["value"] / out["per_lattice_fp32"]["value"]
    return out


def serve_compare(count=8, ramp_every=500, budget_gb=16.0, max_cells=8 << 20):
    """Compact serving figure for the default line: the first `count`
    requests of the seeded Poisson trace (critical-pressure solves in
    constriction ducts, body-force ramp of `ramp_every` steps per beta level,
    at most 13 levels) replayed in real time through the batching server at
    BF16 and through the plain server at FP32 (one request at a time), on
    the host clock as the full serving workload measures them.  Tens of
    seconds in all; the full trace with the stated ramp is
    --workload serve."""
    from paper_2512_01032_gb300 import pflb, shard
    trace = synth.serving_trace(count)
    prepared = []
    for req in trace:
        r = synth.constriction_request(req, ramp_every=ramp_every, max_steps=13 * ramp_every)
        g = r["geometry"]
        geo = dict(nx=g.nx, ny=g.ny, nz=g.nz, solid=g.solid, normals=g.normals(),
                   theta=g.theta())
        prepared.append((geo, r["params"], synth.constriction_spec(r)))
    out = {"workload": f"first {count} requests of the seeded serving trace, beta ramp every "
                       f"{ramp_every} steps, at most {13 * ramp_every} steps",
           "budget_gb": budget_gb}
    for name, cfg in (("batched_bf16", dict(storage="bf16", batched=True,
                                            max_active_cells=max_cells)),
                      ("plain_fp32", dict(storage="fp32", batched=False, max_active=1))):
        S = pflb.Server(hbm_budget_bytes=int(budget_gb * (1 << 30)),
                        steps_per_tick=ramp_every // 2, **cfg)
        tickets, wall = serve_trace(S, prepared, trace)
        st = S.stats()
        res = [S.poll(t) for t in tickets]
        S.close()
        lat = sorted(q["latency_s"] for q in res if q["state"] == pflb.REQ_DONE)
        out[name] = {"solves_per_s": st["completed"] / max(st["makespan_s"], 1e-9),
                     "p50_s": shard.nearest_rank(lat, 0.5),
                     "p99_s": shard.nearest_rank(lat, 0.99),
                     "completed": st["completed"], "failed": st["failed"],
                     "mlups": st["cell_updates"] / max(st["makespan_s"], 1e-9) / 1e6,
                     "broke_through": sum(q["broke_through"] for q in res)}
    out["ratio_solves_per_s"] = out["batched_bf16"]["solves_per_s"] / max(
        out["plain_fp32"]["solves_per_s"], 1e-12)
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--tile", type=str, default="", help="bx,by,lz of the fused kernel")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the compact batching and serving figures of the default line")
    ap.add_argument("--workload", choices=["sessile", "channels", "serve"], default="sessile",
                    help="sessile: the 128^3 sessile droplet (default); channels: many "
                         "uneven channel lattices advanced as one batch; serve: a request "
                         "trace through the batching server and the plain server")
    ap.add_argument("--size", type=int, default=N_BOX,
                    help="sessile: lattice edge (the headline workload is 128; smaller "
                         "sizes are for profiler captures)")
    ap.add_argument("--storage", choices=["fp32", "fp16", "bf16", "fp64"], default="bf16",
                    help="population storage of the channels workload")
    ap.add_argument("--count", type=int, default=64,
                    help="lattices of the channels workload / requests of the serve workload")
    ap.add_argument("--ramp-every", type=int, default=500, help="serve: steps per beta level")
    ap.add_argument("--budget-gb", type=float, default=16.0, help="serve: HBM budget")
    ap.add_argument("--drive", choices=["force", "pressure"], default="force",
                    help="serve: ramp pressure as a body force (periodic) or as a pressure "
                         "difference across open x boundaries")
    ap.add_argument("--max-cells", type=int, default=8 << 20,
                    help="serve: cap on resident cells of the batching server (0 = none)")
    args = ap.parse_args(argv)
    if args.impl == "reference":
        return main_reference(args)
    args.warmup = max(args.warmup, 3)
    if args.workload == "channels":
        return main_channels(args)
    if args.workload == "serve":
        return main_serve(args)

    import torch
    import torch.distributed as dist
    from paper_2512_01032_gb300 import pflb

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)

    g, p, drop = workload(args.size)
    fluid = int(g.N - g.solid.sum())
    L = pflb.Lattice(g.nx, g.ny, g.nz, solid=g.solid, wall_normal=g.normals(),
                     theta_cells=g.theta(), stream=stream, storage="fp32", **p)
    if args.tile:
        bx, by, lz = (int(v) for v in args.tile.split(","))
        L.set_kernel(0, bx, by, lz)
    L.init_tanh(0, drop["center"], drop["R"])
    L.set_diag_every(1)
    if not args.tile:
        # planes per block: the library's autotuner times real steps of this
        # lattice at a few depths and keeps the fastest (before the warm-up)
        L.tune(50)

    # ---------------------------------------------- device-resident timing
    L.step(args.warmup)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    clk = ClockSampler(local)
    clk.start()
    # Clock window: the sampler polls every 100 ms, longer than a short timed
    # region, so the same workload keeps running untimed for about a second
    # before the timed steps; the clock record covers that window and the
    # timed region.
    window_steps, t_win = 0, time.perf_counter()
    while time.perf_counter() - t_win < CLOCK_WINDOW_S:
        L.step(25)
        torch.cuda.synchronize(dev)
        window_steps += 25
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    start.record(stream)
    L.step(args.steps)
    end.record(stream)
    end.synchronize()
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    clocks = clk.stop()
    ms = start.elapsed_time(end)
    if world > 1:
        t = torch.tensor([ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    d = L.last_diag()
    ms_step = ms / args.steps
    value = world * fluid * args.steps / (ms * 1e-3) / 1e6

    launch = L.get_kernel()
    # one launch per step: the pipelined kernel updates each block's wall
    # nodes after its march (per-block lists built for the launch shape)
    launches_per_step = 1
    peak, peak_kind = hbm_peak()
    achieved = fluid * ALGO_BYTES_FP32 / (ms_step * 1e-3) / 1e9
    traffic = recorded_traffic(KERNEL_NAMES.get(launch["kind"], ""))
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic,
                "peak_kind": f"{peak_kind} copy bandwidth (MEASURED_PEAKS hbm_gbs)",
                "algorithmic_bytes_per_cell": ALGO_BYTES_FP32,
                "kernel": KERNEL_NAMES.get(launch["kind"], str(launch["kind"]))}

    # ---------------------------------------------- end to end (host buffers)
    e2e = None
    if not args.no_e2e:
        phi0 = torch.empty(g.N, dtype=torch.float64, pin_memory=True).numpy()
        L2 = pflb.Lattice(g.nx, g.ny, g.nz, solid=g.solid, wall_normal=g.normals(),
                          theta_cells=g.theta(), stream=stream, storage="fp32", **p)
        L2.set_kernel(launch["kind"], launch["bx"], launch["by"], launch["lz"])
        L2.init_tanh(0, drop["center"], drop["R"])
        phi0[:] = L2.read("phi")
        L2.set_diag_every(1)
        force = np.zeros(3)
        # two page-locked landing buffers for the per-step diagnostics: step
        # n's read is queued behind step n and waited for after step n + 1
        # has been queued, so the GPU never idles on the read
        rawsz = ctypes.sizeof(pflb.DiagRaw)
        raw = torch.empty(2 * rawsz, dtype=torch.uint8, pin_memory=True)
        rp = [raw.data_ptr(), raw.data_ptr() + rawsz]
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        L2.init_phi(phi0)
        prev = None
        for n in range(args.steps):
            L2.set_force(force)
            L2.step(1)
            tk = L2.last_diag_async(rp[n & 1])
            if prev is not None:
                L2.diag_wait(prev, rp[(n - 1) & 1])
            prev = tk
        last = L2.diag_wait(prev, rp[(args.steps - 1) & 1])
        phi_out = L2.read("phi")
        t1 = time.perf_counter()
        te = t1 - t0
        if world > 1:
            t = torch.tensor([te], device=dev, dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            te = float(t.item())
        e2e = {"value": world * fluid * args.steps / te / 1e6, "unit": "MLUPS",
               "h2d_bytes_per_step": (8 * g.N + 24 * args.steps) / args.steps,
               "d2h_bytes_per_step": (rawsz * args.steps + 8 * g.N) / args.steps,
               "path": "pflb_init_phi(host phi) + per step pflb_set_force + pflb_step + "
                       "pflb_last_diag_async into page-locked host memory, waited for one "
                       "step later (pflb_diag_wait) + final pflb_read(phi)",
               "final_mass": float(phi_out.sum()), "final_diag_mass": last["mass"]}
        L2.close()

    batch = serve = None
    if rank == 0 and world == 1 and not args.no_batch:
        batch = batch_compare(dev)
        serve = serve_compare()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(g, p, drop)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic",
                "config": dict(config_of(g, fluid, launch["kind"]), launch=launch),
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": args.steps * launches_per_step,
                "clocks": dict(clocks, window=f"{window_steps} untimed steps of the same "
                               f"workload ({CLOCK_WINDOW_S:.1f} s) just before the timed "
                               "region, and the timed region"),
                "diag_last": {"mass": d["mass"], "dp": d["dp"], "u_max": d["u_max"],
                              "nonfinite": d["nonfinite"]},
                "batch": batch, "serve": serve}
        print(json.dumps(line), flush=True)
    L.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
