#!/usr/bin/env python3
"""Benchmark of the sliding-mesh DGSEM hot path on one GB300 (replicas across GPUs).

A step is one low-storage RK4 step (five stages) of the interface-heavy single solve:
two blocks of 4 x 256 x 256 hexahedra (524,288 elements, 65,536 sliding faces per side),
N = 5 (113.2 M DOF), FP32 state with FP64 mapping and mortar matrices, moving block at
v = 0.37, smooth random initial field of 8 seeded Fourier modes per primitive variable.
Every RK step runs the step-parameter kernel once (mapper and mortar matrices of its five
stages) and every stage the fused interface kernel and the element kernel (volume, surface,
RK update), replayed from a CUDA graph.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload interface-heavy|serving|cylinder] [--precision fp32|fp64]

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on the host
cores on a bounded sample of the same workload (fewer elements along z).
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
sys.path.insert(0, ROOT)

METRIC = "interface face-updates/s & DOF-updates/s vs FP64 plain path; p50/p99 solve latency"
UNIT = "DOF-updates/s"
WORKLOAD = ("interface-heavy single solve: 2 blocks x 4x256x256 hexes (524,288 elements, 65,536 "
            "sliding faces), N=5 (113.2M DOF), FP32 state, FP64 mapping and mortar matrices, "
            "v=0.37, 8 seeded Fourier modes per primitive variable on rho=1, p=1")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--fp64-steps", type=int, default=6)
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--profile-steps", type=int, default=10)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--nz", type=int, default=256, help="elements along z (256 = the full workload)")
    ap.add_argument("--workload", choices=["interface-heavy", "serving", "cylinder", "annular", "cone"],
                    default="interface-heavy")
    ap.add_argument("--volume", choices=["weak", "split"], default="weak",
                    help="volume integral of the interface-heavy headline: weak form, or the split form")
    ap.add_argument("--riemann", choices=["rusanov", "roe"], default=None,
                    help="Riemann solver of the headline (default: Rusanov for the weak form, Roe/HH for the split form)")
    ap.add_argument("--two-steps", type=int, default=20,
                    help="timed steps of the two-interface solve (the workload closed in x) beside the headline; 0: skip")
    ap.add_argument("--split-steps", type=int, default=20,
                    help="timed steps of the split-form (Pirozzoli, Roe/HH) solve beside the weak-form headline; 0: skip")
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32", help="cylinder workload state precision")
    ap.add_argument("--requests", type=int, default=256)
    ap.add_argument("--serve-steps", type=int, default=100,
                    help="RK steps per serving request (the configuration asks 500; the default bench line runs "
                         "fewer to stay within minutes and states it); 0 skips the serving leg of the default line")
    ap.add_argument("--load", type=float, default=0.8, help="offered load as a fraction of measured capacity")
    return ap.parse_args()


# ------------------------------------------------------------------------------ helpers
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during a region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 8:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[4 + k].lower().startswith("active")})
        loaded = [x for x in sm if mx and x > 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


class Replicas:
    """Bookkeeping of N independent replicas of the workload, one per rank (the path does not
    shard: no collective on the data path).  Only the timing needs the ranks: a barrier
    around the timed region and the maximum of the per-rank times, over NCCL on GPUs or
    gloo on CPUs; the whole-job value is N x the units one rank processes / that maximum."""

    def __init__(self, world: int, device=None):
        self.world = world
        self.device = device

    def barrier(self):
        import torch
        if self.world > 1:
            import torch.distributed as dist
            dist.barrier()
        if self.device is not None and self.device.type == "cuda":
            torch.cuda.synchronize()

    def max(self, x: float) -> float:
        if self.world == 1:
            return x
        import torch
        import torch.distributed as dist
        t = torch.tensor([x], dtype=torch.float64, device=self.device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    def value(self, units_per_rank: float, seconds: float) -> float:
        return self.world * units_per_rank / seconds


def source_sha(paths):
    h = hashlib.sha256()
    for p in paths:
        h.update(open(os.path.join(ROOT, p), "rb").read())
    return h.hexdigest()[:16]


ELEMENT_SOURCES = ["paper_2008_04356_gb300/csrc/sm_element.cuh", "paper_2008_04356_gb300/csrc/sm_common.cuh"]

# FP64 operations the plain FP64 path executes per DOF-update (N = 5, Rusanov), averaged over
# the five stages of a step: DFMA x 2 + DADD + DMUL counted with ncu on the element kernel
# (426.3 per DOF in a stage, 416.3 in the first stage, which reads no RK register), plus the
# interface kernel's share (16.1 per DOF), counted on 2 x 4 x 256 x 8 hexes
FP64_EXECUTED_FLOP_PER_DOF = (4 * 426.25 + 416.25) / 5 + 16.07


def algorithmic_flop_per_dof(N: int, faces: int, dof: int) -> float:
    """Floating-point operations of one DOF-update of the weak-form operator with the Rusanov
    flux on Cartesian elements, counted from the method (each conforming face's flux once):
      primitives 12 (1/rho, 3 velocities, kinetic energy, pressure), three ALE axis fluxes 27,
      sum-factorised contractions 3 directions x 5 variables x (N+1) multiply-adds = 30 (N+1),
      metric factors 25, the element's share of face fluxes 3 (N+1)^2 per (N+1)^3 nodes x 78
      (two states' primitives 24, normal fluxes 18, sound speeds 6, wave speed 5, flux 20,
      surface element 5), surface lifting 6 (N+1)^2 x 5 multiply-adds per element, 1/J 5,
      RK update 25; plus the interface's share per face pair: the forward projections of both
      sides onto both mortars and the back-projections of both mortars onto both faces,
      8 x 5 (N+1)^3 multiply-adds = 80 (N+1)^3 flop, and 2 (N+1)^2 mortar fluxes x 78."""
    npn = N + 1
    per_node = 12 + 27 + 30 * npn + 25 + 3.0 / npn * 78 + 60.0 / npn + 5 + 25
    per_face = 2 * 40 * npn ** 3 + 2 * npn ** 2 * 78
    return per_node + per_face * faces / dof


def fp64_fma_peak(stream):
    """Measured FP64 FMA throughput of this GPU (GFLOP/s): the library's DFMA probe on every
    SM (SM count from the device properties), best of 5 launches timed with CUDA events, the
    SM clock sampled meanwhile."""
    import torch
    from paper_2008_04356_gb300 import slidemesh
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    sms = props.multi_processor_count
    blocks, threads, iters = sms * 8, 256, 4096
    out = torch.empty(blocks * threads, dtype=torch.float64, device="cuda")
    flop = 16.0 * iters * blocks * threads
    slidemesh.sm_fp64_fma_probe(blocks, threads, iters, out, stream)
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    best = None
    for _ in range(8):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        slidemesh.sm_fp64_fma_probe(blocks, threads, iters, out, stream)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        best = ms if best is None else min(best, ms)
    clk = clocks.stop()
    assert torch.isfinite(out).all().item()
    return {"gflops": flop / (best * 1e-3) / 1e9, "sms": sms, "sm_mhz": clk.get("sm_mhz"),
            "how": "FP64 FMA probe: %d x %d threads x 8 chains x %d fma, best of 8 launches" % (blocks, threads, iters)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "of measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "of fallback"


# elements of the full interface-heavy workload (2 blocks x 4x256x256)
FULL_ELEMENTS = 2 * 4 * 256 * 256


def ncu_traffic(nelem: int = FULL_ELEMENTS):
    """DRAM bytes per element-kernel launch of nelem elements from the committed ncu summary
    (scaled from the full workload by the element count, as the traffic is), if it was taken
    on the current element-kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "dg_element_traffic.json")
    try:
        rec = json.load(open(path))
    except (OSError, ValueError):
        return None
    if rec.get("source_sha") != source_sha(ELEMENT_SOURCES):
        return None
    full = rec.get("dram_bytes_per_launch_full_workload")
    return None if full is None else full * nelem / FULL_ELEMENTS


def cpu_baseline(seconds: float, volume: int = 0, riemann: int = 0):
    """The FP64 oracle, as it stands, on the host cores: whole RK steps of the same workload
    with fewer elements along z (bounded sample)."""
    import numpy as np
    from oracle import oracle as O
    from paper_2008_04356_gb300 import synth
    nz = 4
    p = synth.config_interface_heavy(seed=1, precision=synth.FP64, nz=nz)
    p.volume, p.riemann = volume, riemann
    o = O.Oracle(p)
    U = o.init_state()
    G = np.zeros_like(U)
    dt = synth.cfl_dt(p)
    t = o.step(U, G, 0.0, dt, 1)            # warm-up step
    steps, t0 = 0, time.perf_counter()
    while True:
        t = o.step(U, G, t, dt, 1)
        steps += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return {"value": p.ndof * 5 * steps / el, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
            "sample": "%d RK steps (5 stages each) of 2 blocks x 4x256x%d hexes, N=5 (%d DOF), FP64, %.1f s"
                      % (steps, nz, p.ndof, el),
            "interface_face_updates_per_s": p.n_faces * 5 * steps / el}


# ------------------------------------------------------------------------------ reference arm
def run_reference(args, rank):
    if rank != 0:
        return
    import numpy as np
    from oracle import oracle as O
    from paper_2008_04356_gb300 import synth
    # size the sample so that (warmup + steps) whole RK steps take about two minutes
    volume = synth.VOLUME_SPLIT if args.volume == "split" else synth.VOLUME_WEAK
    riemann = synth.ROE_HH if (args.riemann or ("roe" if args.volume == "split" else "rusanov")) == "roe" \
        else synth.RUSANOV
    probe = synth.config_interface_heavy(seed=1, precision=synth.FP64, nz=1)
    probe.volume, probe.riemann = volume, riemann
    o = O.Oracle(probe)
    U = o.init_state()
    G = np.zeros_like(U)
    dt = synth.cfl_dt(probe)
    t0 = time.perf_counter()
    o.step(U, G, 0.0, dt, 1)
    per_nz = time.perf_counter() - t0
    budget = 120.0 / max(1, args.steps + args.warmup)
    nz = int(max(1, min(256, budget / max(per_nz, 1e-6))))
    p = synth.config_interface_heavy(seed=1, precision=synth.FP64, nz=nz)
    p.volume, p.riemann = volume, riemann
    o = O.Oracle(p)
    U = o.init_state()
    G = np.zeros_like(U)
    dt = synth.cfl_dt(p)
    t = o.step(U, G, 0.0, dt, args.warmup) if args.warmup else 0.0
    t0 = time.perf_counter()
    t = o.step(U, G, t, dt, args.steps)
    el = time.perf_counter() - t0
    value = p.ndof * 5 * args.steps / el
    sample = "%d RK steps of 2 blocks x 4x256x%d hexes, N=5 (%d DOF), FP64 oracle" % (args.steps, nz, p.ndof)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "interface_face_updates_per_s": p.n_faces * 5 * args.steps / el}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------ serving
def serving_stream(n, steps, seed=12345):
    """Requests shaped like the serving configuration: N in {3,5,7}, 4k-200k elements
    (log-uniform, two blocks of 4 x m x m hexes), plane interface, v ~ U[0.1,1], an entropy
    wave carried at Mach ~ U[0.1,0.8], FP32 bulk; seeded SplitMix64 draws."""
    import math
    from paper_2008_04356_gb300 import synth
    u = synth.uniform(seed, 4 * n).reshape(n, 4)
    reqs = []
    for r in range(n):
        N = (3, 5, 7)[min(2, int(u[r, 0] * 3))]
        E = math.exp(math.log(4000) + u[r, 1] * (math.log(200000) - math.log(4000)))
        mm = max(2, int(round(math.sqrt(E / 8.0))))
        h = 1.0 / mm
        c = math.sqrt(1.4)
        ma = 0.1 + 0.7 * u[r, 3]
        p = synth.Problem(N=N, nel_s=(4, mm, mm), nel_m=(4, mm, mm), x0=0.0, x1=4 * h, x2=8 * h, y1=1.0, z1=1.0,
                          v=0.1 + 0.9 * u[r, 2], flow=synth.FLOW_ENTROPY_WAVE,
                          fpar=(1.0, 0.2, 0.0, 1.0, 1.0, ma * c, 0.0, 0.0, 1.0), precision=synth.FP32)
        reqs.append((p, synth.cfl_dt(p), steps))
    return reqs


def run_serving(args):
    import torch
    from paper_2008_04356_gb300 import build as B
    torch.cuda.set_device(0)
    B.build_library()
    line = serving_results(args)
    line.update({"metric": METRIC, "workload": "serving", "n_gpus": 1, "data": "synthetic", "dtype": "f32"})
    print(json.dumps(line), flush=True)


def serving_results(args):
    """The serving stream through sm_server_* (Poisson arrivals at a fraction of the batched
    path's measured capacity, admission under a 120 GB budget), its p50/p99 time to solution
    (submit -> CUDA event after the solve's last step) and throughput, beside the plain FP64
    path one solve at a time on a sample of the same requests."""
    import numpy as np
    import torch
    from paper_2008_04356_gb300 import slidemesh, synth
    reqs = serving_stream(args.requests, args.serve_steps)
    work = [p.ndof * 5 * n for p, _, n in reqs]
    # capacity probe: the batched path on the first 8 requests at once
    probe = [slidemesh.Solver(p) for p, _, _ in reqs[:8]]
    for s_ in probe:
        s_.init_state()
    bt = slidemesh.Batch(probe, [dt for _, dt, _ in reqs[:8]])
    bt.autotune()
    bt.step(2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    bt.step(6)
    torch.cuda.synchronize()
    cap = sum(p.ndof * 5 * 6 for p, _, _ in reqs[:8]) / (time.perf_counter() - t0)
    bt.close()
    for s_ in probe:
        s_.close()
    rate = args.load * cap / (sum(work) / len(work))            # requests per second
    gaps = -np.log(1.0 - synth.uniform(777, len(reqs))) / rate   # Poisson arrivals
    srv = slidemesh.Server(hbm_budget_bytes=120 << 30, max_slots=256)
    tickets = []
    t_start = time.perf_counter()
    t_next = t_start
    for (p, dt, n), g in zip(reqs, gaps):
        t_next += g
        while time.perf_counter() < t_next:
            time.sleep(min(0.002, max(0.0, t_next - time.perf_counter())))
        tickets.append(srv.submit(p, dt, n))
    srv.wait(3600)
    res = [srv.poll(t) for t in tickets]
    st = srv.stats()
    srv.close()
    lat = np.array([r["t_done"] - r["t_submit"] for r in res])
    span = max(r["t_done"] for r in res) - min(r["t_submit"] for r in res)
    thr = sum(work) / span
    # one-at-a-time FP64 plain path on a sample of the same requests
    t64, w64 = 0.0, 0
    for p, dt, n in reqs[:12]:
        q = synth.Problem(**{**p.__dict__, "precision": synth.FP64})
        s64 = slidemesh.Solver(q)
        s64.init_state()
        s64.step(dt, 1)
        torch.cuda.synchronize()
        a = time.perf_counter()
        s64.step(dt, 10)
        torch.cuda.synchronize()
        t64 += time.perf_counter() - a
        w64 += q.ndof * 5 * 10
        s64.close()
    v64 = w64 / t64
    return {"value": thr, "unit": UNIT,
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "requests": len(reqs), "completed": st["completed"], "failed": st["failed"],
            "max_concurrent": st["max_concurrent"], "peak_bytes": st["peak_bytes"],
            "offered_load": args.load, "arrival_rate_per_s": rate, "capacity_probe": cap,
            "makespan_s": span, "steps_per_request": args.serve_steps,
            "fp64_one_at_a_time": {"value": v64, "unit": UNIT, "sample": "12 requests x 10 steps"},
            "batched_fp32_over_fp64_one_at_a_time": thr / v64,
            "config": {"workload": "Poisson stream of %d sliding-mesh Euler solves, N in {3,5,7}, 4k-200k elements, "
                                   "v in U[0.1,1], Mach in U[0.1,0.8], %d steps each, FP32 bulk, FP64 mapping, "
                                   "120 GB budget" % (len(reqs), args.serve_steps),
                       "steps_per_request": args.serve_steps,
                       "steps_note": ("as configured (500 steps per request)" if args.serve_steps == 500 else
                                      "reduced from the configuration's 500 steps per request to %d to keep the "
                                      "default benchmark within minutes; --serve-steps 500 runs it as configured"
                                      % args.serve_steps)},
            "time_to_solution": "submit (host clock) to a CUDA event recorded after the solve's last step"}


# ------------------------------------------------------------------------------ our arm
CYL_WORKLOAD = ("rotating cylindrical sliding interface, Navier-Stokes with BR1 lifting: annular sector "
                "r in [1,1.5], theta in [0,pi/4] periodic, z in [0,0.5]; rotor (inside) and stator blocks "
                "of 24x48x16 curved hexes each (36,864 elements, 768 sliding faces per side), rotor "
                "omega=0.4, N=7 (18.9M DOF), Re=1e4, Pr=0.72, Mach 0.3 axial stream with a pressure pulse")


ANN_WORKLOAD = ("rotating plane annular sliding interface normal to the axis, Euler: rotor z in [0,0.25] below "
                "the stator z in [0.25,0.5], radii r in [1,1.5], theta in [0,pi/4] periodic, slip walls; rotor "
                "and stator blocks of 24x48x16 curved hexes each (36,864 elements, 768 sliding faces per side), "
                "rotor omega=0.4, N=7 (18.9M DOF), fluid at rest with a pressure pulse on the interface")


CONE_WORKLOAD = ("rotating conical sliding interface about the axis, Euler: half-angle pi/6, generator s in "
                 "[0,0.5], normal offset n in [1,1.25] (rotor, inside) and [1.25,1.5] (stator), theta in "
                 "[0,pi/4] periodic, slip walls; rotor and stator blocks of 24x48x16 curved hexes each (36,864 "
                 "elements, 768 sliding faces per side), rotor omega=0.4, N=7 (18.9M DOF), fluid at rest with a "
                 "pressure pulse on the interface")


def shape_problem(workload: str, volume: str, riemann, prec: int):
    """The curved-element workload at full size: the cylinder with Navier-Stokes, or the
    annulus or the cone with Euler; weak or split form (the split form with Roe/HH unless
    Rusanov is asked for; on the cylinder it is the paper's production scheme, split form
    with BR1)."""
    from paper_2008_04356_gb300 import synth
    if workload == "cone":
        p = synth.config_cone(N=7, nel=(24, 48, 16), omega=0.4, alpha=math.pi / 6, flow="pulse", precision=prec)
    elif workload == "annular":
        p = synth.config_annular(N=7, nel=(24, 48, 16), omega=0.4, flow="pulse", precision=prec)
    elif workload == "cylinder":
        p = synth.config_cylinder(N=7, nel=(24, 48, 16), omega=0.4, flow="pulse", precision=prec,
                                  physics=synth.NAVIER_STOKES)
    else:
        raise ValueError(workload)
    if volume == "split":
        p.volume = synth.VOLUME_SPLIT
        p.riemann = synth.RUSANOV if riemann == "rusanov" else synth.ROE_HH
    return p


def run_cylinder(args, rank, world, local):
    """The rotating cylindrical interface with Navier-Stokes at N = 7 (or, --workload annular
    or cone, the plane annular or the conical interface with Euler, weak or split form): RK
    steps through the curvilinear kernels (interface lifting, lifting, viscous interface
    flux, element)."""
    import torch
    from paper_2008_04356_gb300 import build as B, slidemesh, synth
    import torch.distributed as dist
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    rep = Replicas(world, torch.device("cuda", local))
    B.build_library()
    stream = torch.cuda.current_stream()
    prec = synth.FP64 if args.precision == "fp64" else synth.FP32
    annular = args.workload in ("annular", "cone")     # the Euler shapes
    p = shape_problem(args.workload, args.volume, args.riemann, prec)
    split = p.volume == synth.VOLUME_SPLIT
    sol = slidemesh.Solver(p)
    sol.init_state()
    dt = synth.cfl_dt(p)
    sol.step(dt, args.warmup)
    rep.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    rep.barrier()
    e0.record(stream)
    sol.step(dt, args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    rep.barrier()
    clk = clocks.stop()
    ms = rep.max(e0.elapsed_time(e1))
    value = rep.value(p.ndof * 5 * args.steps, ms * 1e-3)
    kms, kcnt = sol.step_profiled(dt, args.profile_steps)
    sb = 8 if prec == synth.FP64 else 4
    # element kernel per DOF-update: U in/out, G in (4 of 5 stages)/out, 13 geometry values,
    # 15 gradients (Navier-Stokes)
    elem_bytes = ((2 + 1 + 0.8) * 5 + 13 + (0 if annular else 15)) * sb * p.ndof
    elem_ms = kms[2] / kcnt[2]
    peaks, peak_kind = measured_peaks()
    hbm = float(peaks["hbm_gbs"])
    achieved = elem_bytes / (elem_ms * 1e-3) / 1e9
    d = sol.diag()
    if rank != 0:
        sol.close()
        if world > 1:
            dist.destroy_process_group()
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if prec == synth.FP64 else "f32", "data": "synthetic",
        "config": {"workload": {"cone": CONE_WORKLOAD, "annular": ANN_WORKLOAD}.get(args.workload, CYL_WORKLOAD),
                   "elements": p.nelem, "N": p.N, "dof": p.ndof,
                   "sliding_faces_per_side": p.n_faces, "riemann": "roe_hh" if p.riemann == synth.ROE_HH else "rusanov",
                   "volume": "split form, Pirozzoli two-point flux" if split else "weak form", "mu": p.mu,
                   "l2": "inputs larger than L2 (%.2f GB state + %.2f GB geometry)" % (
                       p.ndof * 5 * sb / 1e9, p.ndof * 13 * sb / 1e9),
                   "parallelism": "replicas" if world > 1 else "single GPU", "dt": dt, "final_t": d["t"]},
        "interface_face_updates_per_s": rep.value(p.n_faces * 5 * args.steps, ms * 1e-3),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                     "traffic": None, "kernel": "%s<N=7, %s, %s, stage%s>" % (
                         "curved_split_kernel" if split else "curved_element_kernel",
                         "double" if prec == synth.FP64 else "float",
                         "Roe/HH" if p.riemann == synth.ROE_HH else "Rusanov", "" if annular else ", NS"),
                     "peak_source": peak_kind, "algorithmic_bytes_per_launch": elem_bytes, "avg_launch_ms": elem_ms},
        "kernels": {"stage_params": {"launches": kcnt[0], "ms": kms[0]},
                    "lifting_and_interface": {"launches": kcnt[1], "ms": kms[1], "avg_ms": kms[1] / max(kcnt[1], 1)},
                    "curved_element": {"launches": kcnt[2], "ms": kms[2], "avg_ms": elem_ms}},
        # per step: the five stages' parameters in one launch, then per stage the interface
        # kernel and the element kernel (Euler) or interface lifting, lifting, viscous
        # interface flux and element kernel (Navier-Stokes)
        "gpu_launches": (1 + (2 if annular else 4) * 5) * args.steps,
        "clocks": clk,
        "diag": {"n_delta": d["n_delta"], "s_delta": d["s_delta"], "finite": d["status"] == 0,
                 "totals": d["totals"]},
    }
    sol.close()
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.workload == "serving":
        if rank == 0:
            run_serving(args)
        return
    if args.workload in ("cylinder", "annular", "cone"):
        run_cylinder(args, rank, world, local)
        return
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2008_04356_gb300 import build as B, slidemesh, synth

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    B.build_library()
    stream = torch.cuda.current_stream()

    rep = Replicas(world, torch.device("cuda", local))
    barrier, max_over_ranks = rep.barrier, rep.max

    p = synth.config_interface_heavy(seed=1 + rank, precision=synth.FP32, nz=args.nz)
    p.volume = synth.VOLUME_SPLIT if args.volume == "split" else synth.VOLUME_WEAK
    riem = args.riemann or ("roe" if args.volume == "split" else "rusanov")
    p.riemann = synth.ROE_HH if riem == "roe" else synth.RUSANOV
    kname = "%s<N=5, float, %s, stage>" % ("dg_element_split_kernel" if args.volume == "split" else "dg_element_kernel",
                                          "Roe/HH" if riem == "roe" else "Rusanov")
    sol = slidemesh.Solver(p)
    sol.init_state()
    dt = synth.cfl_dt(p)
    sol.step(dt, args.warmup)
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # the timed steps in five consecutive chunks, an event after each: per-chunk step times
    # give the spread (median, min, max) beside the whole-region value
    nrep = 5 if args.steps >= 5 else 1
    cuts = [args.steps * r // nrep for r in range(nrep + 1)]
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(nrep - 1)]
    e0.record(stream)
    for r in range(nrep):
        sol.step(dt, cuts[r + 1] - cuts[r])
        if r < nrep - 1:
            evs[r].record(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1))
    marks = [e0] + evs + [e1]
    rep_ms = sorted(marks[r].elapsed_time(marks[r + 1]) / (cuts[r + 1] - cuts[r]) for r in range(nrep))
    repeats = {"chunks": nrep, "ms_per_step_median": rep_ms[nrep // 2], "ms_per_step_min": rep_ms[0],
               "ms_per_step_max": rep_ms[-1]}
    value = rep.value(p.ndof * 5 * args.steps, ms * 1e-3)
    face_rate = rep.value(p.n_faces * 5 * args.steps, ms * 1e-3)
    d = sol.diag()

    # per-kernel device times of the same stage sequence (event pairs around each launch)
    kms, kcnt = sol.step_profiled(dt, args.profile_steps)
    nn = (p.N + 1) ** 3
    sb = 4
    elem_bytes = (4 * 4 * 5 * sb + 1 * 3 * 5 * sb) / 5.0 * p.nelem * nn   # U in, G in/out, U out (stage 0: no G in)
    elem_ms = kms[2] / kcnt[2]
    iface_bytes = 20 * (p.N + 1) ** 2 * sb * p.n_faces
    iface_ms = kms[1] / kcnt[1]
    peaks, peak_kind = measured_peaks()
    hbm = float(peaks["hbm_gbs"])
    achieved = elem_bytes / (elem_ms * 1e-3) / 1e9
    traffic = ncu_traffic(p.nelem)

    # FP64 plain path, same workload, one solve
    p64 = synth.config_interface_heavy(seed=1 + rank, precision=synth.FP64, nz=args.nz)
    p64.volume, p64.riemann = p.volume, p.riemann
    s64 = slidemesh.Solver(p64)
    s64.init_state()
    s64.step(dt, 1)
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    s64.step(dt, args.fp64_steps)
    f1.record(stream)
    torch.cuda.synchronize()
    ms64 = max_over_ranks(f0.elapsed_time(f1))
    value64 = world * p64.ndof * 5 * args.fp64_steps / (ms64 * 1e-3)
    flop_alg = algorithmic_flop_per_dof(p64.N, p64.n_faces, p64.ndof)
    gflops64 = value64 / world * flop_alg / 1e9
    gflops64_exec = value64 / world * FP64_EXECUTED_FLOP_PER_DOF / 1e9
    s64.close()
    del s64
    fpk = fp64_fma_peak(stream)

    # the split-form volume integral with Roe/HH (the paper's scheme), same workload, FP32
    split = None
    if args.volume == "weak" and args.split_steps > 0:
        ps = synth.config_interface_heavy(seed=1 + rank, precision=synth.FP32, nz=args.nz)
        ps.volume, ps.riemann = synth.VOLUME_SPLIT, synth.ROE_HH
        ss = slidemesh.Solver(ps)
        ss.init_state()
        ss.step(dt, 3)
        torch.cuda.synchronize()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        ss.step(dt, args.split_steps)
        g1.record(stream)
        torch.cuda.synchronize()
        mss = max_over_ranks(g0.elapsed_time(g1))
        skms, skcnt = ss.step_profiled(dt, max(2, args.profile_steps // 2))
        sel_ms = skms[2] / skcnt[2]
        sach = elem_bytes / (sel_ms * 1e-3) / 1e9
        split = {"value": rep.value(ps.ndof * 5 * args.split_steps, mss * 1e-3), "unit": UNIT,
                 "steps": args.split_steps, "ms_per_step": mss / args.split_steps,
                 "volume": "split form, Pirozzoli two-point flux", "riemann": "roe_hh",
                 "roofline": {"bound": "hbm", "achieved": sach, "peak": hbm, "unit": "GB/s", "frac": sach / hbm,
                              "kernel": "dg_element_split_kernel<N=5, float, Roe/HH, stage>",
                              "peak_source": peak_kind, "algorithmic_bytes_per_launch": elem_bytes,
                              "avg_launch_ms": sel_ms},
                 "kernels": {"stage_params": {"launches": skcnt[0], "ms": skms[0]},
                             "sliding_interface": {"launches": skcnt[1], "ms": skms[1]},
                             "dg_element_split": {"launches": skcnt[2], "ms": skms[2], "avg_ms": sel_ms}},
                 "diag_finite": ss.diag()["status"] == 0}
        ss.close()
        del ss

    # two sliding interfaces: the same workload closed in x (periodic x), so the moving block's
    # face x2 meets the static face x0 as well: 2 x 65,536 interface face pairs per stage
    two = None
    if args.volume == "weak" and args.two_steps > 0:
        pp = synth.config_interface_heavy(seed=1 + rank, precision=synth.FP32, nz=args.nz)
        pp.periodic_x = 1
        s2 = slidemesh.Solver(pp)
        s2.init_state()
        s2.step(dt, 3)
        torch.cuda.synchronize()
        h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        h0.record(stream)
        s2.step(dt, args.two_steps)
        h1.record(stream)
        torch.cuda.synchronize()
        ms2 = max_over_ranks(h0.elapsed_time(h1))
        tkms, tkcnt = s2.step_profiled(dt, max(2, args.profile_steps // 2))
        if_ms = tkms[1] / tkcnt[1] / 2.0
        two = {"value": rep.value(pp.ndof * 5 * args.two_steps, ms2 * 1e-3), "unit": UNIT,
               "interface_face_updates_per_s": rep.value(2 * pp.n_faces * 5 * args.two_steps, ms2 * 1e-3),
               "steps": args.two_steps, "ms_per_step": ms2 / args.two_steps,
               "interfaces": "x = x1 and x = x0 = x2 (periodic x), 2 x %d face pairs" % pp.n_faces,
               "kernels": {"stage_params": {"launches": tkcnt[0], "ms": tkms[0]},
                           "sliding_interface": {"launches": 2 * tkcnt[1], "ms": tkms[1], "avg_ms": if_ms,
                                                 "achieved_gbs": iface_bytes / (if_ms * 1e-3) / 1e9,
                                                 "frac_hbm": iface_bytes / (if_ms * 1e-3) / 1e9 / hbm},
                           "dg_element": {"launches": tkcnt[2], "ms": tkms[2], "avg_ms": tkms[2] / tkcnt[2]}},
               "diag_finite": s2.diag()["status"] == 0}
        s2.close()
        del s2

    # end to end through the C-ABI with host buffers: every step is a job streamed from pinned
    # host memory (state in, one RK step, state out) by sm_stream_jobs, whose copies in and out
    # overlap the neighbouring jobs' steps
    Uh, _ = sol.get_state(out=torch.empty(sol.shape(), dtype=torch.float32, pin_memory=True))
    Uo = torch.empty_like(Uh).pin_memory()
    sol.stream_jobs(Uh, Uo, d["t"], dt, 1, count=1)          # staging buffers, copy streams
    barrier()
    t0 = time.perf_counter()
    sol.stream_jobs(Uh, Uo, d["t"], dt, 1, count=args.e2e_steps)
    torch.cuda.synchronize()
    el = max_over_ranks(time.perf_counter() - t0)
    e2e = {"value": world * p.ndof * 5 * args.e2e_steps / el, "unit": UNIT,
           "h2d_bytes_per_step": Uh.numel() * 4, "d2h_bytes_per_step": Uo.numel() * 4,
           "steps": args.e2e_steps,
           "how": "sm_stream_jobs: per step the state in from pinned host memory, one RK step, the state out "
                  "to pinned host memory; the copies of the next and the previous step overlap the step"}

    if rank != 0:
        sol.close()
        if world > 1:
            dist.destroy_process_group()
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "repeats": repeats, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "elements": p.nelem, "N": p.N, "dof": p.ndof,
                   "sliding_faces_per_side": p.n_faces, "state_bytes": p.ndof * 5 * 4,
                   "riemann": "roe_hh" if riem == "roe" else "rusanov",
                   "volume": "split form, Pirozzoli two-point flux" if args.volume == "split" else "weak form",
                   "l2": "inputs %s L2 (%.2f GB state per buffer, L2 129 MB)" % (
                       "larger than" if p.ndof * 5 * 4 > 129e6 else "NOT larger than", p.ndof * 5 * 4 / 1e9),
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "dt": dt, "final_t": d["t"]},
        "interface_face_updates_per_s": face_rate,
        "fp64_plain": {"value": value64, "unit": UNIT, "steps": args.fp64_steps, "ms_per_step": ms64 / args.fp64_steps,
                       "fp32_over_fp64": value / value64,
                       "roofline": {"bound": "alu", "achieved": gflops64, "peak": fpk["gflops"], "unit": "GFLOP/s",
                                    "frac": gflops64 / fpk["gflops"],
                                    "flop_per_dof_update": flop_alg,
                                    "flop_count": "algorithmic: the method's operations, each conforming face once",
                                    "executed_flop_per_dof_update": FP64_EXECUTED_FLOP_PER_DOF,
                                    "achieved_executed": gflops64_exec, "frac_executed": gflops64_exec / fpk["gflops"],
                                    "peak_source": "measured", "peak_probe": fpk}},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                     "traffic": traffic if args.volume == "weak" and riem == "rusanov" else None,
                     "kernel": kname,
                     "peak_source": peak_kind, "algorithmic_bytes_per_launch": elem_bytes,
                     "avg_launch_ms": elem_ms},
        "kernels": {"stage_params": {"launches": kcnt[0], "ms": kms[0]},
                    "sliding_interface": {"launches": kcnt[1], "ms": kms[1], "avg_ms": iface_ms,
                                          "achieved_gbs": iface_bytes / (iface_ms * 1e-3) / 1e9,
                                          "frac_hbm": iface_bytes / (iface_ms * 1e-3) / 1e9 / hbm},
                    "dg_element": {"launches": kcnt[2], "ms": kms[2], "avg_ms": elem_ms}},
        "e2e": e2e,
        # per step: the five stages' parameters in one launch, then per stage the interface
        # kernel and the element kernel
        "gpu_launches": 11 * args.steps,
        "clocks": clk,
        "diag": {"n_delta": d["n_delta"], "s_delta": d["s_delta"], "finite": d["status"] == 0},
    }
    if split is not None:
        line["split_form"] = split
    if two is not None:
        line["two_interfaces"] = two
    if not args.no_cpu_baseline and world >= 1:
        line["cpu_baseline"] = cpu_baseline(args.cpu_seconds, p.volume, p.riemann)
    sol.close()
    if args.serve_steps > 0 and args.volume == "weak" and world == 1:
        line["serving"] = serving_results(args)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
