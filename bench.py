#!/usr/bin/env python3
"""Benchmark of the ghost-point IBM / ADE / LEE hot path on B300.

Default workload: the batched cylinder-pulse sweep -- 512 independent solves,
grid n^2 with n uniform in {256, 384, 512, 768, 1024}, cylinder radius 0.1 n,
R, M, K log-uniform in [0.2, 5] x [0.005, 0.2] x [0.5, 20] (seed 24785), FP32
field storage and stencils with FP64 ghost weights / ADE (ghost projections in
float-float on the FP32 pipe, about 48 significant bits), advanced together by
one ghost launch and one stencil launch per Runge-Kutta stage (CUDA graph).
A step is one time step (four stages) of every instance.  Metric: point-stage
updates per second (fluid nodes x 4 stages x steps / time).  The device
working set (~10 GB) is far larger than L2, so no flush is needed.

--workload cylinder times the single 1024^2 cylinder-pulse solve instead.

Serving (rank 0, unless --no-serve): the first --serve-duration seconds of a
Poisson stream (--serve-rate requests/s, seed 24786) of mixed solves (flat wall
at U[0, 60] deg or cylinder of radius U[0.05, 0.15] n; n in {256 ... 2048};
R/M/K as in the sweep; 1000-10000 steps) through the continuous-batching
server (FP32 bulk, 80 GB budget), then the same trace through the plain
per-solve FP64 path; p50/p99 latency (arrival -> result) and throughput.
--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (the reference arm).

Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mpoint-stage-updates/s"
UNIT = "Mpoint-stage/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="lee", choices=["lee", "reference"])
    ap.add_argument("--workload", default="sweep", choices=["sweep", "rational", "trace", "cylinder", "free", "flat", "monopole"])
    ap.add_argument("--count", type=int, default=512)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="skip the tile / packing autotuner")
    ap.add_argument("--tile", default=None, help="TMA tile WxH (skips the autotuner)")
    ap.add_argument("--strips", type=int, default=0, help="tile strips per SM with --tile (0: library default)")
    ap.add_argument("--fuse", type=int, default=0, help="temporal blocking of stages 1 and 2 (1: on)")
    ap.add_argument("--band-tile", type=int, default=-1,
                    help="stages (bit k) whose band nodes the stencil updates in its band tiles (-1: default)")
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-duration", type=float, default=1.0,
                    help="seconds of Poisson arrivals of the saturated serving trace")
    ap.add_argument("--serve-fp64", type=int, default=16,
                    help="serve the first N requests of the trace per solve in FP64 as well (0: skip)")
    ap.add_argument("--sustained-rate", type=float, default=3.0,
                    help="arrival rate of the sustainable serving trace (0: skip)")
    ap.add_argument("--sustained-duration", type=float, default=30.0)
    ap.add_argument("--serve-chunk-ms", type=float, default=40.0,
                    help="serving chunk length: members join and leave between chunks")
    return ap.parse_args()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def workload_cases(args, rank, accept=None):
    from paper_2609_24785_b300 import workloads
    if args.workload == "sweep":
        cases, rejected = workloads.sweep(args.count, seed=24785 + rank, accept=accept)
        desc = ("batched cylinder-pulse sweep: %d instances, n^2 with n in {256,384,512,768,1024}, "
                "cylinder r = 0.1 n, R/M/K log-uniform, seed %d" % (args.count, 24785 + rank))
        return cases, rejected, desc
    if args.workload == "rational":
        cases, rejected = workloads.rational_sweep(args.count, seed=24785 + rank, accept=accept)
        desc = ("batched cylinder-pulse sweep with broadband walls: %d instances, n^2 with n in "
                "{256,384,512,768,1024}, cylinder r = 0.1 n, two real poles + one complex pair "
                "(4 ADE states per ghost), seed %d" % (args.count, 24785 + rank))
        return cases, rejected, desc
    if args.workload == "trace":
        # the serving mix at steady state: the first second of the 200/s trace
        # as one batch, every request resident from the start
        trace = workloads.serving_trace(rate=200.0, duration=1.0, seed=24786 + rank, accept=accept)
        cases = [c for _, c in trace]
        desc = ("first 1 s of the 200/s serving trace as one static batch: %d instances, n in "
                "{256,...,2048}, half flat walls (ramp 12, 0.4), half cylinders (ramp 12, 0.04), seed %d"
                % (len(cases), 24786 + rank))
        return cases, 0, desc
    if args.workload == "free":
        # diagnostic: no wall, so every tile away from the outer band is interior
        cases = []
        for i in range(args.count if args.count != 512 else 128):
            c = workloads.cylinder_pulse(1024)
            c.name = "free_%d" % i
            c.wall, c.imp = ("none",), ("rigid",)
            cases.append(c)
        return cases, 0, "wall-free 1024^2 pulses, %d instances (diagnostic)" % len(cases)
    if args.workload == "flat":
        c = workloads.flat_wall(128)
        return [c], 0, "flat impedance wall 128^2 at 30 deg, R=1 M=0.05 K=5 (double pole), no ramp"
    if args.workload == "monopole":
        c = workloads.monopole(2048)
        return [c], 0, ("monopole-cylinder 2048^2, r = 100 cells, source at 300 cells, 20 points per wavelength, "
                        "R=1 M=0.1 K=10, 256-probe ring, ramp 12")
    c = workloads.cylinder_pulse(1024)
    return [c], 0, "cylinder pulse 1024^2, r = 50 cells, R=2 M=0.02 K=1, ramp 12"


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.p = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(device_index)],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
            out, _ = self.p.communicate()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate_over_ranks(ms, fluid, device):
    """Replicas (one process per GPU, independent instances, no collective on
    the data path): the job's time is the slowest rank's, its work the sum of
    every rank's fluid nodes.  device: where the process group's tensors live
    (the rank's GPU for NCCL, the CPU for gloo)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    f = torch.tensor([float(fluid)], dtype=torch.float64, device=device)
    dist.all_reduce(f)
    return float(t.item()), float(f.item())


def cpu_baseline(case, target_seconds=15.0):
    """The FP64 oracle as it stands, on one instance of the workload, on all host
    cores (OpenMP); runs a bounded number of steps."""
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from _helpers import make_oracle
    o = make_oracle(case)
    fluid = int((o.kind() == 1).sum())
    t = time.perf_counter()
    o.run(2)
    dt1 = (time.perf_counter() - t) / 2
    n = max(2, min(2000, int(target_seconds / max(dt1, 1e-6))))
    t = time.perf_counter()
    o.run(n)
    el = time.perf_counter() - t
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": fluid * 4 * n / el / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%s (%d fluid nodes), %d steps, %.1f s" % (case.name, fluid, n, el)}


def cpu_baseline_one_core(case_index, target_seconds=10.0):
    """The same oracle on one host thread (a child process with
    OMP_NUM_THREADS=1, so that the parent's OpenMP pool is untouched)."""
    code = (
        "import sys, json; sys.path.insert(0, %r)\n"
        "import bench\n"
        "from paper_2609_24785_b300 import workloads\n"
        "cases, _ = workloads.sweep(512, seed=24785)\n"
        "print(json.dumps(bench.cpu_baseline(cases[%d], %r)))\n" % (ROOT, case_index, target_seconds))
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                             timeout=10 * target_seconds + 60)
        return json.loads(out.stdout.strip().splitlines()[-1])
    except (subprocess.SubprocessError, ValueError, IndexError) as e:
        return {"error": str(e)[:200]}


def run_reference(args):
    ws, rank, local = dist_setup(args)
    if rank != 0:
        return
    from paper_2609_24785_b300 import workloads
    cases, _, desc = workload_cases(args, 0)
    case = min(cases, key=lambda c: c.points) if args.workload == "sweep" else workloads.cylinder_pulse(256)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from _helpers import make_oracle
    o = make_oracle(case)
    fluid = int((o.kind() == 1).sum())
    for _ in range(args.warmup):
        o.run(1)
    t = time.perf_counter()
    for _ in range(args.steps):
        o.run(1)
    el = time.perf_counter() - t
    v = fluid * 4 * args.steps / el / 1e6
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    sample = "%s (%d fluid nodes), one time step per bench step" % (case.name, fluid)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": desc, "sample": sample},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_serving(args):
    """Serving trace through the continuous-batching server (FP32) and, for
    comparison, through the per-solve FP64 path."""
    from paper_2609_24785_b300 import lee, serve, workloads
    rejected = [0]

    def accept(case):
        s = lee.Solver(case.nx, case.ny, case.h, case.cfl, precision="fp32")
        workloads.apply_to(case, s)
        try:
            s.plan()
            return True
        except lee.LeeError:
            rejected[0] += 1
            return False
    def describe(trace, rate, duration, redrawn):
        sizes = sorted({c.nx for _, c in trace})
        flat = sum(1 for _, c in trace if c.wall[0] == "line")
        return ("Poisson %.0f/s for %.3f s (seed 24786): %d requests (%d flat walls, %d cylinders), n in %s, "
                "%d-%d steps, %d draws redrawn (set-up rejected: unstable ADE), absorbing ramp %s (flat walls %s)" %
                (rate, duration, len(trace), flat, len(trace) - flat, sizes, min(c.steps for _, c in trace),
                 max(c.steps for _, c in trace), redrawn, workloads.LONG_RUN_SPONGE, workloads.WALL_EDGE_SPONGE))
    trace = workloads.serving_trace(rate=args.serve_rate, duration=args.serve_duration, accept=accept)
    out = {"trace": describe(trace, args.serve_rate, args.serve_duration, rejected[0]),
           "budget_bytes": 80 * 10**9}
    rep = serve.Server(serve.LeeBackend("fp32"), budget_bytes=80 * 10**9, chunk_ms=args.serve_chunk_ms).run(
        trace, realtime=True)
    out["chunk_ms"] = args.serve_chunk_ms
    out["fp32_batched"] = rep.summary()
    if args.serve_fp64:
        sub = trace[:args.serve_fp64]
        rep32 = serve.Server(serve.LeeBackend("fp32"), budget_bytes=80 * 10**9,
                             chunk_ms=args.serve_chunk_ms).run(sub, realtime=True)
        rep64 = serve.Server(serve.LeeBackend("fp64", batching=False), max_slots=1,
                             budget_bytes=80 * 10**9).run(sub, realtime=True)
        out["subset"] = "first %d requests of the trace, served alone in both modes" % len(sub)
        out["subset_fp32_batched"] = rep32.summary()
        out["subset_fp64_per_solve"] = rep64.summary()
    if args.sustained_rate > 0:
        rejected[0] = 0
        tr = workloads.serving_trace(rate=args.sustained_rate, duration=args.sustained_duration, seed=24787,
                                     accept=accept)
        rep = serve.Server(serve.LeeBackend("fp32"), budget_bytes=80 * 10**9,
                           chunk_ms=args.serve_chunk_ms).run(tr, realtime=True)
        out["sustained_trace"] = describe(tr, args.sustained_rate, args.sustained_duration, rejected[0])
        out["sustained_fp32_batched"] = rep.summary()
    return out


def run_lee(args):
    import torch
    ws, rank, local = dist_setup(args)
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    from paper_2609_24785_b300 import lee, workloads
    lee.load()

    def accept(case):
        s = lee.Solver(case.nx, case.ny, case.h, case.cfl, precision=args.precision)
        workloads.apply_to(case, s)
        try:
            s.plan()
            return True
        except lee.LeeError as e:
            if e.code == lee.LEE_ERR_ADE_UNSTABLE:
                return False
            raise

    t_setup = time.perf_counter()
    cases, rejected, desc = workload_cases(args, rank, accept=accept)
    # tile shape and work packing: autotuned on a sample of the workload (FP32)
    tile, strips, tuned = None, 0, None
    if args.precision == "fp32":
        if args.tile:
            tile = tuple(int(x) for x in args.tile.split("x"))
            strips = args.strips
        elif not args.no_tune:
            from paper_2609_24785_b300 import autotune
            t_tune = time.perf_counter()
            res = autotune.tune(cases)
            tile, strips = res.tile, res.strips_per_sm
            tuned = res.as_dict()
            tuned["seconds"] = round(time.perf_counter() - t_tune, 2)
            torch.cuda.synchronize()
    stream = torch.cuda.Stream(device=dev)
    batch = lee.Batch(args.precision, stream=stream)
    solvers = []
    from concurrent.futures import ThreadPoolExecutor

    def plan(case):
        s = lee.Solver(case.nx, case.ny, case.h, case.cfl, precision=args.precision)
        workloads.apply_to(case, s)
        if tile:
            s.set_tile(*tile)
        if len(case.probes) and case.wall[0] != "none":
            s.set_probes(case.probes, 4096)
        s.plan()
        return s
    with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        solvers = list(ex.map(plan, cases))
    for case, s in zip(cases, solvers):
        s.bind(stream=stream)
        workloads.apply_state(case, s)
        batch.add(s)
    if strips:
        batch.set_strips_per_sm(strips)
    fused_tiles = None
    if args.fuse:
        batch.set_stage_fusion(True)
    if args.band_tile >= 0:
        batch.set_band_in_tile(args.band_tile)
        fused_tiles = batch.fused_tiles()
    t_setup = time.perf_counter() - t_setup
    fluid = sum(s.sizes.n_fluid for s in solvers)
    ghosts = sum(s.sizes.n_ghost for s in solvers)
    elem = 4 if args.precision == "fp32" else 8

    # warm-up (also captures the CUDA graphs)
    batch.step(args.warmup)
    torch.cuda.synchronize()

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    # ---- timed region: K steps of every instance, device time by CUDA events
    clocks = ClockSampler(local)
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    l0 = lee.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    batch.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = lee.launch_count() - l0
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    if ws > 1:
        ms, fluid_all = aggregate_over_ranks(ms, fluid, dev)
    else:
        fluid_all = float(fluid)
    value = fluid_all * 4 * args.steps / (ms / 1e3) / 1e6

    # ---- roofline of the dominant kernel (stencil, stage 2: reads Q(1) and
    # Q^n, writes Q(2): 9 words per fluid node), timed on the launching stream
    reps = 10
    for _ in range(2):
        batch.launch(2, 1)
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    for _ in range(reps):
        batch.launch(2, 1)
    a1.record(stream)
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    for _ in range(reps):
        batch.launch(2, 0)
    g1.record(stream)
    torch.cuda.synchronize()
    st_ms = a0.elapsed_time(a1) / reps
    gh_ms = g0.elapsed_time(g1) / reps
    alg_bytes = 9 * elem * fluid
    peak, peak_kind = peaks()
    achieved = alg_bytes / (st_ms / 1e3) / 1e9
    traffic = None
    kname = batch.stencil_kernel()
    if kname.startswith("stencil_ws"):
        kname += " + band in tile" if (batch.band_in_tile() >> 2) & 1 else " + band_kernel"
    kname += " stage 2"
    tf = os.path.join(ROOT, "profiles", "stencil_traffic.json")
    if os.path.exists(tf):
        try:
            d = json.load(open(tf))
            # counters of another kernel variant do not describe this one
            for e in d.get("entries", []):
                if (e.get("workload") == desc and e.get("precision") == args.precision and
                        e.get("kernel") == kname):
                    traffic = e.get("bytes_per_launch")
        except (ValueError, OSError):
            traffic = None

    # ---- FP64: the stencil is bound by the FP64 pipe, not by HBM.  Its rate of
    # FP64 instructions (32 per interior point-stage: four DRP derivatives of 7,
    # the divergence, three stage FMAs) against this GPU's FP64 FMA rate,
    # measured by a kernel of independent FMA chains on the same stream.
    roofline_fp64 = None
    if args.precision == "fp64":
        sink = torch.zeros(1, dtype=torch.float64, device=dev)
        L = lee.load()
        blocks, iters = 148 * 8, 20000
        for _ in range(2):
            lee._check(L.lee_fp64_fma_probe(blocks, iters, sink.data_ptr(), stream.cuda_stream))
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(5):
            lee._check(L.lee_fp64_fma_probe(blocks, iters, sink.data_ptr(), stream.cuda_stream))
        f1.record(stream)
        torch.cuda.synchronize()
        fma_s = f0.elapsed_time(f1) / 5 / 1e3
        peak_instr = blocks * 256 * 8 * iters / fma_s / 1e9          # G FP64 FMA instructions / s
        instr = 32.0 * fluid / (st_ms / 1e3) / 1e9
        roofline_fp64 = {"bound": "alu", "achieved": instr, "peak": peak_instr, "unit": "G FP64 instr/s",
                         "frac": instr / peak_instr, "peak_kind": "measured (FP64 FMA probe kernel, this run)",
                         "peak_tflops": 2 * peak_instr / 1e3, "instr_per_point_stage": 32,
                         "kernel": kname, "launch_ms": st_ms}

    # ---- end to end through the C ABI with host buffers: every step uploads
    # every instance's state from pinned host memory, advances one step and
    # reads back the step's probe record
    e2e = None
    if not args.no_e2e:
        import ctypes as C
        blobs = [torch.from_numpy(s.read_state()).pin_memory() for s in solvers]
        # every member's probe record of the step, gathered on the device and
        # read back in one copy
        npv = batch.latest_probe_count()
        pr = torch.empty(max(npv, 1), dtype=torch.float64).pin_memory()
        h2d = sum(b.numel() for b in blobs)
        d2h = 8 * npv
        L = lee.load()
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for it in range(args.steps):
            for s, b in zip(solvers, blobs):
                lee._check(L.lee_upload_state_async(s.ctx, C.c_void_p(b.data_ptr())), s.ctx)
            batch.step(1)
            batch.read_latest_probes_async(pr.data_ptr())
            stream.synchronize()
        el = time.perf_counter() - t0
        barrier()
        if ws > 1:
            import torch.distributed as dist
            t = torch.tensor([el], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            el = float(t.item())
        e2e = {"value": fluid_all * 4 * args.steps / el / 1e6, "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "what": "per step: state of every instance H2D from pinned host memory, one step, probe record D2H"}

    serving = None
    if rank == 0 and not args.no_serve:
        serving = run_serving(args)

    cpu = None
    if rank == 0 and not args.no_cpu:
        small = min(cases, key=lambda c: c.points)
        cpu = cpu_baseline(small)
        if args.workload == "sweep" and args.count == 512 and rank == 0:
            cpu["one_core"] = cpu_baseline_one_core(cases.index(small))

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f64",
            "data": "synthetic",
            "config": {"workload": desc, "instances": len(cases), "rejected_unstable_draws": rejected,
                       "fluid_nodes": int(fluid), "ghost_points": int(ghosts),
                       "ghost_dtype": ("float-float (FP64 weights as FP32 pairs), f64 ADE"
                                       if args.precision == "fp32" and os.environ.get("LEE_GHOST_ARITH") != "f64"
                                       else "f64"), "l2": "working set %.1f GB >> 126 MB L2, no flush" %
                       (sum(s.sizes.device_bytes for s in solvers) / 1e9),
                       "parallelism": "replicas" if ws > 1 else "single GPU", "setup_s": round(t_setup, 2),
                       "stencil_kernel": batch.stencil_kernel(), "autotune": tuned,
                       "fused_stage12_tiles": fused_tiles, "band_in_tile_stages": batch.band_in_tile()},
            "roofline_fp64": roofline_fp64,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": kname,
                         "launch_ms": st_ms, "alg_bytes_per_launch": int(alg_bytes),
                         "peak_kind": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else peak_kind},
            "ghost_kernel_ms": gh_ms,
            "gpu_launches": int(launches),
            "clocks": clk,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "serving": serving,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_lee(args)


if __name__ == "__main__":
    main()
