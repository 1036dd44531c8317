"""Serving loop: solves arrive over time and share the GPU by continuous batching.

A request is one solve (geometry, impedance R/M/K, source, grid size, step
count).  Its life:

1. arrival -> host set-up on a worker thread: mask, ghost set, FP64 weight
   rows and ADE coefficients (Sec. 3.1-3.2; ``lee_plan``).  The C calls release
   the GIL, so set-ups overlap each other and the GPU work;
2. admission, first come first served, when a slot is free and its device
   footprint (field buffers, weights, probe history) fits the HBM budget; a
   request that does not fit lets later, smaller ones pass, at most
   ``max_bypass`` times;
3. bind + initial field on its own stream while the running chunk is on the
   GPU (its upload overlaps the others' stencil work);
4. between two chunks it joins the batch: every admitted solve advances by one
   ghost and one stencil launch per stage (``lee_batch_step``, CUDA graphs);
5. when its step count is reached (or its status word reports divergence) it
   leaves the batch between chunks, its probe history is read back and its
   memory returns to the budget.

Chunks are sized from the measured point-stage rate so that one chunk lasts
about ``chunk_ms`` (the admission granularity), and never run past the member
closest to completion.  Latency is arrival -> result on the host; the report
has p50/p99 beside the throughput.

The scheduler talks to a backend (``LeeBackend`` here; tests plug in a host-
only fake) so that its admission and batching logic is testable without a GPU.
"""
from __future__ import annotations

import collections
import concurrent.futures as cf
import math
import time
from dataclasses import dataclass, field
from typing import Callable, List, Optional, Sequence, Tuple

import numpy as np

from . import lee, workloads

STEPS_PER_GRAPH = 8          # the batch replays graphs of 8 steps


@dataclass
class Request:
    rid: int
    case: workloads.Case
    arrival: float                   # seconds after the start of the trace
    steps: int = 0
    points: int = 0                  # fluid nodes (after set-up)
    footprint: int = 0               # device bytes (after set-up)
    t_setup: float = math.nan        # set-up finished
    t_admit: float = math.nan        # bound on the device
    t_done: float = math.nan         # result on the host
    steps_done: int = 0
    status: str = "pending"          # pending | ok | diverged | failed
    error: str = ""
    probes: Optional[np.ndarray] = None
    handle: object = None
    bypassed: int = 0

    @property
    def latency(self) -> float:
        return self.t_done - self.arrival


@dataclass
class Report:
    requests: List[Request]
    makespan: float                  # first arrival -> last result (s)
    point_stages: float              # fluid nodes x 4 x steps over completed requests
    chunks: int
    peak_bytes: int
    peak_members: int
    busy: float = 0.0                # time with a chunk on the GPU (launch -> drained), s

    def latencies(self) -> np.ndarray:
        return np.array([r.latency for r in self.requests if r.status == "ok"])

    def summary(self) -> dict:
        lat = self.latencies()
        ok = [r for r in self.requests if r.status == "ok"]
        q = (lambda p: float(np.percentile(lat, p))) if lat.size else (lambda p: math.nan)
        return {
            "requests": len(self.requests),
            "completed": len(ok),
            "diverged": sum(r.status == "diverged" for r in self.requests),
            # which walls diverged: (flat walls, cylinders), and the angles of
            # the flat walls that did (a straight wall meets the outer band)
            "diverged_flat_cyl": [sum(r.status == "diverged" and r.case.wall[0] == kind for r in self.requests)
                                  for kind in ("line", "cyl")],
            "diverged_flat_angles_deg": sorted(round(math.degrees(r.case.wall[3]), 1) for r in self.requests
                                               if r.status == "diverged" and r.case.wall[0] == "line"),
            # per diverged request: wall, n, angle (deg) or radius (cells), R, M, K, steps done / asked
            "diverged_cases": [(r.case.wall[0], r.case.nx,
                                round(math.degrees(r.case.wall[3]) if r.case.wall[0] == "line"
                                      else r.case.wall[3] / r.case.h, 2),
                                *(round(v, 4) for v in r.case.imp[1:4]), r.steps_done, r.case.steps)
                               for r in self.requests if r.status == "diverged" and r.case.imp[0] == "msd"],
            "failed": sum(r.status == "failed" for r in self.requests),
            "p50_s": q(50), "p99_s": q(99), "mean_s": float(lat.mean()) if lat.size else math.nan,
            "mean_wait_s": float(np.mean([r.t_admit - r.arrival for r in ok])) if ok else math.nan,
            "makespan_s": self.makespan,
            "mpoint_stage_per_s": self.point_stages / self.makespan / 1e6 if self.makespan > 0 else math.nan,
            "requests_per_s": len(ok) / self.makespan if self.makespan > 0 else math.nan,
            "chunks": self.chunks,
            # the share of the makespan with a chunk in flight, and the rate
            # over that time alone (idle gaps, set-up waits and the tail of
            # the trace excluded)
            "busy_s": self.busy,
            "busy_share": self.busy / self.makespan if self.makespan > 0 else math.nan,
            "mpoint_stage_per_busy_s": self.point_stages / self.busy / 1e6 if self.busy > 0 else math.nan,
            "peak_device_bytes": self.peak_bytes,
            "peak_members": self.peak_members,
        }


class LeeBackend:
    """Solves on the GPU through the C ABI (Solver per request, one Batch)."""

    def __init__(self, precision: str = "fp32", batching: bool = True):
        import torch
        self.precision = precision
        self.batching = batching
        self.setup_stream = torch.cuda.Stream()
        self.batch = lee.Batch(precision) if batching else None
        self.members: List[Request] = []

    # host, worker thread
    def setup(self, req: Request):
        c = req.case
        s = lee.Solver(c.nx, c.ny, c.h, c.cfl, precision=self.precision,
                       periodic_x=c.periodic[0], periodic_y=c.periodic[1])
        workloads.apply_to(c, s)
        if len(c.probes):
            s.set_probes(c.probes, max(c.steps, 1))
        sz = s.plan()
        return s, int(sz.device_bytes), int(sz.n_fluid)

    # main thread; may overlap a running chunk (own stream, new memory)
    def bind(self, req: Request):
        s = req.handle
        s.bind(stream=self.setup_stream)
        workloads.apply_state(req.case, s)

    def join(self, reqs: Sequence[Request]):
        for r in reqs:
            if self.batching:
                self.batch.add(r.handle)
            self.members.append(r)

    def leave(self, reqs: Sequence[Request]):
        for r in reqs:
            if self.batching:
                self.batch.remove(r.handle)
            self.members.remove(r)

    def launch(self, nsteps: int):
        if self.batching:
            self.batch.step(nsteps)
        else:
            for r in self.members:
                r.handle.step(nsteps)

    def done(self) -> bool:
        if self.batching:
            return self.batch.stream.query()
        return all(r.handle.stream.query() for r in self.members)

    def wait(self) -> List[int]:
        """Drain the chunk; status word per member (member order)."""
        if self.batching:
            return [int(x) for x in self.batch.status()]
        out = []
        for r in self.members:
            try:
                r.handle.sync()
                out.append(0)
            except lee.LeeError as e:
                out.append(lee.STATUS_DIVERGED if e.code == lee.LEE_ERR_DIVERGED else lee.STATUS_TIMEOUT)
        return out

    def result(self, req: Request) -> np.ndarray:
        return req.handle.probes()

    def release(self, req: Request):
        req.handle = None           # Solver.__del__ destroys the context; the arena returns to torch


class _InlineExecutor:
    """Runs set-ups on the calling thread (setup_workers = 0): deterministic."""

    def submit(self, fn, *args):
        f = cf.Future()
        try:
            f.set_result(fn(*args))
        except Exception as e:                  # delivered through f.result()
            f.set_exception(e)
        return f

    def shutdown(self, wait=True):
        pass


class Server:
    """Continuous-batching request loop over a backend (see the module doc)."""

    def __init__(self, backend, budget_bytes: int = 80 * 10**9, max_slots: int = 512, chunk_ms: float = 40.0,
                 setup_workers: int = 4, max_bypass: int = 8, clock: Callable[[], float] = time.perf_counter,
                 sleep: Callable[[float], None] = time.sleep, rate_guess: float = 5e10):
        self.be = backend
        self.budget = int(budget_bytes)
        self.max_slots = int(max_slots)
        self.chunk_ms = float(chunk_ms)
        self.setup_workers = int(setup_workers)
        self.max_bypass = int(max_bypass)
        self.clock = clock
        self.sleep = sleep
        self.rate = float(rate_guess)            # point-stages per second, updated per chunk

    # ---- policy pieces (pure functions of the state; unit-tested on the host)
    def chunk_steps(self, members: Sequence[Request]) -> int:
        """Steps of the next chunk: about chunk_ms at the measured rate, a
        multiple of the graph length when that is possible, and never past the
        member closest to its step count."""
        left = min(r.steps - r.steps_done for r in members)
        pts = sum(r.points for r in members)
        want = max(1, int(self.chunk_ms * 1e-3 * self.rate / (4.0 * max(pts, 1))))
        if want >= STEPS_PER_GRAPH:
            want -= want % STEPS_PER_GRAPH
        return max(1, min(left, want))

    def pick_admissions(self, ready: "collections.deque[Request]", used: int, nmembers: int) -> List[Request]:
        """First come first served under the slot and byte limits; a request
        that does not fit lets later ones pass at most max_bypass times, then
        blocks the queue until memory frees up."""
        out, blocked = [], []
        for r in ready:
            if nmembers + len(out) >= self.max_slots:
                break
            if used + r.footprint <= self.budget:
                out.append(r)
                used += r.footprint
                for b in blocked:                 # r overtook them
                    b.bypassed += 1
                continue
            blocked.append(r)
            if r.bypassed >= self.max_bypass:
                break
        return out

    # ---- the loop
    def run(self, trace: Sequence[Tuple[float, workloads.Case]], realtime: bool = True) -> Report:
        reqs = [Request(i, c, float(t), steps=int(c.steps)) for i, (t, c) in enumerate(sorted(trace, key=lambda x: x[0]))]
        pending = collections.deque(reqs)
        ready: "collections.deque[Request]" = collections.deque()
        staged: List[Request] = []               # bound, joining at the next chunk boundary
        members: List[Request] = []
        futures = {}
        used = peak = 0
        peak_members = chunks = 0
        point_stages = busy = 0.0
        t0 = self.clock()
        now = lambda: self.clock() - t0
        pool = cf.ThreadPoolExecutor(max_workers=self.setup_workers) if self.setup_workers > 0 else _InlineExecutor()

        def host_work():
            nonlocal used, peak
            # arrivals -> set-up
            while pending and (not realtime or pending[0].arrival <= now()):
                r = pending.popleft()
                if not realtime:
                    r.arrival = now()
                futures[pool.submit(self.be.setup, r)] = r
            # finished set-ups -> ready (arrival order)
            done = [f for f in futures if f.done()]
            for f in sorted(done, key=lambda f: futures[f].rid):
                r = futures.pop(f)
                try:
                    r.handle, r.footprint, r.points = f.result()
                    r.t_setup = now()
                    if r.footprint > self.budget:
                        r.status, r.error, r.t_done = "failed", "footprint exceeds the HBM budget", now()
                        r.handle = None
                    else:
                        ready.append(r)
                except Exception as e:            # geometry / rank / unstable ADE: reported, not served
                    r.status, r.error, r.t_done = "failed", str(e), now()
            ready_sorted = collections.deque(sorted(ready, key=lambda r: r.rid))
            ready.clear()
            ready.extend(ready_sorted)
            # admission -> bind (own stream; overlaps the running chunk)
            for r in self.pick_admissions(ready, used, len(members) + len(staged)):
                ready.remove(r)
                try:
                    self.be.bind(r)
                except Exception as e:
                    r.status, r.error, r.t_done = "failed", str(e), now()
                    self.be.release(r)
                    continue
                r.t_admit = now()
                used += r.footprint
                peak = max(peak, used)
                staged.append(r)

        try:
            while any(r.status == "pending" for r in reqs):
                host_work()
                if staged:
                    self.be.join(staged)
                    members.extend(staged)
                    staged.clear()
                if not members:
                    # idle: wait for the next arrival or set-up
                    if pending and realtime and not futures and not ready:
                        self.sleep(max(0.0, min(pending[0].arrival - now(), 0.05)))
                    else:
                        self.sleep(0.0005)
                    continue
                peak_members = max(peak_members, len(members))
                n = self.chunk_steps(members)
                t_start = self.clock()
                self.be.launch(n)
                while not self.be.done():
                    host_work()
                    self.sleep(0.0002)
                status = self.be.wait()
                dt = self.clock() - t_start
                chunks += 1
                busy += dt
                work = 4.0 * n * sum(r.points for r in members)
                if dt > 0:
                    self.rate = 0.5 * self.rate + 0.5 * work / dt
                leaving = []
                for r, st in zip(list(members), status):
                    r.steps_done += n
                    if st & lee.STATUS_DIVERGED or st & lee.STATUS_TIMEOUT or r.steps_done >= r.steps:
                        leaving.append((r, st))
                if leaving:
                    self.be.leave([r for r, _ in leaving])
                    for r, st in leaving:
                        members.remove(r)
                        if st & lee.STATUS_DIVERGED:
                            r.status, r.error = "diverged", "non-finite ghost, ADE or probe value"
                        elif st & lee.STATUS_TIMEOUT:
                            r.status, r.error = "failed", "device wait timed out"
                        else:
                            r.probes = self.be.result(r)
                            r.status = "ok"
                            point_stages += 4.0 * r.points * r.steps
                        r.t_done = now()
                        used -= r.footprint
                        self.be.release(r)
        finally:
            pool.shutdown(wait=True)
        arrivals = [r.arrival for r in reqs]
        dones = [r.t_done for r in reqs if not math.isnan(r.t_done)]
        makespan = (max(dones) - min(arrivals)) if reqs and dones else 0.0
        return Report(reqs, makespan, point_stages, chunks, peak, peak_members, busy)


def solo_reference(case: workloads.Case, precision: str = "fp32") -> np.ndarray:
    """The same solve alone (own context, own stream, stepped in one call):
    the probe history a served request must reproduce."""
    s = lee.Solver(case.nx, case.ny, case.h, case.cfl, precision=precision,
                   periodic_x=case.periodic[0], periodic_y=case.periodic[1])
    workloads.apply_to(case, s)
    if len(case.probes):
        s.set_probes(case.probes, max(case.steps, 1))
    s.plan()
    s.bind()
    workloads.apply_state(case, s)
    s.step(case.steps)
    s.sync()
    return s.probes()
