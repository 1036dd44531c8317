"""Autotuner of the FP32 stencil's tile shape and work packing.

The tile shape (fixed per instance at plan time) trades the halo overhead of
a tile against the share of edge and wall tiles that need the general code;
the packing is the number of tile strips per SM dealt to the persistent
CTAs (load balance against L2 reuse of the halo rows down a strip).  Which one is
fastest depends on the mix of grid sizes and walls, so it is measured: a
size-stratified sample of the workload is planned and bound once per
candidate shape, and the stage-2 launch (stencil + band pass, the dominant
kernel) is timed with CUDA events for each packing.  The fastest
configuration per fluid node wins.  The sample must fill the GPU as the
whole workload does (a quarter of a 512-instance sweep does; 32 instances
do not), and the packing is relative to the SM count so that it carries
over from the sample to the whole workload."""
from __future__ import annotations

from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field
from typing import List, Sequence, Tuple

from . import lee, workloads

CANDIDATE_TILES: Tuple[Tuple[int, int], ...] = ((128, 28), (64, 60), (64, 40), (64, 32), (64, 24))
CANDIDATE_STRIPS: Tuple[int, ...] = (1, 2, 4, 8)     # tile strips per SM


@dataclass
class TuneResult:
    tile: Tuple[int, int]
    strips_per_sm: int
    ns_per_node: float                       # stage-2 launch time per fluid node of the sample
    table: List[dict] = field(default_factory=list)
    sample: int = 0
    fluid_nodes: int = 0

    def as_dict(self) -> dict:
        return {"tile": "%dx%d" % self.tile, "strips_per_sm": self.strips_per_sm, "ns_per_node": self.ns_per_node,
                "sample_instances": self.sample, "sample_fluid_nodes": self.fluid_nodes,
                "table": self.table}


def stratified_sample(cases: Sequence[workloads.Case], k: int) -> List[workloads.Case]:
    """k cases spread evenly over the workload sorted by grid size."""
    if k >= len(cases):
        return list(cases)
    order = sorted(cases, key=lambda c: c.nx * c.ny)
    return [order[int((i + 0.5) * len(order) / k)] for i in range(k)]


def _plan(case, precision, tile):
    s = lee.Solver(case.nx, case.ny, case.h, case.cfl, precision=precision,
                   periodic_x=case.periodic[0], periodic_y=case.periodic[1])
    workloads.apply_to(case, s)
    s.set_tile(*tile)
    s.plan()
    return s


def tune(cases: Sequence[workloads.Case], precision: str = "fp32", tiles=CANDIDATE_TILES,
         strips=CANDIDATE_STRIPS, sample: int = 128, reps: int = 10, workers: int = 8) -> TuneResult:
    import torch
    chosen = stratified_sample(cases, sample)
    table = []
    fluid = 0
    for tile in tiles:
        with ThreadPoolExecutor(max_workers=workers) as ex:
            solvers = list(ex.map(lambda c: _plan(c, precision, tile), chosen))
        stream = torch.cuda.Stream()
        batch = lee.Batch(precision, stream=stream)
        for c, s in zip(chosen, solvers):
            s.bind(stream=stream)
            workloads.apply_state(c, s)
            batch.add(s)
        fluid = sum(s.sizes.n_fluid for s in solvers)
        batch.step(1)                                    # graph capture, caches warm
        for k in strips:
            batch.set_strips_per_sm(k)
            for _ in range(2):
                batch.launch(2, 1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                batch.launch(2, 1)
            e1.record(stream)
            stream.synchronize()
            ms = e0.elapsed_time(e1) / reps
            table.append({"tile": "%dx%d" % tile, "strips_per_sm": k, "ms": ms, "ns_per_node": ms * 1e6 / fluid})
        del batch, solvers
    best = min(table, key=lambda r: r["ns_per_node"])
    tw, th = (int(x) for x in best["tile"].split("x"))
    return TuneResult((tw, th), best["strips_per_sm"], best["ns_per_node"], table, len(chosen), fluid)
