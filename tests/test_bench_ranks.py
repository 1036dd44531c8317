"""Host logic of bench.py's multi-GPU path (replicas): two gloo ranks on the
CPU.  Each rank draws its own sweep (seed 24785 + rank) of the same size and
size mix, and the job's figures are the slowest rank's time and the sum of
the ranks' fluid nodes; the reference arm runs on rank 0 alone."""
import os
import sys
import types

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        args = types.SimpleNamespace(workload="sweep", count=24)
        cases, rejected, desc = bench.workload_cases(args, rank)
        fluid = sum(c.nx * c.ny for c in cases)          # stands in for the fluid count
        ms = 10.0 + 5.0 * rank
        t, f = bench.aggregate_over_ranks(ms, fluid, torch.device("cpu"))
        out[rank] = (t, f, fluid, [(c.nx, c.ny, c.wall) for c in cases], desc)
    finally:
        dist.destroy_process_group()


def test_replicas_aggregate_over_two_gloo_ranks():
    world = 2
    port = 29500 + os.getpid() % 1000
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    (t0, f0, n0, c0, d0), (t1, f1, n1, c1, d1) = res[0], res[1]
    assert t0 == t1 == 15.0                      # the slowest rank's time
    assert f0 == f1 == float(n0 + n1)            # every rank's work
    assert len(c0) == len(c1) == 24
    assert c0 != c1                              # independent instances per rank
    assert "seed 24785" in d0 and "seed 24786" in d1
    assert sorted(set(x[0] for x in c0)) <= [256, 384, 512, 768, 1024]


def _reference_arm(env_rank):
    import json
    import subprocess
    env = dict(os.environ, RANK=str(env_rank), LOCAL_RANK=str(env_rank), WORLD_SIZE="2", OMP_NUM_THREADS="2")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "2", "--warmup", "1"], env=env, capture_output=True, text=True, timeout=300)
    lines = [json.loads(l) for l in p.stdout.splitlines() if l.startswith("{")]
    return p.returncode, lines


def test_reference_arm_runs_on_rank_zero_only():
    """bench.py --impl reference under torchrun: rank 0 times the oracle and
    prints the one JSON line (impl, cpu_baseline, e2e of the line's own
    metric); the other ranks exit 0 without work."""
    rc1, lines1 = _reference_arm(1)
    assert rc1 == 0 and lines1 == []
    rc0, lines0 = _reference_arm(0)
    assert rc0 == 0 and len(lines0) == 1
    line = lines0[0]
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"]
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
