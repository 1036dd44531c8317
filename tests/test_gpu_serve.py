"""Serving loop on the GPU: every served result equals the same solve run
alone, although members join and leave the batch while others are mid-run;
a diverging solve is evicted without disturbing the others."""
import math

import numpy as np
import pytest

from paper_2609_24785_b300 import lee, serve, workloads

pytestmark = pytest.mark.gpu

H = workloads.H


def _mixed_cases(k=6):
    out = []
    for i in range(k):
        n = (96, 128, 80, 112, 64, 144)[i % 6]
        c = ((n - 1) / 2 * H, (n - 1) / 2 * H)
        if i % 2:
            wall = ("cyl", c[0], c[1], 0.12 * n * H)
            pos = (c[0] + 0.3 * n * H, c[1] + 0.05 * n * H)
        else:
            th = math.radians(10.0 * i)
            wall = ("line", c[0] + 0.37 * H, c[1], th)
            pos = (c[0] - 0.25 * n * H * math.sin(th), c[1] + 0.25 * n * H * math.cos(th))
        out.append(workloads.Case("mix%d" % i, n, n, wall=wall, imp=("msd", 0.5 + 0.3 * i, 0.02, 2.0 + i),
                                  init=("pulse", pos[0], pos[1], 1.0, 4 * H), probes=np.array([pos]),
                                  steps=150 + 97 * i,
                                  sponge=workloads.WALL_EDGE_SPONGE if i % 2 == 0 else workloads.LONG_RUN_SPONGE))
    return out


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_served_results_equal_solo_runs(precision, cuda_device):
    cases = _mixed_cases()
    be = serve.LeeBackend(precision)
    # two slots: a request joins whenever one leaves, while the other is mid-run
    srv = serve.Server(be, max_slots=2, chunk_ms=2.0, setup_workers=2)
    rep = srv.run([(0.0, c) for c in cases], realtime=False)
    assert all(r.status == "ok" for r in rep.requests), [(r.case.name, r.status, r.error) for r in rep.requests]
    reqs = sorted(rep.requests, key=lambda r: r.t_admit)
    # overlap: some request was admitted while an earlier one was still running
    assert any(b.t_admit < a.t_done and b.t_admit > a.t_admit for a in reqs for b in reqs)
    assert rep.chunks > len(cases)
    for r in rep.requests:
        solo = serve.solo_reference(r.case, precision)
        assert r.probes.shape == solo.shape == (r.case.steps, 1)
        # same kernels, same per-node arithmetic: identical, far inside the parity bar
        assert np.array_equal(r.probes, solo), r.case.name


def test_per_solve_fp64_path_matches(cuda_device):
    cases = _mixed_cases(3)
    be = serve.LeeBackend("fp64", batching=False)
    rep = serve.Server(be, max_slots=1, chunk_ms=5.0, setup_workers=1).run([(0.0, c) for c in cases], realtime=False)
    assert rep.peak_members == 1
    for r in rep.requests:
        assert r.status == "ok"
        assert np.array_equal(r.probes, serve.solo_reference(r.case, "fp64"))


def test_diverging_solve_is_evicted(cuda_device):
    cases = _mixed_cases(2)
    bad = workloads.Case("unstable", 96, 96, wall=cases[0].wall, imp=cases[0].imp, init=cases[0].init,
                         probes=cases[0].probes, steps=40000, cfl=1.9)   # far past the RK4/DRP limit
    be = serve.LeeBackend("fp32")
    rep = serve.Server(be, chunk_ms=2.0, setup_workers=1).run([(0.0, bad)] + [(0.0, c) for c in cases],
                                                               realtime=False)
    st = {r.case.name: r for r in rep.requests}
    # evicted at the end of the chunk in which it blew up, long before its 40000 steps
    assert st["unstable"].status == "diverged" and st["unstable"].steps_done < 40000
    for c in cases:
        r = st[c.name]
        assert r.status == "ok" and np.array_equal(r.probes, serve.solo_reference(c, "fp32"))


def test_solver_sync_reports_divergence(cuda_device):
    c = _mixed_cases(1)[0]
    s = lee.Solver(c.nx, c.ny, c.h, 1.9, precision="fp32")
    workloads.apply_to(c, s)
    s.plan()
    s.bind()
    workloads.apply_state(c, s)
    s.step(4000)
    with pytest.raises(lee.LeeError) as e:
        s.sync()
    assert e.value.code == lee.LEE_ERR_DIVERGED
