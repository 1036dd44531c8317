"""CPU tests of the product's host side (no GPU): the C ABI library loads and
exports every symbol of include/lee.h; its FP64 set-up (mask, ghost set,
clouds, weight rows, ADE coefficients, probe stencils) agrees with the oracle;
argument and stability errors are reported with status codes."""
import ctypes as C
import math
import os
import re

import numpy as np
import pytest

import oracle
from paper_2609_24785_b300 import lee, workloads
from _helpers import make_solver

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_library_exports_every_declared_symbol():
    hdr = open(os.path.join(ROOT, "include", "lee.h")).read()
    names = set(re.findall(r"^\s*(?:const\s+)?[a-z_ ]+\*?\s*\**(lee_[a-z_0-9]+)\s*\(", hdr, re.M))
    assert len(names) >= 35
    lib = C.CDLL(lee.LIB_PATH)
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing
    assert set(lee.SIGNATURES) == names


def _compare_plan(case):
    s = make_solver(case, bind=False)
    o = oracle.Oracle(case.nx, case.ny, case.h, case.cfl, periodic_x=case.periodic[0], periodic_y=case.periodic[1])
    workloads.apply_to(case, o)
    o.setup()
    assert np.array_equal(s.mask(), o.kind())
    assert s.sizes.n_ghost == o.n_ghost
    assert s.sizes.n_reduced == o.n_reduced
    worst = 0.0
    for g in range(o.n_ghost):
        a, b = s.ghost(g), o.ghost(g)
        assert a["target"] == b["target"]
        assert a["m"] == b["m"]
        assert sorted(a["cloud"]) == sorted(b["cloud"])
        np.testing.assert_allclose(a["bp"], b["bp"], rtol=0, atol=1e-15)
        np.testing.assert_allclose(a["r"], b["r"], rtol=0, atol=1e-13)
        # the oracle's rows in the paper's form (Eq. ns-ghost), folded
        m, L = b["m"], b["L"]
        pos = {v: i for i, v in enumerate(b["cloud"])}
        perm = [pos[v] for v in a["cloud"]]
        ref = np.stack([L[0],
                        sum(-b["ct"][i] / b["ct"][0] * L[i] for i in range(1, m + 1)),
                        sum(-b["c"][i] / b["c"][0] * L[i] for i in range(1, m + 1)),
                        sum(b["ell"][i] * L[i] for i in range(m + 1))], 1)[perm]
        worst = max(worst, np.abs(a["w"] - ref).max() / np.abs(ref).max())
        kp, ku = case.h / b["ct"][0], 1.0 / b["c"][0]
        worst = max(worst, abs(a["kappa"][0] - kp) / abs(kp), abs(a["kappa"][1] - ku) / abs(ku))
    return worst, s, o


@pytest.mark.parametrize("case", [
    workloads.flat_wall(128),
    workloads.flat_wall(96, angle_deg=0.0),
    workloads.flat_wall(96, angle_deg=58.0),
    workloads.cylinder_pulse(256),
    workloads.cylinder_pulse(300, nx=300, ny=220),
    workloads.monopole(256, radius_cells=13.3, src_cells=40),
    # steep wall leaving the box: clouds on one line take the constant fit
    workloads.Case("steep_line", 48, 48, wall=("line", 23.87 * 0.01, 23.5 * 0.01, math.radians(35.0)),
                   imp=("msd", 1.0, 0.05, 5.0)),
    workloads.Case("steep_line_768", 768, 768, wall=("line", 3.8387, 3.835, 0.8203129105709946),
                   imp=("msd", 1.0, 0.05, 5.0)),
], ids=lambda c: c.name)
def test_plan_matches_oracle(case):
    worst, s, o = _compare_plan(case)
    assert worst < 1e-11, worst


def test_periodic_plan_matches_oracle():
    case = workloads.Case("periodic_flat", 120, 8, wall=("line", 100.5 * 0.01, 0.0, math.pi / 2),
                          imp=("msd", 0.2, 0.025, 40.0), periodic=(False, True))
    worst, s, o = _compare_plan(case)
    assert worst < 1e-11, worst


def test_ade_regimes_and_unstable_pole_rejected():
    base = workloads.flat_wall(64)
    for RMK, reg in (((1.0, 0.05, 5.0), 3), ((2.0, 0.02, 1.0), 2), ((1.0, 0.1, 10.0), 1)):
        case = workloads.flat_wall(64, R=RMK[0], M=RMK[1], K=RMK[2])
        s = make_solver(case, bind=False)
        assert s.sizes.regime == reg
        ro, A, b, c = oracle.ade_regime(*RMK)
        assert ro == reg
        assert abs(s.sizes.ade_amplification - oracle.ade_stability(*RMK, base.h * base.cfl)) < 1e-13
    # the literal reading h = 1 (dx = 1 length unit) puts cfg2's stiff pole
    # (-99.5) at z = -49.7: far outside the RK4 region
    s = lee.Solver(64, 64, 1.0)
    s.set_wall_line(31.5, 31.5, 0.5).set_impedance(2.0, 0.02, 1.0)
    with pytest.raises(lee.LeeError) as e:
        s.plan()
    assert e.value.code == lee.LEE_ERR_ADE_UNSTABLE
    assert oracle.ade_stability(2.0, 0.02, 1.0, 0.5) > 1.0


def test_argument_errors():
    with pytest.raises(lee.LeeError) as e:
        lee.Solver(4, 4, 0.01)
    assert e.value.code == lee.LEE_ERR_ARG
    s = lee.Solver(32, 32, 0.01)
    with pytest.raises(lee.LeeError) as e:
        s.set_impedance(-1.0, 0.1, 1.0)
    assert e.value.code == lee.LEE_ERR_ARG
    with pytest.raises(lee.LeeError) as e:
        s.set_wall_cylinder(0.15, 0.15, 0.02)   # radius 2 h < 3.5 h
        s.plan()
    assert e.value.code == lee.LEE_ERR_GEOMETRY
    s2 = lee.Solver(32, 32, 0.01)
    with pytest.raises(lee.LeeError):
        s2.step(1)                               # not bound


def test_batch_argument_errors():
    """Batch entry points reject bad arguments before any device work: band
    stage masks outside stages 2-4, missing outputs, an unbound batch."""
    L = lee.load()
    b = C.c_void_p()
    assert L.lee_batch_create(C.byref(b), 7) == lee.LEE_ERR_ARG
    assert L.lee_batch_create(C.byref(b), lee.LEE_FP32) == lee.LEE_OK
    try:
        for bad in (1, 2, 32, 64, -2):          # bit 1 = stage 1, bits past stage 4, below -1
            assert L.lee_batch_set_band_in_tile(b, bad) == lee.LEE_ERR_ARG
        for good in (0, 4, 28, -1):
            assert L.lee_batch_set_band_in_tile(b, good) == lee.LEE_OK
        m = C.c_int()
        assert L.lee_batch_band_in_tile(b, None) == lee.LEE_ERR_ARG
        assert L.lee_batch_band_in_tile(b, C.byref(m)) == lee.LEE_OK and m.value in (0, 4, 8, 12, 16, 20, 24, 28)
        n = C.c_longlong()
        assert L.lee_batch_read_latest_probes_async(b, None, None) == lee.LEE_ERR_ARG
        assert L.lee_batch_read_latest_probes_async(b, None, C.byref(n)) == lee.LEE_ERR_ARG   # not bound
        assert L.lee_batch_step(b, 1) == lee.LEE_ERR_ARG                                         # not bound
    finally:
        L.lee_batch_destroy(b)


def test_probe_stencils_match_oracle():
    case = workloads.cylinder_pulse(256)
    s = make_solver(case, bind=False)
    # probe weights are internal; check through the mask that the probe nodes
    # are fluid and through the oracle that the same probes are valid
    o = oracle.Oracle(case.nx, case.ny, case.h)
    workloads.apply_to(case, o)
    o.setup()
    assert o.set_probes(case.probes, 4) == 0


def test_tile_shape_selection():
    """lee_set_tile: supported shapes change the plan's tile count; other
    shapes, FP64 and periodic instances and calls after lee_plan are rejected."""
    case = workloads.cylinder_pulse(256)
    for tw, th in ((128, 28), (64, 60), (64, 24)):
        s = lee.Solver(case.nx, case.ny, case.h, case.cfl, precision="fp32")
        workloads.apply_to(case, s)
        s.set_tile(tw, th)
        assert s.plan().n_tiles == -(-case.nx // tw) * -(-case.ny // th)
        with pytest.raises(lee.LeeError):
            s.set_tile(64, 60)                                 # after lee_plan
    s = lee.Solver(case.nx, case.ny, case.h, case.cfl, precision="fp32")
    with pytest.raises(lee.LeeError):
        s.set_tile(100, 28)
    s.set_tile(0, 0)                                           # back to the default
    s64 = lee.Solver(case.nx, case.ny, case.h, case.cfl, precision="fp64")
    with pytest.raises(lee.LeeError):
        s64.set_tile(128, 28)
    sp = lee.Solver(case.nx, case.ny, case.h, case.cfl, precision="fp32", periodic_y=True)
    with pytest.raises(lee.LeeError):
        sp.set_tile(128, 28)


@pytest.mark.parametrize("wall", [("line", 30.0), ("line", 75.0), ("cyl", 0.12)], ids=["line30", "line75", "cyl"])
def test_tile_flags_follow_the_mask(wall):
    """lee_tile_flags: every class bit of every 64 x 40 tile of a ragged
    200 x 136 grid (ramp of 12 layers) restated from the node kinds and the
    tile's rectangle: band (meets the three outer layers), mixed (a non-fluid
    or out-of-grid output), ramp, band windows all fluid, inert (every node
    solid and none a ghost)."""
    h = workloads.H
    nx, ny, W = 200, 136, 12
    cx, cy = (nx - 1) / 2 * h, (ny - 1) / 2 * h
    geo = ("line", cx + 0.37 * h, cy, math.radians(wall[1])) if wall[0] == "line" else ("cyl", cx, cy, wall[1] * nx * h)
    case = workloads.Case("flags", nx, ny, wall=geo, imp=("msd", 1.0, 0.05, 5.0), sponge=(W, 0.04))
    s = lee.Solver(nx, ny, h, case.cfl, precision="fp32")
    workloads.apply_to(case, s)
    s.set_tile(64, 40)
    s.plan()
    kind = s.mask()
    got = s.tile_flags()
    assert got.shape == (-(-ny // 40), -(-nx // 64))
    assert (got & 32).any() or wall[0] == "cyl"          # straight walls leave whole tiles solid
    for ty in range(got.shape[0]):
        for tx in range(got.shape[1]):
            xa, ya = 64 * tx, 40 * ty
            xb, yb = xa + 64, ya + 40
            k = kind[ya:min(yb, ny), xa:min(xb, nx)]
            band = xa < 3 or xb > nx - 3 or ya < 3 or yb > ny - 3
            f = (1 if band else 0) | (2 if (xb > nx or yb > ny or (k != 1).any()) else 0)
            f |= 4 if (xa < W or xb > nx - W or ya < W or yb > ny - W) else 0
            if band:
                ok = True
                for j in range(ya, min(yb, ny)):
                    for i in range(xa, min(xb, nx)):
                        if not (j < 3 or j > ny - 4 or i < 3 or i > nx - 4):
                            continue
                        sx, sy = min(max(i - 3, 0), nx - 7), min(max(j - 3, 0), ny - 7)
                        ok = ok and (kind[j, sx:sx + 7] == 1).all() and (kind[sy:sy + 7, i] == 1).all()
                f |= 8 if ok else 0
            f |= 32 if (k == 0).all() else 0
            assert int(got[ty, tx]) == f, (tx, ty, int(got[ty, tx]), f)


def test_autotune_sample_is_size_stratified():
    from paper_2609_24785_b300 import autotune
    cases, _ = workloads.sweep(60, seed=7)
    pick = autotune.stratified_sample(cases, 10)
    sizes = sorted(c.nx for c in pick)
    all_sizes = sorted(c.nx for c in cases)
    assert len(pick) == 10 and sizes[0] == all_sizes[3] and sizes[-1] == all_sizes[57]
    assert autotune.stratified_sample(cases[:5], 10) == cases[:5]


def test_rational_admittance_plan():
    """lee_plan of a rational wall (Sec. 2.3): one state per real pole and two
    per pair, regime 4, the RK4 amplification max |P(pole dt)| over every pole
    (computed here from the stability polynomial), and LEE_ERR_ADE_UNSTABLE
    when a real pole times dt leaves the RK4 interval (about -2.785)."""
    import math
    import numpy as np
    from paper_2609_24785_b300 import lee, workloads
    case = workloads.flat_wall(64)
    real = [(-20.0, 5.0), (-200.0, 30.0)]
    pairs = [(-4.0, 39.8, 20.0, 2.0)]
    s = lee.Solver(case.nx, case.ny, case.h, case.cfl, precision="fp64")
    workloads.apply_to(case, s)
    s.set_impedance_rational(real, pairs)
    sz = s.plan()
    assert s.sizes.n_states == 4 and s.sizes.regime == 4
    dt = case.cfl * case.h
    P = lambda z: 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24          # noqa: E731
    amp = max([abs(P(l * dt)) for l, _ in real] + [abs(P(complex(a, b) * dt)) for a, b, _, _ in pairs])
    assert abs(s.sizes.ade_amplification - amp) < 1e-12
    bad = lee.Solver(case.nx, case.ny, case.h, case.cfl, precision="fp64")
    workloads.apply_to(case, bad)
    bad.set_impedance_rational([(-3.0 / dt, 1.0)], [])
    with pytest.raises(lee.LeeError) as e:
        bad.plan()
    assert e.value.code == lee.LEE_ERR_ADE_UNSTABLE
    with pytest.raises(lee.LeeError):
        lee.Solver(case.nx, case.ny, case.h, case.cfl).set_impedance_rational([(1.0, 1.0)], [])
    with pytest.raises(lee.LeeError):
        lee.Solver(case.nx, case.ny, case.h, case.cfl).set_impedance_rational([(-1.0, 1.0)] * 9, [])
