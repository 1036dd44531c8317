"""Seeded synthetic workloads (input recipes only, none of the method's
arithmetic).  Shared by the tests, the benchmark and the oracle side.

Units: grid spacing h = 0.01 in the impedance's length unit (one unit = 100
cells), c0 = rho0 = 1, dt = cfl h.  Positions and widths given in cells are
multiplied by h.  A ``Case`` describes one solve; ``apply_to(case, target)``
calls the generic setter names that both the product binding (``lee.Solver``)
and the oracle wrapper expose.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, List, Optional, Tuple

import numpy as np

H = 0.01
CFL = 0.5
# Opt-in absorbing ramp (width in cells, kappa) of the workloads that run
# thousands of steps (cylinder pulse, sweep, serving, monopole): the outer
# one-sided/radiation closure has slowly growing grid-scale modes that amplify
# rounding (a 1e-16 difference reaches 3e-11 in 3000 steps on the 1024^2
# cylinder, FP32 rounding 5e-3), and this ramp damps them.  The paper adds no
# damping; the flat-wall workload (400 steps) and the short parity cases run
# without it.
LONG_RUN_SPONGE = (12, 0.04)
# The same ramp ten times stronger for straight walls that meet the outer band
# and run thousands of steps (serving): it removes the growing modes of the
# edge nodes next to the wall that the weaker ramp leaves (spectral study).
WALL_EDGE_SPONGE = (12, 0.4)


@dataclass
class Case:
    name: str
    nx: int
    ny: int
    h: float = H
    cfl: float = CFL
    wall: Tuple = ("none",)            # ("line", xw, yw, angle) | ("cyl", xc, yc, r) | ("none",)
    imp: Tuple = ("rigid",)            # ("rigid",) | ("msd", R, M, K) | ("rational", [(lam, A)], [(al, be, B, C)])
    init: Tuple = ("zero",)            # ("pulse", xs, ys, amp, w) | ("packet", xs, ys, ang, amp, k, alpha)
    source: Optional[Tuple] = None     # ("monopole", xs, ys, amp, w, omega)
    probes: np.ndarray = field(default_factory=lambda: np.zeros((0, 2)))
    steps: int = 100
    periodic: Tuple[bool, bool] = (False, False)
    sponge: Tuple[int, float] = (0, 0.0)   # opt-in absorbing ramp (width in cells, kappa); off

    @property
    def centre(self):
        return ((self.nx - 1) / 2 * self.h, (self.ny - 1) / 2 * self.h)

    @property
    def points(self):
        return self.nx * self.ny


def flat_wall(n=128, angle_deg=30.0, steps=400, R=1.0, M=0.05, K=5.0, rigid=False) -> Case:
    """Inclined impedance wall through the centre, Gaussian pulse 20 cells off
    the wall on the fluid side (half-width 3 cells, amplitude 1e-3); probes on
    the normal through the pulse centre, 2..16 cells from the wall."""
    c = ((n - 1) / 2 * H, (n - 1) / 2 * H)
    th = math.radians(angle_deg)
    nrm = np.array([-math.sin(th), math.cos(th)])
    src = np.array(c) + 20 * H * nrm
    probes = np.array([np.array(c) + d * H * nrm for d in (2, 4, 6, 8, 10, 12, 14, 16)])
    return Case("flat_wall_%d" % n, n, n, wall=("line", c[0], c[1], th),
                imp=("rigid",) if rigid else ("msd", R, M, K),
                init=("pulse", src[0], src[1], 1e-3, 3 * H), probes=probes, steps=steps)


def cylinder_pulse(n=1024, steps=3000, R=2.0, M=0.02, K=1.0, rigid=False, nx=None, ny=None,
                   sponge=LONG_RUN_SPONGE) -> Case:
    """Cylinder of radius n/20.48 cells (50 at n = 1024) at the centre, Gaussian
    pulse of half-width 4n/1024 cells and amplitude 1 at n/10.24 cells on +x;
    8 probes on a ring of 1.5 radii; the long-run absorbing ramp by default.
    The physical problem is the same for every n when h = 0.01 * 1024 / n
    (refinement sweeps pass h explicitly)."""
    nx = nx or n
    ny = ny or n
    c = ((nx - 1) / 2 * H, (ny - 1) / 2 * H)
    r = n / 20.48 * H
    w = 4.0 * n / 1024 * H
    xs = c[0] + n / 10.24 * H
    ang = np.arange(8) * math.pi / 4
    probes = np.stack([c[0] + 1.5 * r * np.cos(ang), c[1] + 1.5 * r * np.sin(ang)], 1)
    return Case("cylinder_pulse_%dx%d" % (nx, ny), nx, ny, wall=("cyl", c[0], c[1], r),
                imp=("rigid",) if rigid else ("msd", R, M, K),
                init=("pulse", xs, c[1], 1.0, w), probes=probes, steps=steps, sponge=sponge)


def monopole(n=2048, steps=20000, R=1.0, M=0.1, K=10.0, radius_cells=None, src_cells=None,
             nring=256, sponge=LONG_RUN_SPONGE) -> Case:
    """Cylinder of radius n/20.48 cells scattering a harmonic monopole at
    3 radii on +x (half-width 3 cells, amplitude 1, 20 points per wavelength);
    probe ring of nring points at 1.1 radii; the long-run absorbing ramp by
    default (20000 steps)."""
    c = ((n - 1) / 2 * H, (n - 1) / 2 * H)
    rc = (radius_cells if radius_cells is not None else n / 20.48) * H
    xs = c[0] + (src_cells if src_cells is not None else 3 * n / 20.48) * H
    omega = 2 * math.pi / (20 * H)
    ang = np.arange(nring) * 2 * math.pi / nring
    probes = np.stack([c[0] + 1.1 * rc * np.cos(ang), c[1] + 1.1 * rc * np.sin(ang)], 1)
    return Case("monopole_%d" % n, n, n, wall=("cyl", c[0], c[1], rc), imp=("msd", R, M, K),
                source=("monopole", xs, c[1], 1.0, 3 * H, omega), probes=probes, steps=steps,
                sponge=sponge)


SWEEP_SIZES = (256, 384, 512, 768, 1024)


def sweep(count=512, seed=24785, steps=2000, accept: Optional[Callable[[Case], bool]] = None,
          sizes=SWEEP_SIZES, sponge=LONG_RUN_SPONGE) -> Tuple[List[Case], int]:
    """Batched parametric sweep: grid n uniform in `sizes`, cylinder radius 0.1 n
    cells at the centre, pulse (half-width 4 cells) at 0.25 n cells on +x, R, M,
    K log-uniform in [0.2, 5], [0.005, 0.2], [0.5, 20], the long-run absorbing
    ramp.  Draws rejected by `accept` (e.g. an unstable wall ODE) are redrawn
    from the same stream; returns (cases, rejected)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out, rejected = [], 0
    while len(out) < count:
        n = int(rng.choice(sizes))
        R = float(np.exp(rng.uniform(np.log(0.2), np.log(5.0))))
        M = float(np.exp(rng.uniform(np.log(0.005), np.log(0.2))))
        K = float(np.exp(rng.uniform(np.log(0.5), np.log(20.0))))
        c = ((n - 1) / 2 * H, (n - 1) / 2 * H)
        case = Case("sweep_%d_n%d" % (len(out), n), n, n, wall=("cyl", c[0], c[1], 0.1 * n * H),
                    imp=("msd", R, M, K), init=("pulse", c[0] + 0.25 * n * H, c[1], 1.0, 4 * H),
                    probes=np.array([[c[0] + 0.15 * n * H, c[1]]]), steps=steps, sponge=sponge)
        if accept is None or accept(case):
            out.append(case)
        else:
            rejected += 1
    return out, rejected


def rational_sweep(count=512, seed=24785, steps=2000, accept: Optional[Callable[[Case], bool]] = None,
                   sizes=SWEEP_SIZES, sponge=LONG_RUN_SPONGE) -> Tuple[List[Case], int]:
    """The sweep's geometry with broadband walls (Sec. 2.3, Eq. Yrational with
    Y_inf = 0): two real poles lam in -[5, 200] with residues A in [0.5, 10],
    and one complex pair alpha +- i beta, alpha in -[5, 50], beta in [10, 60],
    residue B + i C with B in [1, 20] and C = -B alpha / beta (so that the pair's
    numerator is a pure multiple of s, as for a mass-spring-damper); all
    log-uniform: four ADE states per ghost point."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lu = lambda a, b: float(np.exp(rng.uniform(np.log(a), np.log(b))))
    out, rejected = [], 0
    while len(out) < count:
        n = int(rng.choice(sizes))
        real = [(-lu(5.0, 200.0), lu(0.5, 10.0)) for _ in range(2)]
        al, be, B = -lu(5.0, 50.0), lu(10.0, 60.0), lu(1.0, 20.0)
        pairs = [(al, be, B, -B * al / be)]
        c = ((n - 1) / 2 * H, (n - 1) / 2 * H)
        case = Case("rational_sweep_%d_n%d" % (len(out), n), n, n, wall=("cyl", c[0], c[1], 0.1 * n * H),
                    imp=("rational", real, pairs), init=("pulse", c[0] + 0.25 * n * H, c[1], 1.0, 4 * H),
                    probes=np.array([[c[0] + 0.15 * n * H, c[1]]]), steps=steps, sponge=sponge)
        if accept is None or accept(case):
            out.append(case)
        else:
            rejected += 1
    return out, rejected


SERVE_SIZES = (256, 384, 512, 768, 1024, 1536, 2048)


def serving_trace(rate=200.0, duration=1.0, seed=24786, accept=None, sizes=SERVE_SIZES,
                  steps_range=(1000, 10000), sponge=LONG_RUN_SPONGE,
                  wall_sponge=WALL_EDGE_SPONGE) -> List[Tuple[float, Case]]:
    """Poisson arrivals (mean `rate` per second over `duration` seconds) of mixed
    solves: half flat walls through the centre at an angle U[0, 60] deg, half
    cylinders of radius U[0.05, 0.15] n; pulse of half-width 4 cells at a
    uniform position at least 20 cells from the wall and the edges; R, M, K as
    in the sweep; steps uniform in steps_range; the long-run absorbing ramp for
    cylinders and the stronger one for flat walls, which meet the outer band
    (runs last up to 10000 steps)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t, out = 0.0, []
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t > duration:
            break
        while True:
            n = int(rng.choice(sizes))
            c = ((n - 1) / 2 * H, (n - 1) / 2 * H)
            R = float(np.exp(rng.uniform(np.log(0.2), np.log(5.0))))
            M = float(np.exp(rng.uniform(np.log(0.005), np.log(0.2))))
            K = float(np.exp(rng.uniform(np.log(0.5), np.log(20.0))))
            steps = int(rng.integers(steps_range[0], steps_range[1] + 1))
            if rng.uniform() < 0.5:
                th = math.radians(float(rng.uniform(0, 60)))
                wall = ("line", c[0] + 0.37 * H, c[1], th)
                nrm = np.array([-math.sin(th), math.cos(th)])
                # fluid side, 20..(n/2 - 20) cells from the wall along the normal
                d = float(rng.uniform(20, max(21, n / 2 - 24)))
                pos = np.array(c) + d * H * nrm
            else:
                rr = float(rng.uniform(0.05, 0.15)) * n
                wall = ("cyl", c[0], c[1], rr * H)
                ang = float(rng.uniform(0, 2 * math.pi))
                d = float(rng.uniform(rr + 20, max(rr + 21, n / 2 - 24)))
                pos = np.array(c) + d * H * np.array([math.cos(ang), math.sin(ang)])
            case = Case("serve_%d_n%d" % (len(out), n), n, n, wall=wall, imp=("msd", R, M, K),
                        init=("pulse", pos[0], pos[1], 1.0, 4 * H),
                        probes=np.array([[pos[0], pos[1]]]), steps=steps,
                        sponge=wall_sponge if wall[0] == "line" else sponge)
            if accept is None or accept(case):
                break
        out.append((t, case))
    return out


def apply_to(case: Case, target):
    """Set geometry, impedance and probes on a product Solver or an oracle via
    their common setter names (the caller then plans / sets up)."""
    w = case.wall
    if w[0] == "line":
        (target.set_wall_line if hasattr(target, "set_wall_line") else target.set_line)(*w[1:])
    elif w[0] == "cyl":
        (target.set_wall_cylinder if hasattr(target, "set_wall_cylinder") else target.set_cylinder)(*w[1:])
    else:
        (target.set_wall_none if hasattr(target, "set_wall_none") else target.set_none)()
    if case.imp[0] == "msd":
        target.set_impedance(*case.imp[1:])
    elif case.imp[0] == "rational":
        target.set_impedance_rational(*case.imp[1:])
    else:
        target.set_rigid()
    if case.sponge[0] > 0:
        target.set_sponge(*case.sponge)
    return target


def apply_state(case: Case, target):
    """Initial field and source (after plan/bind or set-up)."""
    if case.source is not None:
        target.set_monopole(*case.source[1:])
    if case.init[0] == "pulse":
        target.init_pulse(*case.init[1:])
    elif case.init[0] == "packet":
        target.init_packet(*case.init[1:])
    return target


def flat_wall_paper(h=0.005, rigid=False, t_end=2.0) -> Case:
    """The flat immersed wall of Sec. 4.1: domain [-1, 0.8] x [-0.2, 0.2]
    (shifted here by (+1, +0.2) so that node (0, 0) sits at the origin),
    periodic in y, radiation condition at x = -1; wall normal to x at
    x = 0.6 + h/2 (fluid on the left); wave packet p0 = (a/2) exp(-alpha^2 x^2)
    cos(2 pi k x), u0 = p0, v0 = 0, a = 1, k = 7, alpha = k / sqrt(0.8), at
    x = 0; MSD wall M = 0.025, K = 40, R = 0.2 (or rigid); CFL 0.5; probe at
    the microphone (0.5, 0); t_end = 2."""
    nx = int(round(1.8 / h)) + 1
    ny = int(round(0.4 / h))
    k = 7.0
    xw = 1.6 + h / 2
    steps = int(round(t_end / (CFL * h)))
    return Case("flat_wall_paper_h%g%s" % (h, "_rigid" if rigid else ""), nx, ny, h=h,
                wall=("line", xw, 0.2, math.pi / 2),
                imp=("rigid",) if rigid else ("msd", 0.2, 0.025, 40.0),
                init=("packet", 1.0, 0.2, 0.0, 1.0, k, k / math.sqrt(0.8)),
                probes=np.array([[1.5, 0.2]]), steps=steps, periodic=(False, True))


def pulse_cylinder_paper(h=0.04, R=None, M=0.025, K=1.6, t_end=6.0, half=6.0) -> Case:
    """The pulse-cylinder case of Sec. 4.2: domain [-6, 6]^2 (shifted by +6 so
    that node (0, 0) sits at the origin), cylinder of radius 0.5 at the
    centre, Gaussian pulse a = 1, w = 0.2 at (4, 0), radiation condition on
    all sides, CFL 0.5; MSD wall M = 0.025, K = 1.6 and resistance R (the
    paper's impedance case R = 0.2; the sweep of Fig. 8b R in {3, 2, 1, 0.5,
    0.2}), R = None the rigid wall; probe at microphone A (2, 0).  `half` is
    the half-width of the box (the paper's 6; a wider box moves the outer
    boundary's reflections out of the recorded window)."""
    n = int(round(2 * half / h)) + 1
    c = half
    return Case("pulse_cylinder_paper_h%g_%s_L%g" % (h, "rigid" if R is None else "R%g" % R, half), n, n, h=h,
                wall=("cyl", c, c, 0.5), imp=("rigid",) if R is None else ("msd", R, M, K),
                init=("pulse", c + 4.0, c, 1.0, 0.2), probes=np.array([[c + 2.0, c]]),
                steps=int(round(t_end / (CFL * h))))
