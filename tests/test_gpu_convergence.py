"""Convergence of the whole solver on the GPU (FP64 bulk).

Cylinder self-convergence: a pulse reflected by a cylinder, the same physical
problem on 256^2, 512^2 and 1024^2 grids, compared with a 2048^2 run at the
same physical times and probe positions.  Measured on a B300: rigid 5.0e-3,
2.0e-4, 4.2e-5 (orders 4.7, 2.2); impedance 5.4e-3, 1.9e-4, 2.8e-5 (4.9, 2.7).
The last order depends on the cylinder's sub-cell position (rigid 2.2-2.9,
impedance 2.7-3.7 over four centre offsets; energy conserved to 1e-5 on every
grid): a geometry-dependent error component of the ghost configuration, not
the reference's own error.  Asserted per refinement: first order >= 4, second
>= 2, mean >= 3.

Against exact and semi-analytic references: the paper's Sec. 4.1 flat wall
(App. A) and Sec. 4.2 pulse-cylinder (App. B), and the Fig. 8b R sweep."""
import math

import numpy as np
import pytest

from paper_2609_24785_b300 import workloads
from _helpers import make_solver

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

L = 10.24                       # domain side (physical units)
XC = 5.12 + 0.00137             # cylinder centre, off every grid's nodes
R_CYL, W, XS_OFF = 0.5, 0.16, 1.0
T_END = 1.6                     # the reflected pulse has crossed the probe ring


def _case(n, rigid):
    h = L / n
    ang = np.arange(8) * math.pi / 4
    probes = np.stack([XC + 1.5 * R_CYL * np.cos(ang), XC + 1.5 * R_CYL * np.sin(ang)], 1)
    steps = int(round(T_END / (0.5 * h)))
    return workloads.Case("conv_%d" % n, n, n, h=h, wall=("cyl", XC, XC, R_CYL),
                          imp=("rigid",) if rigid else ("msd", 2.0, 0.02, 1.0),
                          init=("pulse", XC + XS_OFF, XC, 1.0, W), probes=probes, steps=steps)


def _probes(n, rigid, precision):
    c = _case(n, rigid)
    s = make_solver(c, precision)
    s.step(c.steps)
    s.sync()
    return s.probes()                          # steps x 8, sample k at t = (k + 1) dt_n


def _orders(rigid, precision):
    ref = _probes(2048, rigid, precision)
    errs = []
    for n in (256, 512, 1024):
        p = _probes(n, rigid, precision)
        stride = 2048 // n                     # the fine run's samples at the coarse times
        fine = ref[stride - 1::stride][:p.shape[0]]
        errs.append(float(np.sqrt(np.mean((p - fine) ** 2)) / np.sqrt(np.mean(fine ** 2))))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    return errs, orders, math.log2(errs[0] / errs[2]) / 2


@pytest.mark.parametrize("rigid", [True, False], ids=["rigid", "impedance"])
def test_cylinder_pulse_converges(rigid, cuda_device):
    errs, orders, mean = _orders(rigid, "fp64")
    print("%s: relative probe errors %s, orders %s, mean %.2f" % (
        "rigid" if rigid else "impedance", ["%.2e" % e for e in errs], ["%.2f" % o for o in orders], mean))
    assert errs[0] > errs[1] > errs[2]
    assert orders[0] >= 4.0 and orders[1] >= 2.0, (errs, orders)
    assert mean >= 3.0, (errs, orders)


@pytest.mark.parametrize("rigid", [False, True], ids=["impedance", "rigid"])
def test_paper_flat_wall_converges_on_gpu(rigid, cuda_device):
    """The flat immersed wall of Sec. 4.1 at the paper's grids h = 0.01, 0.005,
    0.0025 and one finer, 0.00125 (FP64 bulk, periodic in y, radiation
    condition at x = -1), against the App. A exact microphone signal: every
    successive order is at least 3.8 (the paper: 4 in Sec. 4.1, about 4.5 in
    its conclusion), and the h = 0.005 run equals the oracle's to 1e-12."""
    import sys, os
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    from test_oracle_pins import _paper_flat_wall_error
    from _helpers import make_oracle, log_result, rel_l2

    def run(case):
        s = make_solver(case, "fp64")
        s.step(case.steps)
        s.sync()
        return s.probes()[:, 0]
    hs = (0.01, 0.005, 0.0025, 0.00125)
    errs = [_paper_flat_wall_error(h, rigid, run) for h in hs]
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(len(hs) - 1)]
    log_result("flat wall Sec. 4.1 %s (GPU FP64): errors %s, orders %s" % (
        "rigid" if rigid else "impedance", ["%.3e" % e for e in errs], ["%.2f" % o for o in orders]))
    assert min(orders) >= 3.8, (errs, orders)
    case = workloads.flat_wall_paper(0.005, rigid)
    o = make_oracle(case)
    o.run(case.steps)
    assert rel_l2(run(case), o.probes()[:, 0]) <= 1e-12


@pytest.mark.parametrize("R", [None, 0.2], ids=["rigid", "impedance"])
def test_pulse_cylinder_converges_to_app_b_on_gpu(R, cuda_device):
    """Sec. 4.2's pulse-cylinder case on the paper's grids h = 0.08, 0.04,
    0.02 (FP64 bulk), microphone A, window t in [4, 6], against the App. B
    semi-analytic reference: the second order at least 2.8 (the paper: 4
    rigid, about 3 impedance; measured 3.1 and 3.3).  At h = 0.01 the error in
    the paper's [-6, 6]^2 box stops falling (6e-4 rigid, 8e-4 impedance): the
    first-order radiation condition's reflections from the box edge reach the
    microphone inside the window.  In a box twice as wide the h = 0.01 error
    falls below that floor."""
    import sys, os
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    from test_oracle_pins import _app_b_error
    from _helpers import log_result

    def err(h, half=6.0):
        case = workloads.pulse_cylinder_paper(h, R, half=half)
        s = make_solver(case, "fp64")
        s.step(case.steps)
        s.sync()
        return _app_b_error(case, s.probes()[:, 0])
    errs = [err(h) for h in (0.08, 0.04, 0.02, 0.01)]
    wide = err(0.01, half=12.0)
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(3)]
    log_result("pulse-cylinder Sec. 4.2 %s vs App. B (GPU FP64): errors %s, orders %s; h = 0.01 in a "
               "[-12, 12]^2 box %.3e" % ("rigid" if R is None else "R=%g" % R, ["%.3e" % e for e in errs],
                                          ["%.2f" % o for o in orders], wide))
    assert orders[1] >= 2.8, (errs, orders)
    assert wide < errs[3], (wide, errs)


def test_resistance_sweep_against_app_b(cuda_device):
    """Fig. 8b: the MSD wall (M = 0.025, K = 1.6) swept over R in {3, 2, 1,
    0.5, 0.2} and the rigid wall, h = 0.02 on the GPU, each against its App. B
    reference at microphone A (t in [4, 6]); and the sharp first reflection
    (t = 4.89) weakens as R falls from the rigid limit to 1, as in the paper
    (below R = 1 the reactance dominates and the reflection returns, later).
    Measured errors 8.3e-4 (rigid), 1.6e-3, 2.3e-3, 5.6e-3 for R = 3, 2, 1."""
    import sys, os
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    from test_oracle_pins import _app_b_error
    from _helpers import log_result
    peaks = {}
    for R in (None, 3.0, 2.0, 1.0, 0.5, 0.2):
        case = workloads.pulse_cylinder_paper(0.02, R)
        s = make_solver(case, "fp64")
        s.step(case.steps)
        s.sync()
        pr = s.probes()[:, 0]
        e = _app_b_error(case, pr)
        t = (np.arange(len(pr)) + 1) * case.cfl * case.h
        peaks[R] = float(np.abs(pr[np.argmin(np.abs(t - 4.89))]))
        log_result("R sweep h=0.02 %s: error vs App. B %.3e, |p(4.89)| at microphone A %.4e" % (
            "rigid" if R is None else "R=%g" % R, e, peaks[R]))
        # relative to a weaker reflected signal at R = 1 (its sharp reflection
        # is 24 times weaker than the rigid one) the same absolute error is larger
        assert e < 2e-2, (R, e)
    assert peaks[None] > peaks[3.0] > peaks[2.0] > peaks[1.0], peaks
