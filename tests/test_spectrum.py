"""The spectral stability tool (oracle/spectrum.py): the semi-discrete
operator assembled from the oracle, checked against the closed-form DRP
dispersion relation, and the stability findings it supports."""
import math

import numpy as np
import pytest

import oracle
from oracle import spectrum

A = (0.770882380518, -0.166705904415, 0.020843142770)      # Sec. 2.2


def test_periodic_box_spectrum_is_the_drp_dispersion_relation():
    """Without a wall and with periodic axes the semi-discrete LEE is
    p' = -(Dx u + Dy v), u' = -Dx p, v' = -Dy p with the DRP operator, whose
    Fourier symbol is i k*, k* h = 2 sum_j a_j sin(j k h): the eigenvalues
    are 0 (n^2 times) and +-i sqrt(k*x^2 + k*y^2), all on the imaginary axis."""
    n, h = 12, 0.05
    o = oracle.Oracle(n, n, h, 0.5, periodic_x=True, periodic_y=True)
    o.set_none()
    o.setup()
    lam = spectrum.eigenvalues(o)
    assert np.abs(lam.real).max() < 1e-10 / h
    k = 2 * math.pi * np.fft.fftfreq(n, h)
    ks = 2 * sum(a * np.sin((j + 1) * k * h) for j, a in enumerate(A)) / h
    KX, KY = np.meshgrid(ks, ks)
    w = np.sqrt(KX ** 2 + KY ** 2).ravel()
    expect = np.sort(np.concatenate([w, -w, np.zeros(n * n)]))
    np.testing.assert_allclose(np.sort(lam.imag), expect, atol=1e-9 / h)


def test_ade_states_enter_the_operator():
    """With an impedance wall the operator carries two states per ghost; its
    spectrum differs from the rigid wall's, and a wall ODE whose poles lie far
    outside the RK4 region shows up as |P(lambda dt)| >> 1 (the check that
    lee_plan makes on the poles alone)."""
    n, h = 24, 0.01
    c = (n - 1) / 2 * h

    def spec(imp):
        o = oracle.Oracle(n, n, h, 0.5, periodic_x=True, periodic_y=True)
        o.set_cylinder(c + 0.21 * h, c + 0.37 * h, 5.3 * h)
        if imp is None:
            o.set_rigid()
        else:
            o.set_impedance(*imp)
        o.setup()
        L, _, nfield = spectrum.assemble(o)
        return L, nfield, o
    Lr, nf, o = spec(None)
    Li, nf2, oi = spec((1.0, 0.1, 10.0))
    assert nf == nf2 and Li.shape[0] == nf + 2 * oi.n_ghost
    # a stiff wall: poles near -R/M = -4000, dt = 0.005 -> z = -20, far outside
    Ls, _, os_ = spec((40.0, 0.01, 10.0))
    amp = spectrum.rk4_amplification(np.linalg.eigvals(Ls), os_.dt).max()
    assert amp > 100.0
    assert oracle.ade_stability(40.0, 0.01, 10.0, os_.dt) > 100.0


def test_radiation_closure_has_growing_modes_and_the_ramp_damps_them():
    """The outer closure (one-sided DRP rows + radiation condition, Secs. 2.2,
    4.1) alone, no wall: its semi-discrete operator has eigenvalues with a
    positive real part (grid-scale modes, |Im lambda h| near the DRP's largest
    modified wavenumber), which is why rounding errors grow on long runs; the
    opt-in absorbing ramp moves them to (or below) about 1e-3 / h."""
    n, h = 32, 0.01
    o = oracle.Oracle(n, n, h, 0.5)
    o.set_none()
    o.setup()
    lam = spectrum.eigenvalues(o)
    a0 = spectrum.abscissa(lam) * h
    assert a0 > 1e-3, a0
    i = np.argmax(lam.real)
    assert abs(lam[i].imag * h) > 1.0
    o2 = oracle.Oracle(n, n, h, 0.5)
    o2.set_none()
    o2.set_sponge(8, 0.04)
    o2.setup()
    a1 = spectrum.abscissa(spectrum.eigenvalues(o2)) * h
    assert a1 < 0.5 * a0, (a0, a1)


def test_wall_meeting_the_band_is_stabilised_by_the_strong_ramp():
    """An impedance wall through the box at 40 deg (it crosses the radiation
    band on two sides; band derivatives whose window holds a non-fluid node
    are left out, reading R20): without the ramp the operator has modes growing
    at Re lambda h of several 1e-2 (what made long serving runs diverge); the
    ramp of 12 layers at kappa = 0.4 that serving gives flat walls brings the
    spectral abscissa down to rounding level, and the four-stage scheme's
    amplification to 1."""
    n, h = 32, 0.01
    c = (n - 1) / 2 * h

    def build(ramp):
        o = oracle.Oracle(n, n, h, 0.5)
        o.set_line(c + 0.37 * h, c, math.radians(40.0))
        o.set_impedance(1.0, 0.05, 5.0)
        if ramp:
            o.set_sponge(12, 0.4)
        o.setup()
        return o

    lam0 = spectrum.eigenvalues(build(False))
    assert spectrum.abscissa(lam0) * h > 1e-2
    o = build(True)
    lam1 = spectrum.eigenvalues(o)
    assert spectrum.abscissa(lam1) * h < 1e-4
    assert spectrum.rk4_amplification(lam1, o.dt).max() < 1.0 + 1e-6
