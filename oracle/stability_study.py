"""Spectral stability study of the semi-discrete operator (abstract of the
paper: instability of walls tangent to the grid), on small grids with the
oracle-assembled operator of oracle/spectrum.py.  Prints, per configuration,
the spectral abscissa max Re(lambda) h, the imaginary part of that eigenvalue
and max |P(lambda dt)| of the four-stage scheme (growth per step).

    python -m oracle.stability_study          (about five minutes on 8 cores)

TEST INFRASTRUCTURE: an analysis tool; it imports the oracle only.
"""
from __future__ import annotations

import math
import sys

import numpy as np

from . import Oracle
from . import spectrum

H = 0.01


def _row(label, o):
    lam = spectrum.eigenvalues(o)
    i = int(np.argmax(lam.real))
    print("%-46s abscissa*h %+.3e  Im*h %6.3f  max|P| %.5f  (%d unknowns)" % (
        label, lam[i].real * H, lam[i].imag * H, spectrum.rk4_amplification(lam, o.dt).max(), len(lam)),
        flush=True)
    return lam


def closure(n=40):
    """The outer closure alone (no wall), with and without the ramp."""
    for sponge in (0, 8):
        o = Oracle(n, n, H, 0.5)
        o.set_none()
        if sponge:
            o.set_sponge(sponge, 0.04)
        o.setup()
        _row("no wall %d^2, ramp %d" % (n, sponge), o)


def cylinders(n=40):
    """Cylinders in a periodic box (no outer closure): radius and sub-cell
    offset of the centre (where the wall is tangent to grid lines)."""
    c = (n - 1) / 2 * H
    for r in (6.3, 8.3, 10.3, 12.3):
        for off in ((0.0, 0.0), (0.21, 0.37), (0.5, 0.5)):
            for imp in (None, (1.0, 0.1, 10.0)):
                o = Oracle(n, n, H, 0.5, periodic_x=True, periodic_y=True)
                o.set_cylinder(c + off[0] * H, c + off[1] * H, r * H)
                if imp:
                    o.set_impedance(*imp)
                o.setup()
                _row("cylinder r=%.1f offset (%.2f,%.2f) %s" % (r, off[0], off[1], "MSD" if imp else "rigid"), o)


def flat_walls(n=40):
    """Straight walls through the box at angle theta to the x axis (0: tangent
    to the grid lines), ramp of 8 layers against the closure's own modes."""
    c = (n - 1) / 2 * H
    for ang in (0.0, 2.0, 5.0, 10.0, 20.0, 30.0):
        for off in (0.0, 0.25, 0.5):
            o = Oracle(n, n, H, 0.5)
            o.set_line(c, c + off * H, math.radians(ang))
            o.set_sponge(8, 0.04)
            o.setup()
            _row("line %4.1f deg offset %.2f (ramp 8)" % (ang, off), o)


if __name__ == "__main__":
    which = sys.argv[1:] or ["closure", "cylinders", "flat_walls"]
    for w in which:
        print("--", w)
        globals()[w]()
