"""Closed-form and semi-analytic reference solutions of the paper's test
problems, evaluated with numpy/scipy only (no code of the product or the
oracle).  Test infrastructure.

* ``free_pulse``: the Gaussian pressure pulse p0 = a exp(-b r^2), u = v = 0 in
  free space (rho0 = c0 = 1).  Its Hankel transform is a exp(-k^2/4b)/(2b)
  (App. B, the transform of the initial pulse), each wavenumber oscillates as
  cos(k t), so
      p(r, t)   = (a / 2b) int_0^inf exp(-k^2/4b) cos(k t) J0(k r) k dk,
      u_r(r, t) = (a / 2b) int_0^inf exp(-k^2/4b) sin(k t) J1(k r) k dk
  (u_r from du/dt = -grad p).  The integrals are taken by Gauss-Legendre
  quadrature on [0, 12 sqrt(b)], where the Gaussian factor is below 1e-15.
"""
from __future__ import annotations

import numpy as np
from scipy.special import j0, j1


def free_pulse(r, t, a, b, nk=4000):
    """Exact (p, u_r) of the free Gaussian pulse at radii r and time t."""
    kmax = 12.0 * np.sqrt(b)
    x, wq = np.polynomial.legendre.leggauss(nk)
    k = 0.5 * kmax * (x + 1.0)
    wk = 0.5 * kmax * wq * np.exp(-k * k / (4.0 * b)) * k * (a / (2.0 * b))
    r = np.asarray(r, dtype=np.float64)
    kr = np.outer(k, r.ravel())
    p = (np.cos(k * t) * wk) @ j0(kr)
    ur = (np.sin(k * t) * wk) @ j1(kr)
    return p.reshape(r.shape), ur.reshape(r.shape)
