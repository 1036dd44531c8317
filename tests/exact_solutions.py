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


def flat_wall_signal(F, t, x_mic, x_wall, Z=None):
    """App. A: pressure at x_mic (fluid at x < x_wall) of the incident simple
    wave F(x - t) and its reflection from a locally reacting wall,
        p(x_m, t) = F(x_m - t) + r(t - (x_wall - x_m)),
    r = R_c * F(x_wall - tau) with R_c(w) = (Z - 1)/(Z + 1) applied by FFT
    (Z(s) with s = i w; Z = None is the rigid wall, R_c = 1).  t must be a
    uniform grid t_n = (n + 1) dt on which the travel time x_wall - x_mic is a
    whole number of steps; the filtered signal is sampled on the same step
    over a window long enough for it to decay."""
    t = np.asarray(t, dtype=np.float64)
    dt = t[1] - t[0]
    delay = (x_wall - x_mic) / dt
    nd = int(round(delay))
    assert abs(delay - nd) < 1e-6, "travel time must be a whole number of steps"
    T = 1 << int(np.ceil(np.log2(4 * (len(t) + nd) + 1024)))
    tau = np.arange(T) * dt
    sig = F(x_wall - tau)
    w = 2 * np.pi * np.fft.fftfreq(T, dt)
    if Z is None:
        Rc = np.ones(T, dtype=complex)
    else:
        s = 1j * w
        s[0] = 1e-300j
        z = Z(s)
        Rc = (z - 1) / (z + 1)
        Rc[0] = 1.0                      # a spring: Z -> infinity as s -> 0, R_c -> 1
    refl = np.real(np.fft.ifft(Rc * np.fft.fft(sig)))
    # r at times t - (x_wall - x_mic): index n + 1 - nd on the tau grid
    idx = np.round(t / dt).astype(int) - nd
    r = np.where(idx >= 0, refl[np.clip(idx, 0, T - 1)], 0.0)
    return F(x_mic - t) + r


def monopole_cylinder(x, y, xs, ys, xc, yc, a_cyl, omega, amp, w, Z=None, nextra=40):
    """App. C: complex pressure amplitude P (p = Im(P e^{i w t})) of the
    harmonic Gaussian monopole s = amp exp(-b |x - xs|^2) sin(w t),
    b = ln 2 / w^2, scattered by a cylinder of radius a_cyl at (xc, yc) with
    impedance Z(w) = R + i (M w - K / w) (None: rigid), c = rho = 1, k = w:
        P = C H0(k |x - xs|) + C sum_n eps_n H_n(k r_s) S_n H_n(k r) cos(n (th - th_s)),
        C = (w / 4) amp (pi / b) exp(-k^2 / 4b),
        S_n = -(J_n(ka) + i Z J_n'(ka)) / (H_n(ka) + i Z H_n'(ka))   (H = H^(2)),
    the Graf re-expansion of the incident field about the cylinder axis
    (valid for r < r_s), truncated at N = ceil(ka) + nextra modes."""
    from scipy.special import hankel2, h2vp, jv, jvp
    k = float(omega)
    b = np.log(2.0) / w ** 2
    C = (omega / 4.0) * amp * (np.pi / b) * np.exp(-k * k / (4.0 * b))
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    r = np.hypot(x - xc, y - yc)
    th = np.arctan2(y - yc, x - xc)
    rs = np.hypot(xs - xc, ys - yc)
    ths = np.arctan2(ys - yc, xs - xc)
    assert np.all(r < rs), "the Graf expansion holds inside the source radius"
    ka = k * a_cyl
    N = int(np.ceil(ka)) + nextra
    P = C * hankel2(0, k * np.hypot(x - xs, y - ys))
    for n in range(N + 1):
        eps = 1.0 if n == 0 else 2.0
        if Z is None:
            S = -jvp(n, ka) / h2vp(n, ka)
        else:
            S = -(jv(n, ka) + 1j * Z * jvp(n, ka)) / (hankel2(n, ka) + 1j * Z * h2vp(n, ka))
        P = P + C * eps * hankel2(n, k * rs) * S * hankel2(n, k * r) * np.cos(n * (th - ths))
    return P


def harmonic_amplitude(p, t, omega):
    """Least-squares fit p(t) = Re(P) sin(w t) + Im(P) cos(w t) (i.e.
    p = Im(P e^{i w t})) over the samples; returns P per column of p."""
    A = np.stack([np.sin(omega * t), np.cos(omega * t)], 1)
    coef, *_ = np.linalg.lstsq(A, np.asarray(p, dtype=np.float64), rcond=None)
    return coef[0] + 1j * coef[1]


def pulse_cylinder(x, y, t, xs, ys, a_cyl, amp, w, Zfun=None, xc=0.0, yc=0.0, nw=3000, wmax=None,
                   nextra=20, scattered_only=False):
    """App. B: pressure of the Gaussian pulse p0 = amp exp(-b |x - xs|^2),
    u = v = 0 at t = 0 (b = ln 2 / w^2, rho = c = 1), scattered by a cylinder
    of radius a_cyl at (xc, yc), at points (x, y) (inside the source radius)
    and times t.  The initial-value problem equals the causal response to the
    source p0(x) delta'(t); in the e^{-i w t} convention of App. B its
    spectrum is, with k = w,
        P(x, w) = (w / 4) (pi / b) e^{-k^2 / 4b} [H0(k |x - xs|)
                  + sum_n eps_n H_n(k r_s) S_n(w) H_n(k r) cos(n (th - th_s))],
        S_n = -(J_n(ka) - i Z J_n'(ka)) / (H_n(ka) - i Z H_n'(ka))  (H = H^(1)),
    Z(w) = Zfun(w) the impedance in this convention (for the MSD wall
    R - i (M w - K / w)), None: rigid (S_n = -J_n'/H_n'); and
    p(x, t) = (1/pi) Re int_0^wmax P(x, w) e^{-i w t} dw by Gauss-Legendre
    quadrature with nw nodes; wmax defaults to 12 sqrt(b) (the Gaussian factor
    below 1e-15), modes up to ceil(k a) + nextra."""
    from scipy.special import hankel1, h1vp, jv, jvp
    b = np.log(2.0) / w ** 2
    wmax = 12.0 * np.sqrt(b) if wmax is None else wmax
    xg, wq = np.polynomial.legendre.leggauss(nw)
    om = 0.5 * wmax * (xg + 1.0)
    wq = 0.5 * wmax * wq
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    y = np.atleast_1d(np.asarray(y, dtype=np.float64))
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    r = np.hypot(x - xc, y - yc)
    th = np.arctan2(y - yc, x - xc)
    rs = np.hypot(xs - xc, ys - yc)
    ths = np.arctan2(ys - yc, xs - xc)
    assert np.all(r < rs)
    k = om
    C = (om / 4.0) * amp * (np.pi / b) * np.exp(-k * k / (4.0 * b))           # (nw,)
    P = np.zeros((nw, len(x)), dtype=complex)
    if not scattered_only:
        P += hankel1(0, np.outer(k, np.hypot(x - xs, y - ys)))
    ka = k * a_cyl
    N = int(np.ceil(ka.max())) + nextra
    Z = None if Zfun is None else Zfun(om)
    with np.errstate(all="ignore"):
        for n in range(N + 1):
            eps = 1.0 if n == 0 else 2.0
            if Z is None:
                S = -jvp(n, ka) / h1vp(n, ka)
            else:
                S = -(jv(n, ka) - 1j * Z * jvp(n, ka)) / (hankel1(n, ka) - 1j * Z * h1vp(n, ka))
            term = (eps * hankel1(n, k * rs) * S)[:, None] * hankel1(n, np.outer(k, r)) * np.cos(n * (th - ths))[None, :]
            # at low k and high n the factors over- and underflow; the term
            # there is of order (a^2 / (r r_s))^n, far below rounding
            P += np.where(np.isfinite(term), term, 0.0)
    P *= (C * wq)[:, None]
    # p(x_j, t_i) = (1/pi) Re sum_w P(w, x_j) e^{-i w t_i}
    E = np.exp(-1j * np.outer(t, om))                                          # (nt, nw)
    return np.real(E @ P) / np.pi
