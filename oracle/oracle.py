"""ctypes wrapper of the FP64 CPU oracle (test infrastructure only).

Each method names the section of the paper the C routine follows:
  * ``setup``          Sec. 3.1 mask, ghost set, BP/normal, elliptical cloud
                       (Eq. ns-ellipse), LSQ read-out rows (Eqs. ns-poly2d ..
                       ns-readout), Lagrange factors (Eq. ns-ghost); Sec. 2.5 ADE.
  * ``run``            Sec. 2.2 time integration with the six coupling steps
                       of Sec. 3.2 at every stage.
  * ``ghost_rows``     export of the per-ghost cloud and read-out rows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lee_oracle.c")
_LIB = os.path.join(_HERE, "liblee_oracle.so")
_lock = threading.Lock()
_lib = None

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


def lib_path() -> str:
    return _LIB


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               "-Wall", "-o", _LIB + ".tmp", _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        L = C.CDLL(_LIB)
        vp = C.c_void_p
        sig = {
            "orc_create": (vp, [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, C.c_int, C.c_int]),
            "orc_destroy": (None, [vp]),
            "orc_error": (C.c_char_p, [vp]),
            "orc_set_none": (None, [vp]),
            "orc_set_line": (None, [vp, C.c_double, C.c_double, C.c_double]),
            "orc_set_cylinder": (None, [vp, C.c_double, C.c_double, C.c_double]),
            "orc_set_rigid": (None, [vp]),
            "orc_set_msd": (None, [vp, C.c_double, C.c_double, C.c_double]),
            "orc_set_monopole": (None, [vp, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double]),
            "orc_setup": (C.c_int, [vp]),
            "orc_set_f32_storage": (None, [vp, C.c_int]),
            "orc_set_sponge": (None, [vp, C.c_int, C.c_double]),
            "orc_set_rational": (C.c_int, [vp, C.c_int, _dp, _dp, C.c_int, _dp, _dp, _dp, _dp]),
            "orc_n_states": (C.c_int, [vp]),
            "orc_rational_drive": (None, [C.c_int, _dp, _dp, C.c_int, _dp, _dp, _dp, _dp, C.c_double, C.c_long,
                                          C.c_double, _dp]),
            "orc_n_ghost": (C.c_int, [vp]),
            "orc_n_reduced": (C.c_int, [vp]),
            "orc_regime": (C.c_int, [vp]),
            "orc_dt": (C.c_double, [vp]),
            "orc_ghost_meta": (None, [vp, C.c_int, _ip, _dp, _ip, _ip]),
            "orc_ghost_rows": (None, [vp, C.c_int, _ip, _dp, _dp, _dp, _dp]),
            "orc_ghost_fit_degree": (C.c_int, [vp, C.c_int]),
            "orc_get_kind": (None, [vp, C.POINTER(C.c_ubyte)]),
            "orc_init_pulse": (None, [vp, C.c_double, C.c_double, C.c_double, C.c_double]),
            "orc_init_packet": (None, [vp] + [C.c_double] * 6),
            "orc_get_field": (None, [vp, C.c_int, _dp]),
            "orc_set_field": (None, [vp, C.c_int, _dp]),
            "orc_get_ade": (None, [vp, _dp]),
            "orc_set_ade": (None, [vp, _dp]),
            "orc_get_step": (C.c_long, [vp]),
            "orc_set_probes": (C.c_int, [vp, C.c_int, _dp, C.c_long]),
            "orc_get_probes": (C.c_long, [vp, _dp]),
            "orc_run": (None, [vp, C.c_long, C.c_int]),
            "orc_fill_ghosts": (None, [vp, _dp]),
            "orc_fill_ghosts_bc": (None, [vp, _dp]),
            "orc_eval_rhs": (None, [vp, C.c_double, _dp, _dp, _dp, _dp]),
            "orc_energy": (C.c_double, [vp]),
            "orc_deriv_1d": (None, [C.c_int, _dp, C.c_double, C.c_int, _dp]),
            "orc_ade_drive": (None, [C.c_double, C.c_double, C.c_double, C.c_double, C.c_long, C.c_double, _dp, _dp]),
            "orc_ade_regime": (C.c_int, [C.c_double, C.c_double, C.c_double, _dp, _dp, _dp]),
            "orc_ade_stability": (C.c_double, [C.c_double, C.c_double, C.c_double, C.c_double]),
            "orc_stage_forcing": (C.c_double, [C.c_double, C.c_double, C.c_double, C.c_int]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
        return L


def _d(a):
    return a.ctypes.data_as(_dp)


def deriv_1d(f, h, periodic=False):
    """Sec. 2.2 derivative operator (DRP interior, one-sided outer layers)."""
    L = _load()
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.empty_like(f)
    L.orc_deriv_1d(len(f), _d(f), h, int(periodic), _d(out))
    return out


def ade_drive(R, M, K, dt, nsteps, omega):
    """Sec. 2.5 wall ODE forced by sin(omega t); returns (u_n series, final X)."""
    L = _load()
    un = np.empty(nsteps)
    X = np.empty(2)
    L.orc_ade_drive(R, M, K, dt, nsteps, omega, _d(un), _d(X))
    return un, X


def _poles(real, pairs):
    """(n, lam, A, m, al, be, B, C) arrays from real = [(lam, A)], pairs =
    [(alpha, beta, B, C)] (Eq. Yrational)."""
    real = np.asarray(real, dtype=np.float64).reshape(-1, 2)
    pairs = np.asarray(pairs, dtype=np.float64).reshape(-1, 4)
    cols = [np.ascontiguousarray(real[:, i]) for i in range(2)] + [np.ascontiguousarray(pairs[:, i]) for i in range(4)]
    cols = [c if c.size else np.zeros(1) for c in cols]
    return len(real), cols[0], cols[1], len(pairs), cols[2], cols[3], cols[4], cols[5]


def rational_drive(real, pairs, dt, nsteps, omega):
    """Eqs. ADEgeneral/unGeneral alone forced by sin(omega t): u_n per step."""
    L = _load()
    n, lam, A, m, al, be, B, Cc = _poles(real, pairs)
    un = np.empty(nsteps)
    L.orc_rational_drive(n, _d(lam), _d(A), m, _d(al), _d(be), _d(B), _d(Cc), dt, nsteps, omega, _d(un))
    return un


def ade_regime(R, M, K):
    """Returns (regime, A (2x2), b, c): 1 complex pair, 2 real poles, 3 double pole."""
    L = _load()
    A = np.empty(4); b = np.empty(2); c = np.empty(2)
    reg = L.orc_ade_regime(R, M, K, _d(A), _d(b), _d(c))
    return reg, A.reshape(2, 2), b, c


def stage_forcing(omega, tn, dt, k):
    """Forcing value of stage k (1..4) for sin(omega t) over [tn, tn + dt]."""
    return _load().orc_stage_forcing(omega, tn, dt, k)


def ade_stability(R, M, K, dt):
    """max |P(pole dt)| of the four-stage RK4 polynomial over the MSD poles."""
    return _load().orc_ade_stability(R, M, K, dt)


class Oracle:
    """One problem instance of the oracle."""

    def __init__(self, nx, ny, h, cfl=0.5, x0=0.0, y0=0.0, periodic_x=False, periodic_y=False):
        self._L = _load()
        self.nx, self.ny, self.h = nx, ny, h
        self._o = self._L.orc_create(nx, ny, h, cfl, x0, y0, int(periodic_x), int(periodic_y))
        self.dt = self._L.orc_dt(self._o)
        self._nprobe = 0

    def __del__(self):
        if getattr(self, "_o", None):
            self._L.orc_destroy(self._o)
            self._o = None

    # geometry / impedance / source
    def set_none(self):
        self._L.orc_set_none(self._o)

    def set_line(self, xw, yw, angle):
        self._L.orc_set_line(self._o, xw, yw, angle)

    def set_cylinder(self, xc, yc, r):
        self._L.orc_set_cylinder(self._o, xc, yc, r)

    def set_rigid(self):
        self._L.orc_set_rigid(self._o)

    def set_impedance(self, R, M, K):
        self._L.orc_set_msd(self._o, R, M, K)

    def set_monopole(self, xs, ys, amp, halfwidth, omega):
        self._L.orc_set_monopole(self._o, xs, ys, amp, halfwidth, omega)

    def set_f32_storage(self, on=True):
        """Emulate FP32 storage of the field (tolerance studies only)."""
        self._L.orc_set_f32_storage(self._o, int(bool(on)))

    def set_impedance_rational(self, real=(), pairs=()):
        """Rational admittance of Eq. Yrational (Y_inf = 0): real = [(lam, A)],
        pairs = [(alpha, beta, B, C)] for poles alpha +- i beta, residues B +- i C."""
        n, lam, A, m, al, be, B, Cc = _poles(real, pairs)
        rc = self._L.orc_set_rational(self._o, n, _d(lam), _d(A), m, _d(al), _d(be), _d(B), _d(Cc))
        if rc:
            raise ValueError("rational admittance: 1..8 states")

    @property
    def n_states(self):
        return self._L.orc_n_states(self._o)

    def set_sponge(self, width, kappa=0.04):
        """Opt-in absorbing ramp over `width` outer layers (0 = off, the default);
        a departure from the paper, which adds no damping (Sec. 4.3)."""
        self._L.orc_set_sponge(self._o, int(width), float(kappa))

    def set_bf16_storage(self):
        """Emulate bfloat16 storage of the field (precision study only)."""
        self._L.orc_set_f32_storage(self._o, 2)

    def setup(self):
        rc = self._L.orc_setup(self._o)
        if rc:
            raise RuntimeError(self._L.orc_error(self._o).decode())
        return self

    @property
    def n_ghost(self):
        return self._L.orc_n_ghost(self._o)

    @property
    def n_reduced(self):
        return self._L.orc_n_reduced(self._o)

    @property
    def regime(self):
        return self._L.orc_regime(self._o)

    @property
    def step(self):
        return self._L.orc_get_step(self._o)

    def kind(self):
        out = np.empty(self.nx * self.ny, dtype=np.uint8)
        self._L.orc_get_kind(self._o, out.ctypes.data_as(C.POINTER(C.c_ubyte)))
        return out.reshape(self.ny, self.nx)

    def ghost(self, g):
        """Returns dict(target, bp, n, r, m, k, cloud, L ((m+1) x N), c, ct, ell);
        k is the degree of the cloud fit, m that of the normal extrapolation."""
        t = C.c_int(); m = C.c_int(); ncl = C.c_int()
        meta = np.empty(5)
        self._L.orc_ghost_meta(self._o, g, C.byref(t), _d(meta), C.byref(m), C.byref(ncl))
        N, mm = ncl.value, m.value
        cl = np.empty(N, dtype=np.int32)
        Lr = np.empty((mm + 1) * N)
        c = np.empty(5); ct = np.empty(5); ell = np.empty(5)
        self._L.orc_ghost_rows(self._o, g, cl.ctypes.data_as(_ip), _d(Lr), _d(c), _d(ct), _d(ell))
        return dict(target=t.value, bp=meta[0:2].copy(), n=meta[2:4].copy(), r=meta[4], m=mm,
                    k=int(self._L.orc_ghost_fit_degree(self._o, g)), cloud=cl, L=Lr.reshape(mm + 1, N), c=c[:mm + 1], ct=ct[:mm + 1], ell=ell[:mm + 1])

    # state
    def init_pulse(self, xs, ys, amp, halfwidth):
        self._L.orc_init_pulse(self._o, xs, ys, amp, halfwidth)

    def init_packet(self, xs, ys, angle, amp, k, alpha):
        self._L.orc_init_packet(self._o, xs, ys, angle, amp, k, alpha)

    def field(self, which):
        out = np.empty(self.nx * self.ny)
        self._L.orc_get_field(self._o, which, _d(out))
        return out.reshape(self.ny, self.nx)

    def set_field(self, which, arr):
        a = np.ascontiguousarray(arr, dtype=np.float64).reshape(-1)
        self._L.orc_set_field(self._o, which, _d(a))

    def ade(self):
        ns = self.n_states
        out = np.empty(ns * max(self.n_ghost, 1))
        self._L.orc_get_ade(self._o, _d(out))
        return out[:ns * self.n_ghost].reshape(-1, ns)

    def set_ade(self, X):
        a = np.ascontiguousarray(X, dtype=np.float64).reshape(-1)
        self._L.orc_set_ade(self._o, _d(a))

    def set_probes(self, xy, capacity):
        xy = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1)
        self._nprobe = len(xy) // 2
        return self._L.orc_set_probes(self._o, self._nprobe, _d(xy), capacity)

    def probes(self):
        n = self._nprobe
        if n == 0:
            return np.zeros((0, 0))
        buf = np.empty(max(1, self.step) * max(n, 1))
        rec = self._L.orc_get_probes(self._o, _d(buf))
        return buf[:rec * n].reshape(rec, n)

    def run(self, nsteps, classical=False):
        self._L.orc_run(self._o, nsteps, int(classical))

    def fill_ghosts(self):
        ns = self.n_states
        Xd = np.empty(ns * max(self.n_ghost, 1))
        self._L.orc_fill_ghosts(self._o, _d(Xd))
        return Xd[:ns * self.n_ghost].reshape(-1, ns)

    def fill_ghosts_bc(self, bc):
        """Ghost fill from given (w_BP, dp/dn_BP) per ghost (steps 4-5 only)."""
        a = np.ascontiguousarray(bc, dtype=np.float64).reshape(-1)
        self._L.orc_fill_ghosts_bc(self._o, _d(a))

    def eval_rhs(self, t):
        n = self.nx * self.ny
        rp, ru, rv = np.empty(n), np.empty(n), np.empty(n)
        ns = self.n_states
        Xd = np.empty(ns * max(self.n_ghost, 1))
        self._L.orc_eval_rhs(self._o, t, _d(rp), _d(ru), _d(rv), _d(Xd))
        sh = (self.ny, self.nx)
        return rp.reshape(sh), ru.reshape(sh), rv.reshape(sh), Xd[:ns * self.n_ghost].reshape(-1, ns)

    def energy(self):
        return self._L.orc_energy(self._o)
