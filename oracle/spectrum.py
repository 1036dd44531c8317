"""Spectral stability of the linear semi-discrete operator (TEST
INFRASTRUCTURE: an analysis tool built on the oracle, used by the tests).

The coupled system of Secs. 2-3 without a source is dQ/dt = L Q with
Q = (p, u, v at the fluid nodes; the ADE states of every ghost point).  L is
assembled here column by column from the oracle's right-hand side (steps 1-6
of Sec. 3.2 on a unit state), and its eigenvalues give the stability of the
semi-discrete scheme; the fully discrete four-stage scheme is stable when
every |P(lambda dt)| <= 1, P(z) = 1 + z + z^2/2 + z^3/6 + z^4/24.  The abstract
of the paper reports such an analysis for walls tangent to the grid.
"""
from __future__ import annotations

import numpy as np


def assemble(o):
    """Dense L of an oracle instance after setup (source off); returns
    (L, fluid mask, number of field unknowns)."""
    kind = o.kind().reshape(-1)
    fl = np.nonzero(kind == 1)[0]
    nf = len(fl)
    ns = o.n_states if o.n_ghost else 0
    nx = ns * o.n_ghost
    N = 3 * nf + nx
    L = np.zeros((N, N))
    n = o.nx * o.ny
    X0 = np.zeros(max(nx, 1))
    for col in range(N):
        fields = [np.zeros(n), np.zeros(n), np.zeros(n)]
        X = X0.copy()
        if col < 3 * nf:
            f, i = divmod(col, nf)
            fields[f][fl[i]] = 1.0
        else:
            X[col - 3 * nf] = 1.0
        for f in range(3):
            o.set_field(f, fields[f])
        if nx:
            o.set_ade(X[:nx])
        rp, ru, rv, Xd = o.eval_rhs(0.0)
        L[:3 * nf, col] = np.concatenate([rp.reshape(-1)[fl], ru.reshape(-1)[fl], rv.reshape(-1)[fl]])
        if nx:
            L[3 * nf:, col] = Xd.reshape(-1)
    return L, kind == 1, 3 * nf


def eigenvalues(o):
    L, _, _ = assemble(o)
    return np.linalg.eigvals(L)


def rk4_amplification(lam, dt):
    """|P(lambda dt)| of the four-stage scheme for every eigenvalue."""
    z = np.asarray(lam) * dt
    return np.abs(1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24)


def abscissa(lam):
    """Largest real part (the semi-discrete growth rate)."""
    return float(np.max(np.real(lam)))
