"""Central differences of J for one parameter on a window of the grid.

J = sum_s sum_i softplus(vref - v_{s,i} - margin)^2 over a backward-Euler RC
transient (Eq. 2) from a parameter-independent DC point v_0 = Vdd.  Perturbing
one resistor or capacitor by sigma eps changes M = C/h + G + G0 (and C) by a
rank-one term; the change of the trajectory, dv_s = v'_s - v_s, solves the
exact recurrence

    (M + dM) dv_s = ((C + dC)/h) dv_{s-1} - dM v_s + (dC/h) v_{s-1},   dv_0 = 0,

for a resistor (a, b): dM = sigma eps (e_a - e_b)(e_a - e_b)^T, dC = 0, and for a
capacitor at node i: dM = dC/h = (sigma eps / h) e_i e_i^T.  Its only sources sit
at the parameter's nodes, and the pads to the supply make the response decay
about twofold every four lattice nodes on the recipe's single-layer meshes, so
dv is solved on a box of half-width R around the parameter with dv = 0 outside
(direct sparse LU).  The change of J is formed per term without cancellation:
with d = softplus(u - dv) - softplus(u) = log1p(sigmoid(u) expm1(-dv)),

    softplus(u - dv+)^2 - softplus(u - dv-)^2 = (d+ - d-) (2 softplus(u) + d+ + d-),

and the central difference is the sum over terms divided by 2 eps.  The
trajectory v comes from the caller (the GPU's, or the oracle's in the pin).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def window_nodes(lattice, node, R):
    """Node ids (all layers) of the box of half-width R around ``node``'s (x, y)."""
    nx, ny, nl = lattice
    x0, y0 = node % nx, (node // nx) % ny
    xs = np.arange(max(0, x0 - R), min(nx, x0 + R + 1))
    ys = np.arange(max(0, y0 - R), min(ny, y0 + R + 1))
    l, y, x = np.meshgrid(np.arange(nl), ys, xs, indexing="ij")
    return ((l * ny + y) * nx + x).ravel()


def _softplus(u):
    return np.logaddexp(0.0, u)


def _sigmoid(u):
    return 0.5 * (1.0 + np.tanh(0.5 * u))


def central_difference(Mw, chw, V, v0, kind, nodes, eps, h, vref=1.0, margin=0.05):
    """(J(p + eps) - J(p - eps)) / (2 eps) for one parameter, on one window.

    Mw: the window's block of the system matrix (sparse), chw: its C/h diagonal,
    V: (S, n) trajectory on the window (steps 1..S), v0: the window's DC point.
    kind "r": resistor between window-local ``nodes`` = (ia, ib); "c": capacitor
    at window-local ``nodes`` = (i,).  dM = c u u^T with u = e_a - e_b or e_i is
    rank one, so one LU of Mw serves both signs (Sherman-Morrison)."""
    S, n = V.shape
    lu = spla.splu(sp.csc_matrix(Mw), permc_spec="MMD_AT_PLUS_A")
    u = np.zeros(n)
    if kind == "r":
        ia, ib = nodes
        u[ia], u[ib] = 1.0, -1.0
        cs = np.array([eps, -eps])                 # dM = c u u^T
    else:
        (i,) = nodes
        u[i] = 1.0
        cs = np.array([eps, -eps]) / h             # dM = dC/h = c e_i e_i^T
    z = lu.solve(u)
    uz = float(u @ z)
    dv = np.zeros((n, 2))
    dj = 0.0
    for s in range(S):
        vs = V[s]
        if kind == "r":
            drive = vs[ia] - vs[ib]
        else:
            drive = vs[i] - (V[s - 1][i] if s > 0 else v0[i])
        rhs = chw[:, None] * dv
        if kind == "c":
            rhs[i] += cs * dv[i]                     # (C + dC)/h dv_{s-1}
        rhs -= np.outer(u, cs * drive)               # -dM v_s (+ dC/h v_{s-1})
        y = lu.solve(rhs)
        dv = y - np.outer(z, cs * (u @ y) / (1.0 + cs * uz))
        uu = vref - vs - margin
        spu, sig = _softplus(uu), _sigmoid(uu)
        dp = np.log1p(sig * np.expm1(-dv[:, 0]))
        dm = np.log1p(sig * np.expm1(-dv[:, 1]))
        dj += float(np.sum((dp - dm) * (2.0 * spu + dp + dm)))
    return dj / (2.0 * eps)


def parameter_window(M, c_over_h, lattice, kind, terminals, R):
    """(window node ids, Mw, chw, window-local terminal indices) of one parameter."""
    win = window_nodes(lattice, int(terminals[0]), R)
    pos = {int(g): k for k, g in enumerate(win)}
    return win, M[win][:, win], np.asarray(c_over_h)[win], tuple(pos[int(t)] for t in terminals)
