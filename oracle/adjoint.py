"""Discrete adjoint of the backward-Euler RC transient (FP64, direct solves).

The paper has no adjoint; this is the exact gradient of the discrete
recurrence the paper solves (Eq. 2 / Eq. 10 with L = 0), for the objective

    J = sum_{s=1..S} sum_i softplus(V_ref - v_{s,i} - margin)^2

(worst IR drop beyond a margin).  With F_s = M v_s - (C/h) v_{s-1} - b_s = 0,
b_s = -A_i^T I_s(t_s) - G_s v_d, and the DC point G v_0 = b_0 (capacitors open),
the Lagrangian gives the backward recurrence

    M lambda_s = dJ/dv_s + (C/h) lambda_{s+1},   lambda_{S+1} = 0,
    G mu       = (C/h) lambda_1                    (adjoint of the DC point)

and the parameter gradients (inductors: see :func:`gradients`)

    dJ/dg_e = -sum_s (lambda_{s,a} - lambda_{s,b}) (v_{s,a} - v_{s,b}) - (mu_a - mu_b)(v_{0,a} - v_{0,b})
    dJ/dC_k = -sum_s lambda_{s,k} (v_{s,k} - v_{s-1,k}) / h

for a resistor e = (a, b) (a terminal that is a source or ground has lambda = mu = 0
and its fixed voltage) and a grounded capacitor on node k.
"""
from __future__ import annotations

import numpy as np

from .matrices import nodal_matrices
from .transient import DirectSolver, dc_operating_point, simulate


def softplus(u):
    return np.logaddexp(0.0, u)


def sigmoid(u):
    return 0.5 * (1.0 + np.tanh(0.5 * u))


def objective_terms(v, vref, margin):
    u = vref - v - margin
    return softplus(u) ** 2


def objective(net, h, nsteps, vref=1.0, margin=0.05) -> float:
    """J by the forward recurrence (math.fsum over per-step sums)."""
    import math
    parts = []
    for s, v, _ in simulate(net, h, nsteps):
        if s > 0:
            parts.append(math.fsum(objective_terms(v, vref, margin)))
    return math.fsum(parts)


def _term_voltage(t, v, vd):
    return np.where(t >= 0, v[np.maximum(t, 0)], np.where(t == -1, 0.0, vd[np.maximum(-2 - t, 0)]))


def _term_adjoint(t, lam):
    return np.where(t >= 0, lam[np.maximum(t, 0)], 0.0)


def gradients(net, h, nsteps, vref=1.0, margin=0.05, with_l=False):
    """Return ``(J, dJ/dg per resistor, dJ/dC per capacitor)``, plus ``dJ/dL per
    inductor`` when ``with_l`` (grids with inductors need it).

    With inductors the explicit form (Eq. 10) has two constraint families,
    ``F_s = M v_s - (C/h) v_(s-1) + A_l^T i_(s-1) + A_i^T I_s + G_s v_d + h L_s v_d``
    and ``H_s = i_s - i_(s-1) - h Ldiag^-1 u_s`` with ``u_s = A_l v_s + A_ls v_d``.
    Their multipliers obey

        mu_s     = mu_(s+1) - A_l lambda_(s+1)                       (mu_S = 0)
        M lambda_s = dJ/dv_s + (C/h) lambda_(s+1) + h A_l^T Ldiag^-1 mu_s

    and ``dJ/dL_e = (h / L_e^2) sum_s u_(s,e) ((A_l lambda_s)_e - mu_(s,e))``; the
    resistor and capacitor gradients keep their RC form.  The DC point (inductors
    carrying i_l(0) = 0) does not depend on L."""
    mats = nodal_matrices(net)
    m_l = mats.A_l.shape[0]
    if m_l and not with_l:
        raise ValueError("grids with inductors: call with with_l=True")
    V = [v for _, v, _ in simulate(net, h, nsteps, mats=mats)]
    V = np.stack(V)                                   # [S+1, n]
    M = mats.system_matrix(h)
    solver = DirectSolver(M)
    Ch = mats.C.diagonal() / h
    vd = mats.vd
    ra, rb = np.asarray(net.r_a), np.asarray(net.r_b)
    ca = np.asarray(net.c_a)
    cnode = np.where(ca >= 0, ca, np.asarray(net.c_b))
    Lval = np.asarray(net.l_val, dtype=np.float64)
    A_l = mats.A_l.tocsr()
    dG = np.zeros(len(net.r_g))
    dC = np.zeros(len(net.c_val))
    dL = np.zeros(m_l)
    J = 0.0
    lam_next = np.zeros(net.n_nodes)
    mu_next = np.zeros(m_l)
    for s in range(nsteps, 0, -1):
        v = V[s]
        u = vref - v - margin
        J += float(np.sum(softplus(u) ** 2))
        dJdv = -2.0 * softplus(u) * sigmoid(u)
        rhs = dJdv + Ch * lam_next
        if m_l:
            mu = mu_next - A_l @ lam_next
            rhs = rhs + h * (A_l.T @ (mats.Ldiag_inv * mu))
        lam = solver.solve(rhs)
        dG -= (_term_adjoint(ra, lam) - _term_adjoint(rb, lam)) * (_term_voltage(ra, v, vd) - _term_voltage(rb, v, vd))
        dC -= lam[cnode] * (V[s][cnode] - V[s - 1][cnode]) / h
        if m_l:
            ub = A_l @ v + mats.A_ls @ vd
            dL += h / Lval ** 2 * ub * (A_l @ lam - mu)
            mu_next = mu
        lam_next = lam
    # DC point: G v_0 = b_0 depends on the resistors
    nu = DirectSolver(mats.G.tocsc()).solve(Ch * lam_next)
    v0 = V[0]
    dG -= (_term_adjoint(ra, nu) - _term_adjoint(rb, nu)) * (_term_voltage(ra, v0, vd) - _term_voltage(rb, v0, vd))
    if with_l:
        return J, dG, dC, dL
    return J, dG, dC
