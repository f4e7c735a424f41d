"""The paper's topology-based node update, natural ordering, pure Python.

Section IV-A.  KCL at a representative node ``i`` (Eq. 12) with resistor
neighbours ``N_i^R``, inductor neighbours ``N_i^L``, load ``I_i`` and
grounded capacitance ``C_i``.  A neighbour may be a source node (its voltage
is the fixed ``V_dd`` of that source) or ground (0 V).  Nothing here builds a
matrix: each node reads its own element lists, which is the "no matrix
construction" property the paper claims for Algorithm 1.

Two per-node fixed-point forms ``V_i = sum_j w_ij V_j + K_i`` (Eq. 15):

* explicit inductor currents (backward Euler of Eq. 12 with
  ``I_ij(t+h) = I_ij(t) + (h/L_ij)(V_i - V_j)(t+h)``):
  ``(sum g + sum h/L + C/h) V_i = sum g V_j + sum (h/L) V_j
  + (C/h) V_i(t) - sum I_ij(t) - I_i(t+h)``
* the three-level form of Eq. 14 (Eq. 13 discretised):
  ``(sum g + h sum 1/L + C/h) V_i(t+h) = sum g V_j(t+h) + sum (h/L) V_j(t+h)
  + (2C/h + sum g) V_i(t) - sum g V_j(t) - I_i(t+h) + I_i(t) - (C/h) V_i(t-h)``

The iteration is Gauss-Seidel in natural index order (Eq. 16) with the SOR
blend of Eq. 17, stopped when ``max |V^(k) - V^(k-1)| < tol`` (Algorithm 1).
"""
from __future__ import annotations

import numpy as np

from .pwl import pwl_values


class NodeTopology:
    """Per-node element lists read straight from the netlist."""

    def __init__(self, net):
        n = net.n_nodes
        self.n = n
        self.vd = np.asarray(net.vdd, float)
        self.R = [[] for _ in range(n)]    # (other terminal, g)
        self.L = [[] for _ in range(n)]    # (other terminal, L, branch, sign)
        self.I = [[] for _ in range(n)]    # (source index, sign): +1 when the current leaves i
        self.C = np.zeros(n)
        for a, b, g in zip(net.r_a, net.r_b, net.r_g):
            if a >= 0:
                self.R[a].append((int(b), float(g)))
            if b >= 0:
                self.R[b].append((int(a), float(g)))
        for e, (a, b, l) in enumerate(zip(net.l_a, net.l_b, net.l_val)):
            if a >= 0:
                self.L[a].append((int(b), float(l), e, +1.0))
            if b >= 0:
                self.L[b].append((int(a), float(l), e, -1.0))
        for a, b, c in zip(net.c_a, net.c_b, net.c_val):
            if a >= 0 and b < 0:
                self.C[a] += c
            elif b >= 0 and a < 0:
                self.C[b] += c
            else:
                raise ValueError("node-to-node capacitors are outside the per-node form of Eq. 12")
        for e, (a, b) in enumerate(zip(net.i_a, net.i_b)):
            if a >= 0:
                self.I[a].append((e, +1.0))
            if b >= 0:
                self.I[b].append((e, -1.0))
        self.net = net

    def volt(self, term: int, v: np.ndarray) -> float:
        if term >= 0:
            return v[term]
        if term == -1:
            return 0.0
        return self.vd[-2 - term]

    def injected(self, t: float) -> np.ndarray:
        """``I_i(t)``: total load current leaving each node."""
        vals = pwl_values(self.net.i_ptr, self.net.i_t, self.net.i_v, t)
        out = np.zeros(self.n)
        for i in range(self.n):
            for e, sgn in self.I[i]:
                out[i] += sgn * vals[e]
        return out


def _sweep_until(topo: NodeTopology, diag, K, nbr, v, omega, tol, max_iter):
    """Gauss-Seidel / SOR (Eq. 16-17) on ``diag_i V_i = sum_j c_ij V_j + K_i``."""
    for k in range(1, max_iter + 1):
        delta = 0.0
        for i in range(topo.n):
            acc = K[i]
            for (j, c) in nbr[i]:
                acc += c * (v[j] if j >= 0 else topo.volt(j, v))
            vt = acc / diag[i]
            vn = omega * vt + (1.0 - omega) * v[i]
            delta = max(delta, abs(vn - v[i]))
            v[i] = vn
        if delta < tol:
            return v, k
    raise RuntimeError(f"Gauss-Seidel did not reach tol={tol} in {max_iter} sweeps")


def gs_step_explicit(topo: NodeTopology, h, v_prev, il_prev, t, omega=1.0, tol=1e-13,
                     max_iter=200000, v_init=None):
    """One BE step in the explicit-inductor-current node form.  Returns ``(v, il, sweeps)``."""
    n = topo.n
    I_now = topo.injected(t)
    diag = np.zeros(n); K = np.zeros(n); nbr = [[] for _ in range(n)]
    for i in range(n):
        d = topo.C[i] / h
        k = topo.C[i] / h * v_prev[i] - I_now[i]
        for j, g in topo.R[i]:
            d += g
            if j >= 0:
                nbr[i].append((j, g))
            else:
                k += g * topo.volt(j, v_prev)
        for j, l, e, sgn in topo.L[i]:
            d += h / l
            if j >= 0:
                nbr[i].append((j, h / l))
            else:
                k += h / l * topo.volt(j, v_prev)
            k -= sgn * il_prev[e]          # current leaving i through inductor e at time t
        diag[i] = d; K[i] = k
    v = np.array(v_prev if v_init is None else v_init, dtype=float)
    v, sweeps = _sweep_until(topo, diag, K, nbr, v, omega, tol, max_iter)
    il = np.array(il_prev, dtype=float)
    net = topo.net
    for e, (a, b, l) in enumerate(zip(net.l_a, net.l_b, net.l_val)):
        il[e] = il_prev[e] + h / l * (topo.volt(int(a), v) - topo.volt(int(b), v))
    return v, il, sweeps


def gs_step_three_level(topo: NodeTopology, h, v_prev, v_prev2, t, omega=1.0, tol=1e-13,
                        max_iter=200000):
    """One step of Eq. 14 (three-level form), solved by Eq. 16-17."""
    n = topo.n
    I_now = topo.injected(t)
    I_old = topo.injected(t - h)
    diag = np.zeros(n); K = np.zeros(n); nbr = [[] for _ in range(n)]
    for i in range(n):
        sg = sum(g for _, g in topo.R[i])
        d = sg + topo.C[i] / h
        k = (2.0 * topo.C[i] / h + sg) * v_prev[i] - topo.C[i] / h * v_prev2[i] \
            - I_now[i] + I_old[i]
        for j, g in topo.R[i]:
            k -= g * topo.volt(j, v_prev)
            if j >= 0:
                nbr[i].append((j, g))
            else:
                k += g * topo.volt(j, v_prev)          # a source neighbour at t+h
        for j, l, e, sgn in topo.L[i]:
            d += h / l
            if j >= 0:
                nbr[i].append((j, h / l))
            else:
                k += h / l * topo.volt(j, v_prev)
        diag[i] = d; K[i] = k
    v = np.array(v_prev, dtype=float)
    v, sweeps = _sweep_until(topo, diag, K, nbr, v, omega, tol, max_iter)
    return v, sweeps


def gs_dc(topo: NodeTopology, t=0.0, il0=None, omega=1.0, tol=1e-13, max_iter=200000, v_init=None):
    """DC operating point by the same node update, capacitors open and inductors as
    current sources ``i_l(0)`` (first step of the initial-condition procedure)."""
    n = topo.n
    I_now = topo.injected(t)
    il0 = np.zeros(len(topo.net.l_val)) if il0 is None else il0
    diag = np.zeros(n); K = np.zeros(n); nbr = [[] for _ in range(n)]
    for i in range(n):
        d = 0.0
        k = -I_now[i]
        for j, g in topo.R[i]:
            d += g
            if j >= 0:
                nbr[i].append((j, g))
            else:
                k += g * topo.volt(j, np.zeros(n))
        for j, l, e, sgn in topo.L[i]:
            k -= sgn * il0[e]
        diag[i] = d; K[i] = k
    v = np.full(n, float(np.mean(topo.vd)) if v_init is None else 0.0)
    if v_init is not None:
        v[:] = v_init
    return _sweep_until(topo, diag, K, nbr, v, omega, tol, max_iter)
