"""Backward-Euler transient of RC and RLC power grids (FP64, direct solves).

Derivation followed (Section III-A; source-term signs taken from KVL, Eq. 7,
``v_b = A v_n + A_s v_d``, because the printed Eq. 9-10 carry the opposite
sign on ``G_s v_d`` and ``A_ls v_d`` and would drive the grid to ``-Vdd``):

    C dv/dt + G v + A_l^T i_l + A_i^T I_s + G_s v_d = 0          (Eq. 9, line 1)
    Ldiag di_l/dt = A_l v + A_ls v_d                             (Eq. 9, line 2)

Backward Euler (Eq. 10) with step ``h`` and the inductor current kept as a
state variable gives, with ``M = C/h + G + h L`` (Eq. 11's system matrix):

    M v(t+h) = (C/h) v(t) - A_l^T i_l(t) - A_i^T I_s(t+h) - G_s v_d - h L_s v_d
    i_l(t+h) = i_l(t) + h Ldiag^-1 (A_l v(t+h) + A_ls v_d)

and without inductors this is Eq. 2 with the pads inside ``G`` and the
``G_0 V_dd`` term equal to ``-G_s v_d``.  Subtracting the line-1 equation at
``t`` from the one at ``t+h`` eliminates ``i_l`` and gives the three-level
form of Eq. 11:

    M v(t+h) = (2C/h + G) v(t) - (C/h) v(t-h) - A_i^T (I_s(t+h) - I_s(t)) - h L_s v_d

Initial conditions (Section IV-B): the DC operating point at ``t = 0`` with
the capacitors carrying no current and every inductor acting as a current
source of value ``i_l(0)`` (default 0):

    G v(0) = -A_i^T I_s(0) - G_s v_d - A_l^T i_l(0)

The first transient step is an ordinary backward-Euler step from
``(v(0), i_l(0))``; the paper's explicit half-step (its step 2) is replaced by
this consistent BE step.  The paper's own three-step procedure (DC with the
capacitors as voltage sources, a forward update of ``v_c`` and ``i_l``, DC at
``h``), which yields the two levels ``v(0)``, ``v(h)`` of the three-level
form, is :func:`paper_initial_conditions`.

Solves are direct: a dense Cholesky for tiny systems, otherwise a sparse LU
factorisation (SuperLU, symmetric minimum-degree ordering) computed once per
``h``.  The system matrix is SPD (Lemma 1), so both are exact up to rounding.
"""
from __future__ import annotations

from typing import Iterator, Optional, Tuple

import numpy as np
import scipy.linalg as sla_dense
import scipy.sparse as sp
import scipy.sparse.linalg as sla

from .matrices import NodalMatrices, nodal_matrices
from .pwl import pwl_values

DENSE_MAX = 2000


class DirectSolver:
    """Factor an SPD matrix once, solve many right-hand sides."""

    def __init__(self, M):
        n = M.shape[0]
        self.n = n
        if n <= DENSE_MAX:
            self.kind = "dense-cholesky"
            self._c = sla_dense.cho_factor(np.asarray(M.todense()), lower=True)
        else:
            self.kind = "sparse-lu"
            self._lu = sla.splu(sp.csc_matrix(M), permc_spec="MMD_AT_PLUS_A")

    def solve(self, b: np.ndarray) -> np.ndarray:
        if self.kind == "dense-cholesky":
            return sla_dense.cho_solve(self._c, b)
        return self._lu.solve(np.asarray(b, dtype=np.float64))


def load_current(net, mats: NodalMatrices, t: float) -> np.ndarray:
    """``A_i^T I_s(t)``: the load current leaving each trivial node."""
    return mats.A_i.T @ pwl_values(net.i_ptr, net.i_t, net.i_v, t)


def source_terms(mats: NodalMatrices, h: float) -> np.ndarray:
    """``-G_s v_d - h L_s v_d``: the constant injection from the source nodes."""
    return -(mats.G_s @ mats.vd) - h * (mats.L_s @ mats.vd)


def dc_operating_point(net, mats: Optional[NodalMatrices] = None, il0=None, t: float = 0.0):
    """DC solution ``G v = -A_i^T I_s(t) - G_s v_d - A_l^T i_l(0)``."""
    mats = mats or nodal_matrices(net)
    rhs = -load_current(net, mats, t) - mats.G_s @ mats.vd
    if il0 is not None and mats.A_l.shape[0]:
        rhs = rhs - mats.A_l.T @ il0
    return DirectSolver(mats.G).solve(rhs)


def simulate(net, h: float, nsteps: int, v0=None, il0=None,
             mats: Optional[NodalMatrices] = None, s0: int = 0) -> Iterator[Tuple[int, np.ndarray, np.ndarray]]:
    """Yield ``(s, v(s), i_l(s))`` for ``s = 0 .. nsteps`` (explicit-i_l form).

    ``s0`` shifts the time axis: the given state is the one at ``t = s0 h`` and
    step ``s`` lands at ``t = (s0 + s) h``."""
    mats = mats or nodal_matrices(net)
    m_l = mats.A_l.shape[0]
    il = np.zeros(m_l) if il0 is None else np.asarray(il0, dtype=np.float64).copy()
    v = dc_operating_point(net, mats, il) if v0 is None else np.asarray(v0, dtype=np.float64).copy()
    yield 0, v, il
    M = mats.system_matrix(h)
    solver = DirectSolver(M)
    Ch = mats.C / h
    const = source_terms(mats, h)
    for s in range(1, nsteps + 1):
        t = (s0 + s) * h
        rhs = Ch @ v - load_current(net, mats, t) + const
        if m_l:
            rhs -= mats.A_l.T @ il
        v = solver.solve(rhs)
        if m_l:
            il = il + h * mats.Ldiag_inv * (mats.A_l @ v + mats.A_ls @ mats.vd)
        yield s, v, il


def transient(net, h: float, nsteps: int, v0=None, il0=None, s0: int = 0) -> Tuple[np.ndarray, np.ndarray]:
    """Full waveforms ``V[s, node]`` and ``IL[s, inductor]``, ``s = 0..nsteps``."""
    vs, ils = [], []
    for _, v, il in simulate(net, h, nsteps, v0, il0, s0=s0):
        vs.append(v); ils.append(il)
    return np.stack(vs), np.stack(ils)


def simulate_three_level(net, h: float, nsteps: int, v0: np.ndarray, v1: np.ndarray,
                         mats: Optional[NodalMatrices] = None):
    """Eq. 11 literally: needs ``v(0)`` and ``v(1)``; yields ``(s, v(s))`` for ``s >= 2``.

    ``v(0)`` and ``v(1)`` come from the initial-condition procedure
    (Section IV-B); Algorithm 1 starts its loop at ``s = 2``.
    """
    mats = mats or nodal_matrices(net)
    solver = DirectSolver(mats.system_matrix(h))
    A = (2.0 * mats.C / h + mats.G).tocsr()
    Ch = mats.C / h
    const = -h * (mats.L_s @ mats.vd)
    vm, vc = np.asarray(v0, float), np.asarray(v1, float)
    for s in range(2, nsteps + 1):
        dI = load_current(net, mats, s * h) - load_current(net, mats, (s - 1) * h)
        rhs = A @ vc - Ch @ vm - dI + const
        vn = solver.solve(rhs)
        yield s, vn
        vm, vc = vc, vn


def _dc_with_fixed_caps(mats: NodalMatrices, net, t: float, v_cap: np.ndarray, capped: np.ndarray,
                        il: np.ndarray):
    """One DC analysis of the initial-condition procedure (Section IV-B, steps 1
    and 3): every node that carries a capacitor is held at ``v_cap`` (the
    capacitors act as voltage sources), every inductor acts as a current source
    of value ``il``; the remaining nodes solve their rows of
    ``G v = -G_s v_d - A_i^T I_s(t) - A_l^T i_l``.  Returns ``v`` and the
    capacitor currents ``i_c = -(G v + G_s v_d + A_i^T I_s(t) + A_l^T i_l)``
    (zero on nodes without a capacitor)."""
    n = mats.n
    rest = -(mats.G_s @ mats.vd) - load_current(net, mats, t)
    if mats.A_l.shape[0]:
        rest = rest - mats.A_l.T @ il
    v = np.where(capped, v_cap, 0.0)
    free = ~capped
    if free.any():
        G = mats.G.tocsr()
        Gff = G[free][:, free]
        Gfc = G[free][:, capped]
        b = rest[free] - Gfc @ v[capped]
        v[free] = DirectSolver(Gff.tocsc()).solve(b)
    i_c = np.where(capped, -(mats.G @ v) + rest, 0.0)
    return v, i_c


def paper_initial_conditions(net, h: float, vc0=None, il0=None, mats: Optional[NodalMatrices] = None):
    """The three-step initial-condition procedure of Section IV-B.

    1. DC at t = 0 with capacitors as voltage sources ``v_c(0)`` and inductors
       as current sources ``i_l(0)``: gives ``v(0)``, the capacitor currents
       ``i_c(0)`` and the inductor voltages ``v_l(0) = A_l v(0) + A_ls v_d``.
    2. ``v_c(h) = v_c(0) + h i_c(0) / C`` and ``i_l(h) = i_l(0) + h v_l(0) / L``.
    3. DC at t = h with capacitors as voltage sources ``v_c(h)`` and inductors
       as current sources ``i_l(h)``: gives ``v(h)``.

    ``vc0`` holds one voltage per capacitor element (netlist order; parallel
    capacitors on one node must agree); None takes the DC operating point with
    the capacitors open.  ``il0`` defaults to zero.  Returns
    ``(v(0), v(h), i_l(h))``, the two levels the three-level form (Eq. 11)
    starts from, with the inductor currents the explicit form needs."""
    mats = mats or nodal_matrices(net)
    n = mats.n
    m_l = mats.A_l.shape[0]
    il = np.zeros(m_l) if il0 is None else np.asarray(il0, dtype=np.float64).copy()
    cdiag = mats.C.diagonal()
    capped = cdiag > 0.0
    ca, cb = np.asarray(net.c_a), np.asarray(net.c_b)
    cnode = np.where(ca >= 0, ca, cb)
    if vc0 is None:
        vdc = dc_operating_point(net, mats, il)
        v_cap = np.where(capped, vdc, 0.0)
    else:
        vc0 = np.asarray(vc0, dtype=np.float64)
        v_cap = np.zeros(n)
        v_cap[cnode[::-1]] = vc0[::-1]          # the first capacitor of a node wins
        if not np.allclose(v_cap[cnode], vc0, rtol=0.0, atol=0.0):
            raise ValueError("parallel capacitors on one node need one voltage")
    v0, i_c = _dc_with_fixed_caps(mats, net, 0.0, v_cap, capped, il)
    if m_l:
        v_l = mats.A_l @ v0 + mats.A_ls @ mats.vd
        il1 = il + h * mats.Ldiag_inv * v_l
    else:
        il1 = il
    v_cap1 = np.where(capped, v_cap + h * np.divide(i_c, cdiag, out=np.zeros(n), where=capped), 0.0)
    v1, _ = _dc_with_fixed_caps(mats, net, h, v_cap1, capped, il1)
    return v0, v1, il1
