"""Multicore CPU baseline: red-black SOR of the paper's node update on all host cores.

TEST AND BENCHMARK INFRASTRUCTURE ONLY.  This is the paper's relaxation
(Eq. 16 with the SOR blend of Eq. 17; Algorithm 1's step loop) run on the CPU.
The sweep is in C with OpenMP (``rbsor.c``).  It solves the same
backward-Euler steps as the GPU library, under the same certified stopping
rule, and is timed beside it.  It shares no code with the CUDA library.
Parity tests use the direct solves of ``transient``, not this module.

Stopping rule: ``M`` is an M-matrix (Lemma 1), so the error of a step is at
most ``kappa max_i |r_i| / D_i`` with ``kappa = ||M^-1 D||_inf``.  Step errors
accumulate by at most ``kacc = ||1 + G^-1 (C/h) 1||_inf`` (RC).  Each step
stops once ``kappa R <= 0.9 tol / kacc``.  ``kappa`` and ``kacc`` come from
the direct solves of ``bounds`` (setup, not timed).

Ordering and relaxation factor: the nodes are 2-coloured by a breadth-first
search over the couplings; lattice grids, vias included, are bipartite.  The
relaxation factor is Young's, from a power-iteration estimate of the Jacobi
radius, with ``omega - 1`` taken 1 % high.  This is the same rule as the GPU
library, stated here independently.

On lattice netlists the column-block form (``block=True``) relaxes whole
``(x, y)`` columns.  Each column's layers, coupled by the vias, are solved
exactly, with columns coloured by the parity of ``x + y``.  That is the
algorithm of the GPU's lattice inner solve, so the two can be compared on the
same iteration.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import time

import numpy as np
import scipy.sparse as sp
from scipy.sparse.csgraph import breadth_first_order

from . import bounds
from .matrices import nodal_matrices
from .transient import dc_operating_point, load_current, source_terms

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "rbsor.c")
LIB = os.path.join(HERE, "_build", "librbsor.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``rbsor.c`` with gcc and OpenMP (in-tree, ``oracle/_build``)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        os.makedirs(os.path.dirname(LIB), exist_ok=True)
        tmp = LIB + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", SRC, "-o", tmp, "-lm"], check=True)
        os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P = C.POINTER
        _lib.rbsor_step.restype = C.c_int
        _lib.rbsor_step.argtypes = [C.c_int, P(C.c_int), P(C.c_int), P(C.c_double), P(C.c_double), P(C.c_int),
                                    C.c_int, P(C.c_double), P(C.c_double), C.c_double, C.c_double, C.c_int,
                                    C.c_int, P(C.c_double)]
        _lib.rbsor_block_step.restype = C.c_int
        _lib.rbsor_block_step.argtypes = [C.c_int, C.c_int, C.c_int] + [P(C.c_double)] * 8 + \
            [C.c_double, C.c_double, C.c_int, C.c_int, P(C.c_double)]
        _lib.rbsor_threads.restype = C.c_int
        _lib.rbsor_set_threads.argtypes = [C.c_int]
    return _lib


def set_threads(t: int) -> None:
    """OpenMP threads of the sweeps (the default is every core the process may use)."""
    lib().rbsor_set_threads(int(t))


def two_colouring(W: sp.csr_matrix) -> np.ndarray:
    """Colour 0/1 per node with no coupling inside a colour (breadth-first search
    over every connected part); raises ValueError if the couplings are not bipartite."""
    n = W.shape[0]
    colour = np.full(n, -1, np.int8)
    for root in range(n):
        if colour[root] >= 0:
            continue
        order, pred = breadth_first_order(W, root, directed=False, return_predecessors=True)
        colour[root] = 0
        for v in order[1:]:
            colour[v] = 1 - colour[pred[v]]
    rows, cols = W.nonzero()
    if np.any(colour[rows] == colour[cols]):
        raise ValueError("the coupling graph is not bipartite: red-black ordering does not apply")
    return colour


def jacobi_radius(D: np.ndarray, W: sp.csr_matrix, iters: int = 300, seed: int = 0) -> float:
    """Rayleigh-quotient estimate (a lower bound) of rho(D^-1 W), from power iteration
    on the shifted symmetric form (I + D^-1/2 W D^-1/2) / 2; the shift keeps the -rho
    eigenvalue of a bipartite graph from cancelling the +rho one."""
    s = 1.0 / np.sqrt(D)
    S = sp.diags(s) @ W @ sp.diags(s)
    x = np.random.default_rng(seed).uniform(0.5, 1.0, D.size)
    x /= np.linalg.norm(x)
    mu = 0.0
    for _ in range(iters):
        y = 0.5 * (x + S @ x)
        mu = float(x @ y)
        x = y / np.linalg.norm(y)
    return 2.0 * mu - 1.0


class StepSystem:
    """One h: the CSR couplings, diagonal, colour order and relaxation factor."""

    def __init__(self, net, h: float, mats=None):
        self.mats = mats or nodal_matrices(net)
        M = self.mats.system_matrix(h).tocsr()
        self.D = M.diagonal().copy()
        W = (sp.diags(self.D) - M).tocsr()
        W.eliminate_zeros()
        W.sort_indices()
        self.W = W
        colour = two_colouring(W)
        self.order = np.concatenate([np.nonzero(colour == 0)[0], np.nonzero(colour == 1)[0]]).astype(np.int32)
        self.n_first = int(np.sum(colour == 0))
        self.rowptr = W.indptr.astype(np.int32)
        self.col = W.indices.astype(np.int32)
        self.w = W.data.astype(np.float64)
        self.rho = min(jacobi_radius(self.D, W), 1.0 - 1e-12)
        young = 2.0 / (1.0 + np.sqrt(1.0 - self.rho ** 2))
        self.omega = min(1.0 + 1.01 * (young - 1.0), 0.5 * (young + 2.0))

    def solve(self, b: np.ndarray, x: np.ndarray, target: float, max_sweeps: int = 20000,
              check_every: int = 4) -> int:
        """Relax ``x`` in place until ``max |r| / D <= target``; returns the sweeps used."""
        P = C.POINTER
        R = C.c_double(0.0)
        k = lib().rbsor_step(self.D.size, self.rowptr.ctypes.data_as(P(C.c_int)),
                             self.col.ctypes.data_as(P(C.c_int)), self.w.ctypes.data_as(P(C.c_double)),
                             self.D.ctypes.data_as(P(C.c_double)), self.order.ctypes.data_as(P(C.c_int)),
                             self.n_first, b.ctypes.data_as(P(C.c_double)), x.ctypes.data_as(P(C.c_double)),
                             float(self.omega), float(target), int(max_sweeps), int(check_every), C.byref(R))
        if k < 0:
            raise RuntimeError(f"red-black SOR did not converge (status {k}, residual {R.value:.3e})")
        return k


class LatticeSystem:
    """One h on a lattice netlist, for the column-block form: the couplings by direction
    (+x, +y, +l), the diagonal, each column block's elimination factors and omega.

    A column block is the tridiagonal system of one (x, y) column's layers (the vias).
    Its elimination uses pivots ``p_0 = D_0`` and ``p_l = D_l - wU_(l-1) m_l``, with
    multipliers ``m_l = wU_(l-1) / p_(l-1)``."""

    def __init__(self, net, h: float, mats=None):
        if net.lattice is None:
            raise ValueError("the column-block form needs a lattice netlist")
        nx, ny, nl = net.lattice
        self.nx, self.ny, self.nl = nx, ny, nl
        plane, n = nx * ny, nx * ny * nl
        self.mats = mats or nodal_matrices(net)
        M = self.mats.system_matrix(h).tocoo()
        self.D = np.zeros(n)
        self.D[M.row[M.row == M.col]] = M.data[M.row == M.col]
        up = M.col > M.row
        r, c, w = M.row[up], M.col[up], -M.data[up]
        d = c - r
        east = (d == 1) & (r % nx != nx - 1)
        north = (d == nx) & ((r // nx) % ny != ny - 1)
        via = d == plane
        if not np.all(east | north | via):
            raise ValueError("a coupling joins nodes that are not lattice neighbours")
        self.wE, self.wN, self.wU = np.zeros(n), np.zeros(n), np.zeros(n)
        self.wE[r[east]] = w[east]
        self.wN[r[north]] = w[north]
        self.wU[r[via]] = w[via]
        Dl, Ul = self.D.reshape(nl, plane), self.wU.reshape(nl, plane)
        piv = Dl.copy()
        Tm = np.zeros((nl, plane))
        for l in range(1, nl):
            Tm[l] = Ul[l - 1] / piv[l - 1]
            piv[l] = Dl[l] - Ul[l - 1] * Tm[l]
        self.Tm, self.Tip = Tm.ravel(), (1.0 / piv).ravel()
        self.rho = min(self._block_jacobi_radius(), 1.0 - 1e-12)
        young = 2.0 / (1.0 + np.sqrt(1.0 - self.rho ** 2))
        self.omega = min(1.0 + 1.01 * (young - 1.0), 0.5 * (young + 2.0))

    def _in_plane(self, x):
        """(W x)_i: the in-plane neighbours' couplings (the part outside the blocks)."""
        nx = self.nx
        y = self.wE * np.roll(x, -1)          # wE is 0 on the last column: the wrap adds nothing
        y[1:] += self.wE[:-1] * x[:-1]
        y += self.wN * np.roll(x, -nx)        # likewise wN on the last row of each layer
        y[nx:] += self.wN[:-nx] * x[:-nx]
        return y

    def _block_solve(self, f):
        nl, plane = self.nl, self.nx * self.ny
        g = f.reshape(nl, plane).copy()
        Tm, Tip, U = self.Tm.reshape(nl, plane), self.Tip.reshape(nl, plane), self.wU.reshape(nl, plane)
        for l in range(1, nl):
            g[l] += Tm[l] * g[l - 1]
        z = np.empty_like(g)
        z[nl - 1] = g[nl - 1] * Tip[nl - 1]
        for l in range(nl - 2, -1, -1):
            z[l] = (U[l] * z[l + 1] + g[l]) * Tip[l]
        return z.ravel()

    def _block_apply(self, x):
        """(B x)_i: the diagonal and the via couplings inside the column blocks."""
        plane = self.nx * self.ny
        y = self.D * x
        y[:-plane] -= self.wU[:-plane] * x[plane:]
        y[plane:] -= self.wU[:-plane] * x[:-plane]
        return y

    def _block_jacobi_radius(self, iters: int = 300, seed: int = 0) -> float:
        """Rayleigh quotient x.Wx / x.Bx (a lower bound of rho(B^-1 W)) after power
        iteration on (I + B^-1 W) / 2; the shift keeps -rho from cancelling +rho."""
        x = np.random.default_rng(seed).uniform(0.5, 1.0, self.D.size)
        mu = 0.0
        for _ in range(iters):
            wx = self._in_plane(x)
            mu = float(x @ wx) / float(x @ self._block_apply(x))
            x = 0.5 * (x + self._block_solve(wx))
            x /= np.max(np.abs(x))
        return mu

    def solve(self, b: np.ndarray, x: np.ndarray, target: float, max_sweeps: int = 20000,
              check_every: int = 4) -> int:
        """Relax ``x`` in place until ``max |r| / D <= target``; returns the sweeps used."""
        P = C.POINTER
        R = C.c_double(0.0)
        arr = [a.ctypes.data_as(P(C.c_double)) for a in (self.wE, self.wN, self.wU, self.D, self.Tm, self.Tip, b, x)]
        k = lib().rbsor_block_step(self.nx, self.ny, self.nl, *arr, float(self.omega), float(target),
                                   int(max_sweeps), int(check_every), C.byref(R))
        if k < 0:
            raise RuntimeError(f"column-block SOR did not converge (status {k}, residual {R.value:.3e})")
        return k


def transient(net, h: float, nsteps: int, tol: float = 1e-6, keep: bool = True, mats=None,
              block: bool = False, consts=None, theta: float = 1.0, theta_static=None, check_every: int = 4):
    """Backward-Euler RC transient from the DC point by red-black SOR on all host cores:
    point updates (Eq. 16-17), or with ``block`` the column-block form on a lattice.

    Returns ``(V, stats)``, where ``V`` is ``None`` unless ``keep`` is set; then
    ``V[s]`` holds step ``s = 0..nsteps``.  ``stats`` holds the sweeps, the timed
    seconds of the step loop, the threads used and the per-step target.
    ``consts`` may pass ``(kappa, kacc)`` already computed for this ``h``.

    Warm start: ``v(s-1) + theta (v(s-1) - v(s-2))``.  The default ``theta = 1`` is
    the GPU library's linear extrapolation.  With ``theta_static`` set, that value
    replaces ``theta`` on steps where no load current changed over the last two
    intervals.  ``check_every``: sweeps between residual checks."""
    mats = mats or nodal_matrices(net)
    if mats.A_l.shape[0]:
        raise ValueError("the CPU baseline covers RC grids")
    t0 = time.perf_counter()
    sysm = LatticeSystem(net, h, mats) if block else StepSystem(net, h, mats)
    if consts is None:
        consts = (bounds.scaled_minv_inf_norm(net, h, mats), bounds.accumulation_gain(net, h, mats))
    kappa, kacc = consts
    step_tol = 0.9 * tol / kacc
    target = step_tol / kappa - 1e-13
    v = dc_operating_point(net, mats)
    Ch = mats.C.diagonal() / h
    const = source_terms(mats, h)
    setup_s = time.perf_counter() - t0
    V = [v.copy()] if keep else None
    v_prev = v.copy()
    sweeps = 0
    i_hist = [load_current(net, mats, 0.0)] * 2           # A_i^T I at the last two step times
    t1 = time.perf_counter()
    for s in range(1, nsteps + 1):
        i_now = load_current(net, mats, s * h)
        b = Ch * v - i_now + const
        th = theta
        if theta_static is not None and np.array_equal(i_now, i_hist[-1]) and np.array_equal(i_hist[-1], i_hist[-2]):
            th = theta_static
        i_hist = [i_hist[-1], i_now]
        x = v + th * (v - v_prev) if s > 1 else v.copy()   # extrapolated warm start
        sweeps += sysm.solve(b, x, target, check_every=check_every)
        v_prev, v = v, x
        if keep:
            V.append(v.copy())
    run_s = time.perf_counter() - t1
    stats = dict(sweeps=sweeps, run_s=run_s, setup_s=setup_s, threads=lib().rbsor_threads(), n=net.n_nodes,
                 omega=sysm.omega, kappa=kappa, kacc=kacc, step_tol=step_tol)
    return (np.stack(V) if keep else None), stats
