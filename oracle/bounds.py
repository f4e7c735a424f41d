"""Constants of the rigorous stopping rule, by direct solves.

The system matrix ``M = C/h + G + h L`` is symmetric, has a positive diagonal,
non-positive off-diagonals and is weakly diagonally dominant and irreducible
(Lemma 1), so it is a non-singular M-matrix and ``M^-1 >= 0`` elementwise.
Hence

* ``||M^-1||_inf = max_i (M^-1 1)_i`` exactly, and any iterate ``v`` with
  residual ``r = b - M v`` satisfies ``||v - v*||_inf <= ||M^-1||_inf ||r||_inf``;
* for RC grids the error carried from one step to the next is multiplied by
  ``M^-1 (C/h)``, a non-negative matrix with ``||M^-1 (C/h)||_inf =
  max_i (M^-1 (C/h) 1)_i = q < 1`` whenever some row has a pad.

Algorithm 1 stops on ``||V^(k) - V^(k-1)|| < tol`` with an unspecified norm;
these two numbers turn a per-step residual target into a bound on the
accumulated voltage error: ``||e_s|| <= eps_step / (1 - q)``.
"""
from __future__ import annotations

import numpy as np

from .matrices import nodal_matrices
from .transient import DirectSolver


def minv_inf_norm(net, h: float, mats=None) -> float:
    mats = mats or nodal_matrices(net)
    x = DirectSolver(mats.system_matrix(h)).solve(np.ones(net.n_nodes))
    return float(np.max(x))


def step_gain(net, h: float, mats=None) -> float:
    mats = mats or nodal_matrices(net)
    c = mats.C.diagonal() / h
    y = DirectSolver(mats.system_matrix(h)).solve(c)
    return float(np.max(y))


def scaled_minv_inf_norm(net, h: float, mats=None) -> float:
    """``||M^-1 D||_inf = max_i (M^-1 D 1)_i`` with ``D = diag(M)`` (exact, by a direct solve).

    Used with the scaled residual ``max_i |r_i| / D_i``:
    ``||v - v*||_inf <= ||M^-1 D||_inf * max_i |r_i| / D_i`` because ``M^-1 D >= 0``.
    """
    mats = mats or nodal_matrices(net)
    M = mats.system_matrix(h)
    x = DirectSolver(M).solve(M.diagonal())
    return float(np.max(x))
