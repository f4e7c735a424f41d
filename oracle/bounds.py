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


def accumulation_gain(net, h: float, mats=None) -> float:
    """``|| sum_j T^j 1 ||_inf`` with ``T = M^-1 C/h``: the factor by which per-step
    errors of a backward-Euler RC transient can accumulate (``T >= 0``).

    Computed from its closed form ``(I - T)^-1 1 = 1 + (M - C/h)^-1 (C/h) 1``
    (``M - C/h = G`` with the pads inside), by a direct solve.
    """
    mats = mats or nodal_matrices(net)
    c = mats.C.diagonal() / h
    z = DirectSolver(mats.G.tocsc()).solve(c)
    return float(1.0 + np.max(z))


# ---------------------------------------------------------------------------
# certified upper bounds for grids too large for a direct factorisation
# ---------------------------------------------------------------------------

def certified_max_solution(A, rhs, rtol: float = 1e-9, maxiter: int = 20000) -> float:
    """A verified upper bound of ``max_i (A^-1 rhs)_i`` for a non-singular M-matrix ``A``
    and ``rhs > 0``.

    If ``z >= 0`` satisfies ``A z >= rhs`` componentwise, then ``A^-1 rhs <= z``
    (``A^-1 >= 0``), so ``max z`` bounds the maximum.  ``z`` starts from a
    conjugate-gradient solve (any approximation will do; the check is what makes
    the bound rigorous) scaled up until the inequality holds with a margin that
    covers the rounding of the FP64 product (``|fl(Az) - Az| <= 2 n_i eps |A||z|``
    with ``n_i <= 16`` terms per row).
    """
    import scipy.sparse.linalg as sla

    A = A.tocsr()
    rhs = np.asarray(rhs, dtype=np.float64)
    assert np.all(rhs > 0)
    d = A.diagonal()
    pre = sla.LinearOperator(A.shape, matvec=lambda x: x / d)
    z, info = sla.cg(A, rhs, rtol=rtol, maxiter=maxiter, M=pre)
    z = np.maximum(z, 0.0)
    scale = 1.0
    for _ in range(60):
        zz = z * scale
        if is_super_solution(A, rhs, zz):
            return float(np.max(zz))
        err = _ROUND_TERMS * _EPS * (abs(A) @ zz + rhs)
        worst = np.max((rhs + err - A @ z * scale) / np.maximum(rhs, 1e-300))
        scale *= 1.0 + max(2.0 * worst, 1e-12)
    raise RuntimeError("could not certify a super-solution")


_EPS = 2.0 ** -52
_ROUND_TERMS = 2 * 16      # 2 n_i eps |A||z| with at most 16 terms per row (rows here have <= 8)


def is_super_solution(A, rhs, z) -> bool:
    """True when ``A z >= rhs`` holds componentwise even after the rounding of the
    FP64 product is charged against it, i.e. ``fl(A z) - rhs >= 2 n_i eps (|A| |z| + rhs)``.
    For an M-matrix ``A`` this makes ``z >= A^-1 rhs`` (``A^-1 >= 0``, Lemma 1), which
    also implies ``z >= 0`` when ``rhs > 0``."""
    A = A.tocsr()
    z = np.asarray(z, dtype=np.float64)
    lhs = A @ z - rhs
    err = _ROUND_TERMS * _EPS * (abs(A) @ z + rhs)
    return bool(np.all(lhs >= err))


def certified_bounds(net, h: float, tau: float = 1e-6) -> dict:
    """Verified upper bounds of ``kappa = ||M^-1 D||_inf`` and of the RC accumulation
    gain ``1 + ||G^-1 (C/h) 1||_inf`` (``G`` with the pads inside), without a
    factorisation.  The gain's right-hand side is lifted by ``tau * diag(G)`` so that
    it is positive on nodes without capacitors; that only enlarges the bound."""
    mats = nodal_matrices(net)
    M = mats.system_matrix(h)
    kappa = certified_max_solution(M, M.diagonal())
    G = mats.G.tocsr()
    c = mats.C.diagonal() / h
    gain = 1.0 + certified_max_solution(G, c + tau * G.diagonal())
    return {"kappa_upper": kappa, "gain_upper": gain, "tau": tau}
