"""Incidence matrices and nodal system matrices, assembled literally.

Section III-A of the paper: with ``n`` trivial nodes, ``p`` source nodes and
``m`` branches, the modified incidence ``A`` (m x n, Eq. 4) has +1 where a
trivial node is the branch source and -1 where it is the sink; the source
incidence ``A_s`` (m x p, Eq. 5) does the same for source nodes.  Ground has
no column.  Branches are grouped into resistors, capacitors, inductors and
current sources (Eq. 6).  The nodal matrices of Eq. 9 and Eq. 11 are

    G   = A_g^T  Gdiag  A_g          G_s = A_g^T Gdiag A_gs
    C   = A_c^T  Cdiag  A_c
    L   = A_l^T  Ldiag^-1 A_l        L_s = A_l^T Ldiag^-1 A_ls

where ``Gdiag``, ``Cdiag``, ``Ldiag`` hold the branch conductances,
capacitances and inductances (Eq. 8; the paper calls the first "resistance",
it is the conductance).  ``L_s`` is printed as ``A_l Ldiag^-1 A_ls``, which
does not type-check; the transpose on ``A_l`` is the reading used here.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp


def incidence(a: np.ndarray, b: np.ndarray, n: int, p: int):
    """Return ``(A, A_s)`` for branches oriented ``a -> b`` (Eq. 4 and 5).

    Terminal codes: ``t >= 0`` trivial node, ``-1`` ground, ``-2-k`` source
    node ``k``.
    """
    a = np.asarray(a, dtype=np.int64)
    b = np.asarray(b, dtype=np.int64)
    m = a.size
    rows = np.arange(m)
    ta, tb = a >= 0, b >= 0
    sa, sb = a <= -2, b <= -2
    A_coo = sp.coo_matrix(
        (np.concatenate([np.ones(ta.sum()), -np.ones(tb.sum())]),
         (np.concatenate([rows[ta], rows[tb]]), np.concatenate([a[ta], b[tb]]))),
        shape=(m, n))
    As_coo = sp.coo_matrix(
        (np.concatenate([np.ones(sa.sum()), -np.ones(sb.sum())]),
         (np.concatenate([rows[sa], rows[sb]]), np.concatenate([-2 - a[sa], -2 - b[sb]]))),
        shape=(m, p))
    return A_coo.tocsr(), As_coo.tocsr()


@dataclass
class NodalMatrices:
    n: int
    p: int
    G: sp.csr_matrix
    C: sp.csr_matrix
    L: sp.csr_matrix
    G_s: sp.csr_matrix
    L_s: sp.csr_matrix
    A_i: sp.csr_matrix
    A_is: sp.csr_matrix
    A_l: sp.csr_matrix
    A_ls: sp.csr_matrix
    Ldiag_inv: np.ndarray
    vd: np.ndarray

    def system_matrix(self, h: float) -> sp.csc_matrix:
        """M = C/h + G + h L (Eq. 11; Eq. 2 when there are no inductors)."""
        return (self.C / h + self.G + h * self.L).tocsc()


def nodal_matrices(net) -> NodalMatrices:
    n, p = net.n_nodes, net.n_sources
    A_g, A_gs = incidence(net.r_a, net.r_b, n, p)
    A_c, _ = incidence(net.c_a, net.c_b, n, p)
    A_l, A_ls = incidence(net.l_a, net.l_b, n, p)
    A_i, A_is = incidence(net.i_a, net.i_b, n, p)
    Gd = sp.diags(np.asarray(net.r_g, dtype=np.float64))
    Cd = sp.diags(np.asarray(net.c_val, dtype=np.float64))
    Linv = 1.0 / np.asarray(net.l_val, dtype=np.float64)
    Ld = sp.diags(Linv)
    G = (A_g.T @ Gd @ A_g).tocsr()
    C = (A_c.T @ Cd @ A_c).tocsr()
    L = (A_l.T @ Ld @ A_l).tocsr()
    G_s = (A_g.T @ Gd @ A_gs).tocsr()
    L_s = (A_l.T @ Ld @ A_ls).tocsr()
    return NodalMatrices(n=n, p=p, G=G, C=C, L=L, G_s=G_s, L_s=L_s, A_i=A_i, A_is=A_is,
                         A_l=A_l, A_ls=A_ls, Ldiag_inv=Linv,
                         vd=np.asarray(net.vdd, dtype=np.float64))
