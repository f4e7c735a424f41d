"""Pins of the windowed central differences used by the full-size per-parameter
gradient check (window_fd.py), against the oracle's exact discrete adjoint.

* With a box that holds the whole grid the windowed difference is a central
  difference of the exact recurrence: it must equal the adjoint gradient up to
  the difference's own O(eps^2) truncation (eps = 1e-3 of the parameter).
* With the 257 x 257 box the full-size check uses, on a grid larger than the
  box, the truncation of the response at the box's edge must stay well below
  the full-size check's 1e-4.
Both on the 2048x2048 recipe drawn smaller, over 60 steps of its load switching.
"""
import numpy as np
import pytest

import pgsynth
import window_fd
from oracle import adjoint, matrices, transient


@pytest.fixture(scope="module")
def case():
    net = pgsynth.config4(nx=400, ny=400)
    h, S = net.meta["h"], 60
    mats = matrices.nodal_matrices(net)
    J, dG, dC = adjoint.gradients(net, h, S)
    V = np.stack([v for _, v, _ in transient.simulate(net, h, S, mats=mats)])
    M = mats.system_matrix(h).tocsr()
    ch = mats.C.diagonal() / h
    rng = np.random.default_rng(8)
    nx = net.lattice[0]
    central = lambda i: abs(i % nx - nx // 2) < 40 and abs(i // nx - nx // 2) < 40
    seg = np.where((net.r_a >= 0) & (net.r_b >= 0))[0]
    cnode = np.where(net.c_a >= 0, net.c_a, net.c_b)
    rs = [int(e) for e in rng.choice(seg, 2000, replace=False) if central(int(net.r_a[e]))][:3]
    cs = [int(k) for k in rng.choice(len(net.c_val), 2000, replace=False) if central(int(cnode[k]))][:3]
    params = [("r", e, (net.r_a[e], net.r_b[e]), net.r_g[e], dG[e]) for e in rs]
    params += [("c", k, (cnode[k],), net.c_val[k], dC[k]) for k in cs]
    return net, h, V, M, ch, params


def _rel_errors(case, R):
    net, h, V, M, ch, params = case
    out = []
    for kind, _, term, p, exact in params:
        win, Mw, chw, loc = window_fd.parameter_window(M, ch, net.lattice, kind, term, R)
        fd = window_fd.central_difference(Mw, chw, V[1:, win], V[0, win], kind, loc, 1e-3 * p, h)
        out.append(abs(fd - exact) / abs(exact))
    return np.array(out)


def test_window_fd_whole_grid_equals_adjoint(case):
    V = case[2]
    assert np.ptp(V[0]) < 1e-12          # the DC point is the supply: dv_0 = 0
    rel = _rel_errors(case, 500)
    assert rel.max() <= 2e-6, rel


def test_window_fd_box_truncation(case):
    rel = _rel_errors(case, 128)
    assert rel.max() <= 1e-6, rel
    # a box a fifth as wide misses the far response: the pin is not vacuous
    assert _rel_errors(case, 24).max() > 1e-3
