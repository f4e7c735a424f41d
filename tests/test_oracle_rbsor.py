"""The multicore red-black SOR baseline (``oracle/rbsor``) against the direct
solves of the oracle, on the CPU.

The baseline runs the paper's relaxation (Eq. 16-17, red-black order) under the
certified stopping rule.  Its trajectory must stay within the accumulated bound,
``0.9 tol``, of the exact backward-Euler trajectory at every step.  Red-black
order makes each colour's updates independent, so the result must not depend on
the thread count.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import pgsynth
from oracle import rbsor, transient

TOL = 1e-6


@pytest.mark.parametrize("block", [False, True])
@pytest.mark.parametrize("make,steps", [(lambda: pgsynth.config0(nx=30, ny=25), 40),
                                        (lambda: pgsynth.config1(nx=24, ny=20), 40),
                                        (lambda: pgsynth.config1(nx=13, ny=9, nl=2), 30)])
def test_rbsor_transient_within_certified_bound(make, steps, block):
    net = make()
    h = net.meta["h"]
    Vo, _ = transient.transient(net, h, steps)
    V, st = rbsor.transient(net, h, steps, tol=TOL, block=block)
    err = np.max(np.abs(V - Vo))
    assert err <= 0.9 * TOL, err
    assert st["sweeps"] > 0 and 1.0 < st["omega"] < 2.0 and st["kacc"] >= 1.0


def test_column_blocks_take_fewer_sweeps_on_layered_grids():
    """With stiff vias inside the blocks, block SOR needs far fewer sweeps than point SOR."""
    net = pgsynth.config1(nx=24, ny=20)
    h = net.meta["h"]
    _, pt = rbsor.transient(net, h, 20, keep=False)
    _, bl = rbsor.transient(net, h, 20, keep=False, block=True)
    assert bl["sweeps"] < 0.6 * pt["sweeps"]


@pytest.mark.parametrize("block", [False, True])
def test_rbsor_is_independent_of_the_thread_count(block):
    net = pgsynth.config1(nx=18, ny=14)
    h = net.meta["h"]
    out = []
    for t in (1, 3):
        rbsor.set_threads(t)
        V, st = rbsor.transient(net, h, 15, tol=TOL, block=block)
        out.append((V, st["sweeps"], st["threads"]))
    rbsor.set_threads(0)
    assert out[0][2] == 1 and out[1][2] == 3
    assert np.array_equal(out[0][0], out[1][0]) and out[0][1] == out[1][1]


def test_column_blocks_need_a_lattice():
    from pgsynth import GROUND, make_netlist, source_terminal as S
    net = make_netlist(2, [1.0], R=[(0, S(0), 1.0), (0, 1, 2.0)], C=[(1, GROUND, 1e-15)])
    with pytest.raises(ValueError):
        rbsor.LatticeSystem(net, 1e-12)


def test_two_colouring():
    # a 3 x 3 lattice is bipartite; a triangle is not
    n = 9
    e = [(y * 3 + x, y * 3 + x + 1) for y in range(3) for x in range(2)] + \
        [(y * 3 + x, (y + 1) * 3 + x) for y in range(2) for x in range(3)]
    a, b = np.array(e).T
    W = sp.csr_matrix((np.ones(2 * len(e)), (np.r_[a, b], np.r_[b, a])), shape=(n, n))
    colour = rbsor.two_colouring(W)
    assert np.all(colour[a] != colour[b])
    assert np.array_equal(colour, np.array([(i % 3 + i // 3) % 2 for i in range(n)]) ^ colour[0])
    T = sp.csr_matrix((np.ones(6), ([0, 1, 1, 2, 2, 0], [1, 0, 2, 1, 0, 2])), shape=(3, 3))
    with pytest.raises(ValueError):
        rbsor.two_colouring(T)


def test_damped_predictor_stays_within_bound():
    """The warm start only changes where the iteration starts: any predictor meets the
    same certified bound."""
    net = pgsynth.config1(nx=20, ny=16)
    h = net.meta["h"]
    Vo, _ = transient.transient(net, h, 60)
    for kw in (dict(theta=0.5), dict(theta=1.0, theta_static=0.5), dict(theta=0.0)):
        V, _ = rbsor.transient(net, h, 60, tol=TOL, block=True, **kw)
        assert np.max(np.abs(V - Vo)) <= 0.9 * TOL, kw

