"""Pins of the CPU oracle against closed forms, hand derivations and invariants.

Each test fixes the oracle to something other than itself: an exact
discrete solution, a hand-solved small circuit, a conservation law, a
symmetry, or the paper's own theorems (Lemma 1, Theorem 1).  They are chosen
so that a dropped term, a wrong sign or a transposed index in the oracle
fails at least one of them.
"""
import json
import os

import numpy as np
import pytest

import pgsynth
from pgsynth import GROUND, make_netlist, source_terminal as S
from oracle import bounds, matrices, pwl, relax, transient

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


# ---------------------------------------------------------------- closed forms

def test_single_node_rc_discrete_closed_form():
    """One node, cap C to ground, pad G0 to Vdd, no load, v(0) != Vdd.
    Backward Euler gives v_k - Vdd = (v_0 - Vdd) (1 + h G0 / C)^-k exactly (Eq. 2)."""
    fx = _load("single_node_rc.json")
    C, g0, vdd, v0, h, K = fx["C"], fx["G0"], fx["Vdd"], fx["v0"], fx["h"], fx["steps"]
    net = make_netlist(1, [vdd], R=[(0, S(0), g0)], C=[(0, GROUND, C)])
    V, _ = transient.transient(net, h, K, v0=np.array([v0]))
    k = np.arange(K + 1)
    exact = vdd + (v0 - vdd) * (1.0 + h * g0 / C) ** (-k)
    np.testing.assert_allclose(V[:, 0], exact, rtol=0, atol=1e-14)
    # continuous limit exp(-t G0/C): BE error at most O(h) (first-order method)
    tau = C / g0
    cont = vdd + (v0 - vdd) * np.exp(-k * h / tau)
    err = np.max(np.abs(V[:, 0] - cont))
    assert err < 0.5 * abs(v0 - vdd) * (h / tau)


def test_single_node_bounds_closed_form():
    """||M^-1||_inf = 1/(C/h + G0) and q = (C/h)/(C/h + G0) for one node."""
    C, g0, h = 50e-15, 10.0, 10e-12
    net = make_netlist(1, [1.0], R=[(0, S(0), g0)], C=[(0, GROUND, C)])
    assert bounds.minv_inf_norm(net, h) == pytest.approx(1.0 / (C / h + g0), rel=1e-14)
    assert bounds.step_gain(net, h) == pytest.approx((C / h) / (C / h + g0), rel=1e-14)


def test_scaled_minv_inf_norm_single_node_is_one():
    """With one node M = D, so ||M^-1 D||_inf = 1 whatever C, G0 and h are."""
    for C, g0, h in ((50e-15, 10.0, 10e-12), (1e-12, 0.1, 1e-9), (0.0, 3.0, 1e-12)):
        net = make_netlist(1, [1.0], R=[(0, S(0), g0)], C=[(0, GROUND, C)] if C else [])
        assert bounds.scaled_minv_inf_norm(net, h) == pytest.approx(1.0, rel=1e-15)


def _two_node_system(fx):
    """The two-node circuit of ``two_node_rc.json`` written out by hand: node 0 has the pad
    G0 and no capacitor, node 1 has C1; the segment g joins them (Eq. 12 with Eq. 2)."""
    g0, g, C1, h = fx["G0"], fx["g"], fx["C1"], fx["h"]
    M = np.array([[g0 + g, -g], [-g, g + C1 / h]])
    G = np.array([[g0 + g, -g], [-g, g]])          # M - C/h: the pad stays on the diagonal
    net = make_netlist(2, [fx["Vdd"]], R=[(0, S(0), g0), (0, 1, g)], C=[(1, GROUND, C1)])
    return net, M, G


def _cramer(A, b):
    det = A[0, 0] * A[1, 1] - A[0, 1] * A[1, 0]
    return np.array([(b[0] * A[1, 1] - A[0, 1] * b[1]) / det, (A[0, 0] * b[1] - b[0] * A[1, 0]) / det])


def test_bounds_of_two_node_circuit_by_cramer():
    """kappa = max (M^-1 D 1), q = max (M^-1 (C/h) 1) and the accumulation gain
    1 + max (G^-1 (C/h) 1) of the hand circuit, each by Cramer's rule.  Written out:
    M^-1 D 1 = [(g + C1/h)(G0 + 2g), (G0 + g)(2g + C1/h)] / det M, and
    G^-1 (C/h) 1 = [C1/(h G0), (G0 + g) C1 / (h G0 g)]."""
    fx = _load("two_node_rc.json")
    net, M, G = _two_node_system(fx)
    h, g0, g, C1 = fx["h"], fx["G0"], fx["g"], fx["C1"]
    detM = M[0, 0] * M[1, 1] - M[0, 1] ** 2
    kappa = max((g + C1 / h) * (g0 + 2 * g), (g0 + g) * (2 * g + C1 / h)) / detM
    np.testing.assert_allclose(_cramer(M, np.diag(M)), [(g + C1 / h) * (g0 + 2 * g) / detM,
                                                        (g0 + g) * (2 * g + C1 / h) / detM], rtol=1e-15)
    assert bounds.scaled_minv_inf_norm(net, h) == pytest.approx(kappa, rel=1e-13)
    assert bounds.step_gain(net, h) == pytest.approx(np.max(_cramer(M, [0.0, C1 / h])), rel=1e-13)
    gain = 1.0 + max(C1 / (h * g0), (g0 + g) * C1 / (h * g0 * g))
    assert bounds.accumulation_gain(net, h) == pytest.approx(gain, rel=1e-13)


def test_certified_bounds_of_two_node_circuit():
    """The certified (factorisation-free) bounds enclose the hand values from above and
    stay within the CG tolerance of them: kappa_upper >= max(M^-1 D 1), and gain_upper >=
    1 + max(G^-1 (C/h 1 + tau diag G)), the right-hand side with its stated lift."""
    fx = _load("two_node_rc.json")
    net, M, G = _two_node_system(fx)
    h, tau = fx["h"], 1e-6
    cb = bounds.certified_bounds(net, h, tau=tau)
    kappa = np.max(_cramer(M, np.diag(M)))
    lifted = 1.0 + np.max(_cramer(G, np.array([0.0, fx["C1"] / h]) + tau * np.diag(G)))
    assert kappa <= cb["kappa_upper"] <= kappa * (1 + 1e-8)
    assert lifted <= cb["gain_upper"] <= lifted * (1 + 1e-8)
    assert cb["tau"] == tau


@pytest.mark.parametrize("recipe", ["config0_40x30", "config1_24x20x3", "config0_64x64"])
def test_certified_bounds_enclose_direct_solves(recipe):
    """On grids small enough for the direct solver the certified bounds must lie above
    the exact constants (a sub-solution accepted by the check would fall below) and
    close to them: kappa within the CG tolerance (1e-7 relative), and the gain within
    the lift tau ||G^-1 diag G||_inf it adds on purpose plus 1e-5 relative.  The
    accumulation gain itself is pinned by the error-propagation test below."""
    from oracle.transient import DirectSolver
    net = {"config0_40x30": lambda: pgsynth.config0(nx=40, ny=30),
           "config1_24x20x3": lambda: pgsynth.config1(nx=24, ny=20),
           "config0_64x64": lambda: pgsynth.config0(nx=64, ny=64)}[recipe]()
    h = net.meta["h"]
    mats = matrices.nodal_matrices(net)
    kappa = bounds.scaled_minv_inf_norm(net, h, mats)
    gain = bounds.accumulation_gain(net, h, mats)
    cb = bounds.certified_bounds(net, h)
    assert kappa <= cb["kappa_upper"] <= kappa * (1 + 1e-7)
    G = mats.G.tocsc()
    lift = cb["tau"] * np.max(DirectSolver(G).solve(G.diagonal()))
    assert gain <= cb["gain_upper"] <= gain + lift + 1e-5 * gain
    assert cb["gain_upper"] - gain >= 0.5 * lift        # the lift is on the right-hand side, not removed


def test_super_solution_check_direction():
    """The check that makes the certified bounds rigorous: with x = M^-1 D 1 exact, a
    vector 1e-8 above x passes and one 1e-8 below fails, as does a copy of x lowered at a
    single node.  Raised by 3e-11 only, x has a computed residual M z - D 1 that is
    positive in every row yet inside the rounding of the FP64 product, so the check must
    refuse it: the rounding margin is charged."""
    from oracle.transient import DirectSolver
    net = pgsynth.config1(nx=24, ny=20)
    h = net.meta["h"]
    M = matrices.nodal_matrices(net).system_matrix(h).tocsr()
    rhs = M.diagonal()
    x = DirectSolver(M.tocsc()).solve(rhs)
    assert bounds.is_super_solution(M, rhs, x * (1 + 1e-8))
    assert not bounds.is_super_solution(M, rhs, x * (1 - 1e-8))
    low = x * (1 + 1e-8)
    k = int(np.argmax(x))
    low[k] = x[k] * (1 - 1e-6)
    assert not bounds.is_super_solution(M, rhs, low)
    thin = x * (1 + 3e-11)
    assert np.all(M @ thin - rhs > 0)
    assert not bounds.is_super_solution(M, rhs, thin)


def test_accumulation_gain_bounds_error_propagation():
    """Per-step errors eta_k with |eta_k| <= 1 propagate through e_s = T e_{s-1} + eta_s,
    T = M^-1 C/h; the accumulation gain bounds |e_s| for every sign pattern, is
    attained by eta = 1, and never exceeds 1/(1-q)."""
    net = pgsynth.config1(nx=9, ny=7)
    h = net.meta["h"]
    mats = matrices.nodal_matrices(net)
    M = mats.system_matrix(h).toarray()
    T = np.linalg.solve(M, np.diag(mats.C.diagonal() / h))
    K = bounds.accumulation_gain(net, h)
    q = bounds.step_gain(net, h)
    assert K <= 1.0 / (1.0 - q) + 1e-9
    rng = np.random.default_rng(2)
    for trial in range(5):
        e = np.zeros(net.n_nodes)
        worst = 0.0
        for s in range(3000):
            eta = np.ones(net.n_nodes) if trial == 0 else rng.choice([-1.0, 1.0], net.n_nodes)
            e = T @ e + eta
            worst = max(worst, np.max(np.abs(e)))
        assert worst <= K * (1 + 1e-9)
        if trial == 0:
            assert worst == pytest.approx(K, rel=1e-6)     # the all-ones pattern attains it


def test_two_node_rc_hand_derived():
    """Pad(G0) - node0 - R(g) - node1 with C1 and a constant load I at node 1.

    KCL, backward Euler:
      node0: G0 (v0 - Vdd) + g (v0 - v1) = 0
      node1: g (v1 - v0) + C1 (v1 - v1p)/h + I = 0
    Cramer's rule on the 2x2 system; DC: v0 = Vdd - I/G0, v1 = v0 - I/g."""
    fx = _load("two_node_rc.json")
    g0, g, C1, I, vdd, h = fx["G0"], fx["g"], fx["C1"], fx["I"], fx["Vdd"], fx["h"]
    net = make_netlist(2, [vdd], R=[(0, S(0), g0), (0, 1, g)], C=[(1, GROUND, C1)],
                       I=[(1, GROUND, [0.0, 1.0], [I, I])])
    V, _ = transient.transient(net, h, 5, v0=np.array([vdd, vdd]))
    v1p = vdd
    for k in range(1, 6):
        a11, a12, b1 = g0 + g, -g, g0 * vdd
        a21, a22, b2 = -g, g + C1 / h, C1 / h * v1p - I
        det = a11 * a22 - a12 * a21
        v0 = (b1 * a22 - a12 * b2) / det
        v1 = (a11 * b2 - b1 * a21) / det
        np.testing.assert_allclose(V[k], [v0, v1], rtol=0, atol=1e-13)
        v1p = v1
    vdc = transient.dc_operating_point(net)
    np.testing.assert_allclose(vdc, [vdd - I / g0, vdd - I / g0 - I / g], rtol=0, atol=1e-13)


def test_ladder_dc_closed_form():
    """A chain of N nodes with a pad at node 0 and a load I at the far end:
    the whole load current flows through every segment, so
    v_k = Vdd - I (1/G0 + sum_{j<k} 1/g_j)."""
    rng = np.random.default_rng(7)
    N, vdd, g0, I = 12, 1.1, 8.0, 2e-3
    g = rng.uniform(0.5, 2.0, N - 1)
    net = make_netlist(N, [vdd], R=[(0, S(0), g0)] + [(k, k + 1, g[k]) for k in range(N - 1)],
                       I=[(N - 1, GROUND, [0.0], [I])])
    v = transient.dc_operating_point(net)
    exact = vdd - I * (1.0 / g0 + np.concatenate([[0.0], np.cumsum(1.0 / g)]))
    np.testing.assert_allclose(v, exact, rtol=0, atol=1e-14)
    # the node form (Eq. 12 with C = 0) solved by Gauss-Seidel agrees
    vg, _ = relax.gs_dc(relax.NodeTopology(net), tol=1e-15)
    np.testing.assert_allclose(vg, exact, rtol=0, atol=1e-12)


def test_lc_tank_eigen_solution_and_energy_decay():
    """One node, cap C to ground, inductor L from the node to Vdd (explicit i_l).

    With x = (v - Vdd, i_l): (C/h + h/L) x1' = (C/h) x1 - x2, x2' = x2 + (h/L) x1',
    a 2x2 linear recurrence x_{k+1} = T x_k solved by its eigen-decomposition.
    Backward Euler is dissipative: the energy C x1^2/2 + L x2^2/2 must fall."""
    fx = _load("lc_tank.json")
    C, Lh, vdd, v0, h, K = fx["C"], fx["L"], fx["Vdd"], fx["v0"], fx["h"], fx["steps"]
    net = make_netlist(1, [vdd], C=[(0, GROUND, C)], L=[(0, S(0), Lh)])
    V, IL = transient.transient(net, h, K, v0=np.array([v0]), il0=np.zeros(1))
    d = C / h + h / Lh
    T = np.array([[C / h / d, -1.0 / d],
                  [h / Lh * C / h / d, 1.0 - h / Lh / d]])
    w, P = np.linalg.eig(T)
    x0 = np.array([v0 - vdd, 0.0])
    c = np.linalg.solve(P, x0)
    for k in range(K + 1):
        xk = np.real(P @ (c * w ** k))
        np.testing.assert_allclose([V[k, 0] - vdd, IL[k, 0]], xk, rtol=0, atol=1e-12)
    E = 0.5 * C * (V[:, 0] - vdd) ** 2 + 0.5 * Lh * IL[:, 0] ** 2
    assert np.all(np.diff(E) < 0)
    # and it oscillates (complex eigenvalues, |lambda| < 1)
    assert np.all(np.abs(np.imag(w)) > 0) and np.all(np.abs(w) < 1)


# ---------------------------------------------------------------- invariants

def _small(cfg, **kw):
    return pgsynth.CONFIGS[cfg](**kw)


def test_lemma1_system_matrix_is_spd_m_matrix():
    """Lemma 1: M = C/h + G + hL is symmetric, weakly diagonally dominant with a
    positive diagonal and non-positive off-diagonals, hence SPD; M^-1 >= 0."""
    for net in (_small(0, nx=9, ny=7), _small(2, nx=8, ny=6)):
        mats = matrices.nodal_matrices(net)
        M = mats.system_matrix(net.meta["h"]).toarray()
        assert np.allclose(M, M.T, rtol=0, atol=0)
        off = M - np.diag(np.diag(M))
        assert np.all(off <= 0)
        assert np.all(np.diag(M) > 0)
        assert np.all(M.sum(axis=1) >= -1e-12 * np.abs(np.diag(M)))
        np.linalg.cholesky(M)
        assert np.all(np.linalg.inv(M) >= -1e-12)


def test_row_sums_equal_grounded_conductance():
    """M 1 collects only the branches that leave the trivial nodes: C/h, the
    pad conductances and h/L of pad inductors (computed here from the element
    lists, not from the assembly)."""
    net = _small(2, nx=10, ny=6)
    h = net.meta["h"]
    mats = matrices.nodal_matrices(net)
    rs = mats.system_matrix(h) @ np.ones(net.n_nodes)
    expect = np.zeros(net.n_nodes)
    for a, b, c in zip(net.c_a, net.c_b, net.c_val):
        expect[a] += c / h
    for a, b, g in zip(net.r_a, net.r_b, net.r_g):
        if b < 0:
            expect[a] += g
    for a, b, l in zip(net.l_a, net.l_b, net.l_val):
        if b < 0:
            expect[a] += h / l
    np.testing.assert_allclose(rs, expect, rtol=1e-12, atol=1e-12)


def test_zero_load_keeps_vdd():
    """With every load at zero and v(0) = Vdd, v = Vdd at every node and step
    (G 1 = 0 and the pads balance), for RC and RLC."""
    for cfg in (0, 2):
        net = _small(cfg, nx=11, ny=9)
        net.i_v[:] = 0.0
        V, IL = transient.transient(net, net.meta["h"], 15)
        np.testing.assert_allclose(V, 1.0, rtol=0, atol=1e-13)
        if IL.size:
            np.testing.assert_allclose(IL, 0.0, rtol=0, atol=1e-12)


def test_global_charge_balance():
    """Summing KCL over all trivial nodes: the current delivered by the sources
    through pad resistors and pad inductors equals the load current plus the
    capacitor charging current, at every step (RC and RLC)."""
    for cfg in (0, 2):
        net = _small(cfg, nx=10, ny=8)
        h = net.meta["h"]
        V, IL = transient.transient(net, h, 60)
        Cn = np.zeros(net.n_nodes)
        np.add.at(Cn, net.c_a, net.c_val)
        pad_r = net.r_b < 0
        pad_l = net.l_b < 0
        for s in range(1, V.shape[0]):
            v = V[s]
            supply = np.sum(net.r_g[pad_r] * (1.0 - v[net.r_a[pad_r]]))
            supply -= np.sum(IL[s][pad_l])  # inductor current a->b flows into the source
            load = np.sum(pwl.pwl_values(net.i_ptr, net.i_t, net.i_v, s * h))
            charge = np.sum(Cn * (V[s] - V[s - 1]) / h)
            assert supply == pytest.approx(load + charge, rel=1e-9, abs=1e-12)


def test_mirror_symmetry():
    """Uniform segments, one central pad and a uniform load on a square grid:
    the voltage map is invariant under x<->y and x -> nx-1-x (catches transposed
    or shifted indices)."""
    n = 9
    ids = np.arange(n * n).reshape(n, n)
    R = [(int(ids[y, x]), int(ids[y, x + 1]), 1.0) for y in range(n) for x in range(n - 1)]
    R += [(int(ids[y, x]), int(ids[y + 1, x]), 1.0) for y in range(n - 1) for x in range(n)]
    R += [(int(ids[4, 4]), S(0), 10.0)]
    C = [(int(i), GROUND, 20e-15) for i in range(n * n)]
    I = [(int(i), GROUND, [0.0, 50e-12], [0.0, 1e-4]) for i in range(n * n)]
    net = make_netlist(n * n, [1.0], R=R, C=C, I=I)
    V, _ = transient.transient(net, 5e-12, 20)
    for s in (5, 20):
        m = V[s].reshape(n, n)
        np.testing.assert_allclose(m, m.T, atol=1e-14)
        np.testing.assert_allclose(m, m[:, ::-1], atol=1e-14)
        assert m[4, 4] == m.max()


def test_three_level_form_matches_explicit_form():
    """Eq. 11 (three-level, no inductor state) and Eq. 10 (explicit i_l) are the
    same recurrence once v(0), v(1) agree: trajectories match to rounding."""
    net = _small(2, nx=9, ny=8)
    h = net.meta["h"]
    V, _ = transient.transient(net, h, 80)
    for s, v in transient.simulate_three_level(net, h, 80, V[0], V[1]):
        np.testing.assert_allclose(v, V[s], rtol=0, atol=1e-11)


def test_large_inductance_limit_is_rc():
    """L -> infinity removes the inductive paths: an RLC grid with huge L
    reproduces the RC grid without those inductors."""
    net = _small(2, nx=8, ny=7)
    h = net.meta["h"]
    big = pgsynth.Netlist(**{**net.__dict__, "l_val": np.full_like(net.l_val, 1e9)})
    rc = pgsynth.Netlist(**{**net.__dict__, "l_a": net.l_a[:0], "l_b": net.l_b[:0],
                            "l_val": net.l_val[:0]})
    V1, _ = transient.transient(big, h, 40)
    V2, _ = transient.transient(rc, h, 40)
    np.testing.assert_allclose(V1, V2, rtol=0, atol=1e-12)


# ---------------------------------------------------------------- Theorem 1

@pytest.mark.parametrize("omega", [1.0, 1.6])
def test_gauss_seidel_converges_to_direct_rc(omega):
    """Theorem 1 / Eq. 17: the node-by-node GS/SOR of Algorithm 1 converges to
    the unique solution of the BE system (RC)."""
    net = _small(0, nx=7, ny=6)
    h = net.meta["h"]
    topo = relax.NodeTopology(net)
    V, IL = transient.transient(net, h, 30)
    for s in (10, 20, 30):
        v, _, _ = relax.gs_step_explicit(topo, h, V[s - 1], IL[s - 1], s * h, omega=omega,
                                         tol=1e-15)
        np.testing.assert_allclose(v, V[s], rtol=0, atol=1e-11)


@pytest.mark.parametrize("omega", [1.0, 1.5])
def test_gauss_seidel_converges_to_direct_rlc(omega):
    """Same for RLC, in both the explicit-i_l node form and Eq. 14."""
    net = _small(2, nx=6, ny=5)
    h = net.meta["h"]
    topo = relax.NodeTopology(net)
    V, IL = transient.transient(net, h, 40)
    for s in (15, 30, 40):
        v, il, _ = relax.gs_step_explicit(topo, h, V[s - 1], IL[s - 1], s * h, omega=omega,
                                          tol=1e-15)
        np.testing.assert_allclose(v, V[s], rtol=0, atol=1e-11)
        np.testing.assert_allclose(il, IL[s], rtol=1e-9, atol=1e-12)
        v3, _ = relax.gs_step_three_level(topo, h, V[s - 1], V[s - 2], s * h, omega=omega,
                                          tol=1e-15)
        np.testing.assert_allclose(v3, V[s], rtol=0, atol=1e-10)


# ---------------------------------------------------------------- PWL and solver

def test_pwl_vectorised_matches_loop_and_breakpoints():
    rng = np.random.default_rng(3)
    ptr, ts, vs = [0], [], []
    for _ in range(200):
        k = int(rng.integers(1, 6))
        t = np.sort(rng.uniform(0, 1e-9, k))
        if k > 2 and rng.random() < 0.3:
            t[1] = t[2]                       # a zero-length segment (a jump)
        ts.extend(t); vs.extend(rng.uniform(-1e-3, 1e-3, k)); ptr.append(len(ts))
    ptr, ts, vs = np.array(ptr), np.array(ts), np.array(vs)
    for t in np.concatenate([rng.uniform(-1e-10, 1.2e-9, 50), ts[:40]]):
        got = pwl.pwl_values(ptr, ts, vs, t)
        for e in range(len(ptr) - 1):
            assert got[e] == pwl.pwl_scalar(ts[ptr[e]:ptr[e + 1]], vs[ptr[e]:ptr[e + 1]], t)
    # triangular source: 0 before t0, the peak at t0+tr, half the peak mid-fall
    tri = (np.array([0, 3]), np.array([1.0, 2.0, 4.0]), np.array([0.0, 5.0, 0.0]))
    assert pwl.pwl_values(*tri, 0.5)[0] == 0.0
    assert pwl.pwl_values(*tri, 2.0)[0] == 5.0
    assert pwl.pwl_values(*tri, 3.0)[0] == 2.5
    assert pwl.pwl_values(*tri, 1.5)[0] == 2.5
    assert pwl.pwl_values(*tri, 9.0)[0] == 0.0


def test_sparse_and_dense_solvers_agree():
    net = _small(0, nx=50, ny=45)   # 2250 nodes -> sparse path
    mats = matrices.nodal_matrices(net)
    M = mats.system_matrix(net.meta["h"])
    assert M.shape[0] > transient.DENSE_MAX
    b = np.random.default_rng(1).standard_normal(M.shape[0])
    x = transient.DirectSolver(M).solve(b)
    np.testing.assert_allclose(M @ x, b, rtol=0, atol=1e-10)
    xd = np.linalg.solve(M.toarray(), b)
    np.testing.assert_allclose(x, xd, rtol=1e-10, atol=1e-13)


# ---------------------------------------------------------------- generator

def test_generator_config0_counts_and_ranges():
    net = pgsynth.config0()
    c = net.counts()
    assert c["n"] == 10000 and c["p"] == 1
    assert c["R"] == 19800 + 100          # 2*100*99 segments + 100 pads
    assert c["C"] == 10000 and c["I"] == 2000 and c["L"] == 0
    seg = net.r_b >= 0
    assert net.r_g[seg].min() >= 0.5 and net.r_g[seg].max() <= 2.0
    assert np.all(net.r_g[~seg] == 10.0)
    pads = net.r_a[~seg]
    assert np.all((pads % 100) % 10 == 0) and np.all((pads // 100) % 10 == 0)
    assert 10e-15 <= net.c_val.min() and net.c_val.max() <= 100e-15
    assert len(np.unique(net.i_a)) == 2000
    t = net.i_t.reshape(-1, 3); v = net.i_v.reshape(-1, 3)
    assert np.all(v[:, 0] == 0) and np.all(v[:, 2] == 0) and v[:, 1].max() <= 1e-3
    assert np.all(np.diff(t, axis=1) >= 20e-12) and np.all(np.diff(t, axis=1) <= 100e-12)
    assert t[:, 0].min() >= 0 and t[:, 0].max() <= 1e-9
    # same seed, same netlist; different seed, different draw
    assert np.array_equal(pgsynth.config0().r_g, net.r_g)
    assert not np.array_equal(pgsynth.config0(seed=5).r_g, net.r_g)


def test_generator_multilayer_counts():
    nx, ny = 64, 40
    net = pgsynth.config1(nx=nx, ny=ny)
    c = net.counts()
    seg = 3 * (2 * nx * ny - nx - ny)
    vias = 2 * nx * ny
    pads = len(range(0, nx, 32)) * len(range(0, ny, 32))
    assert c["R"] == seg + vias + pads
    assert c["C"] == nx * ny and c["I"] == round(0.3 * nx * ny)
    assert np.all(net.c_a < nx * ny)                  # decaps on the bottom layer
    assert np.all(net.r_a[net.r_b < 0] >= 2 * nx * ny)  # pads on the top layer
    r = pgsynth.config2(nx=32, ny=32).counts()
    assert r["L"] == 32 * 32 + 4  # every via and every pad


def test_generator_config4_counts():
    """The 2048 x 2048 single-layer mesh: 2 * 2048 * 2047 segments, pads where x and y
    are multiples of 10 (205 x 205), a capacitor on every node, loads on 20 % of them."""
    net = pgsynth.config4()
    c = net.counts()
    n = 2048 * 2048
    assert c["n"] == n and c["L"] == 0 and c["C"] == n
    seg = net.r_b >= 0
    assert int(seg.sum()) == 2 * 2048 * 2047 == 8_384_512
    assert int((~seg).sum()) == 205 * 205 == 42_025
    assert c["I"] == round(0.2 * n) == 838_861
    assert net.meta["h"] == 10e-12 and net.meta["nsteps"] == 500


def test_generator_config3_structure():
    """Batched grids: each part is a lattice of side 64..512 with 1 or 2 layers, drawn from
    its own child seed; parts sit back to back; 2-layer parts have one via per column."""
    parts = pgsynth.config3_parts(n_grids=8)
    off = 0
    for o, p in parts:
        nx, ny, nl = p.lattice
        assert o == off and nx == ny and 64 <= nx <= 512 and nl in (1, 2)
        c = p.counts()
        assert c["n"] == nx * ny * nl
        seg = nl * 2 * nx * (nx - 1)
        pads = len(range(0, nx, 10)) ** 2
        assert c["R"] == seg + (nx * nx if nl == 2 else 0) + pads
        assert c["C"] == nx * nx and c["I"] == round(0.2 * nx * nx)
        off += c["n"]
    # the batch is the parts side by side
    net = pgsynth.config3(n_grids=8)
    assert net.n_nodes == off and [l[0] for l in net.lattices] == [o for o, _ in parts]


# ---------------------------------------------------------------- adjoint (not in the paper)

def _adjoint_case():
    net = pgsynth.config0(nx=7, ny=6)
    # a resistor to ground and loads already on at t = 0 make the DC point depend on G
    net.r_a = np.concatenate([net.r_a, np.array([20], np.int32)])
    net.r_b = np.concatenate([net.r_b, np.array([GROUND], np.int32)])
    net.r_g = np.concatenate([net.r_g, np.array([0.3])])
    net.i_v = net.i_v.copy() * 40.0                 # drops of tens of mV
    net.i_v[0::3] = 5e-3
    return net


def test_generator_config3_single_part_matches_batch():
    """config3_part(k) draws grid k alone, with the values and offset it has in the batch;
    config3_shapes lists every grid's side and layer count without drawing them."""
    parts = pgsynth.config3_parts(n_grids=9, side_lo=16, side_hi=30)
    shapes = pgsynth.config3_shapes(n_grids=9, side_lo=16, side_hi=30)
    for k in (0, 4, 8):
        off, p = pgsynth.config3_part(k, n_grids=9, side_lo=16, side_hi=30)
        o2, p2 = parts[k]
        assert off == o2 and p.lattice == p2.lattice and shapes[k] == (p.lattice[0], p.lattice[2])
        for a in ("r_a", "r_b", "r_g", "c_val", "i_a", "i_t", "i_v"):
            np.testing.assert_array_equal(getattr(p, a), getattr(p2, a))


def test_adjoint_matches_central_differences():
    """The oracle's discrete adjoint against central finite differences of the
    oracle's own forward objective (exact direct solves), for resistors (segments,
    pads, a resistor to ground: DC-point term) and capacitors."""
    from oracle import adjoint
    net = _adjoint_case()
    h, S = 10e-12, 25
    J, dG, dC = adjoint.gradients(net, h, S)
    assert J == pytest.approx(adjoint.objective(net, h, S), rel=1e-12)
    rng = np.random.default_rng(4)
    picks = [("r", int(k)) for k in rng.choice(len(net.r_g), 8, replace=False)]
    picks += [("r", len(net.r_g) - 1), ("r", int(np.nonzero(net.r_b < -1)[0][0]))]
    picks += [("c", int(k)) for k in rng.choice(len(net.c_val), 6, replace=False)]
    for kind, k in picks:
        arr = net.r_g if kind == "r" else net.c_val
        d = 1e-4 * arr[k]
        vals = []
        for sgn in (+1, -1):
            pert = arr.copy(); pert[k] += sgn * d
            n2 = pgsynth.Netlist(**{**net.__dict__, ("r_g" if kind == "r" else "c_val"): pert})
            vals.append(adjoint.objective(n2, h, S))
        fd = (vals[0] - vals[1]) / (2 * d)
        ad = dG[k] if kind == "r" else dC[k]
        assert ad == pytest.approx(fd, rel=2e-5, abs=1e-9 * abs(J) / arr[k]), (kind, k)


def test_adjoint_scaling_identity():
    """Multiplying every conductance and capacitance by a maps v - Vdd to
    (v - Vdd)/a when the supply is the only source (Eq. 2 with the DC point
    G v_0 = b_0), so sum_e g_e dJ/dg_e + sum_k C_k dJ/dC_k equals
    sum_{s,i} 2 softplus(u) sigmoid(u) (v_{s,i} - Vdd): a closed-form check of
    every gradient entry at once, including the DC-point term (loads on at t = 0)."""
    from oracle import adjoint, transient
    net = pgsynth.config0(nx=9, ny=8)
    net.i_v = net.i_v.copy() * 40.0
    net.i_v[0::4] = 3e-3
    h, S = 10e-12, 20
    J, dG, dC = adjoint.gradients(net, h, S)
    V, _ = transient.transient(net, h, S)
    u = 1.0 - V[1:] - 0.05
    rhs = float(np.sum(2.0 * adjoint.softplus(u) * adjoint.sigmoid(u) * (V[1:] - net.vdd[0])))
    lhs = float(np.dot(net.r_g, dG) + np.dot(net.c_val, dC))
    assert abs(V[0] - net.vdd[0]).max() > 1e-4          # the DC point is not trivial
    assert lhs == pytest.approx(rhs, rel=1e-10)


# ---------------------------------------------------------------- initial conditions of Section IV-B

def test_paper_initial_conditions_capped_and_free_node():
    """Node 0 carries C and a pad G0; node 1 has no capacitor, joins node 0
    through g, has a pad g2 and a load I1 (constant) -- solved by hand:
      step 1: v1 = (g vc0 + g2 Vdd - I1) / (g + g2),
              i_c = -(G0 (vc0 - Vdd) + g (vc0 - v1))
      step 2: vc(h) = vc0 + h i_c / C
      step 3: v1(h) = (g vc(h) + g2 Vdd - I1) / (g + g2), v0(h) = vc(h)."""
    G0, g, g2, C, I1, vdd, vc0, h = 6.0, 1.5, 0.7, 40e-15, 2e-3, 1.0, 0.93, 10e-12
    net = make_netlist(2, [vdd], R=[(0, S(0), G0), (0, 1, g), (1, S(0), g2)], C=[(0, GROUND, C)],
                       I=[(1, GROUND, [0.0], [I1])])
    v0, v1, il1 = transient.paper_initial_conditions(net, h, vc0=[vc0])
    f0 = (g * vc0 + g2 * vdd - I1) / (g + g2)
    ic = -(G0 * (vc0 - vdd) + g * (vc0 - f0))
    vch = vc0 + h * ic / C
    f1 = (g * vch + g2 * vdd - I1) / (g + g2)
    np.testing.assert_allclose(v0, [vc0, f0], rtol=0, atol=1e-14)
    np.testing.assert_allclose(v1, [vch, f1], rtol=0, atol=1e-12)
    assert il1.size == 0


def test_paper_initial_conditions_lc_node():
    """C to ground and L to Vdd on one node, load I(t) ramping from I0 at t = 0:
    i_c(0) = -(i_l(0) + I0) (the inductor and the load both draw from the node),
    v(h) = vc0 + h i_c(0) / C, i_l(h) = i_l(0) + h (vc0 - Vdd) / L."""
    C, Lh, vdd, vc0, il0, I0, h = 50e-15, 4e-12, 1.0, 0.97, 3e-4, 1e-4, 2e-12
    net = make_netlist(1, [vdd], C=[(0, GROUND, C)], L=[(0, S(0), Lh)],
                       I=[(0, GROUND, [0.0, 1e-9], [I0, 0.0])])
    v0, v1, il1 = transient.paper_initial_conditions(net, h, vc0=[vc0], il0=[il0])
    ic = -(il0 + I0)
    np.testing.assert_allclose(v0, [vc0], rtol=0, atol=0)
    np.testing.assert_allclose(v1, [vc0 + h * ic / C], rtol=1e-15, atol=1e-15)
    np.testing.assert_allclose(il1, [il0 + h * (vc0 - vdd) / Lh], rtol=1e-14, atol=0)


def test_paper_initial_conditions_consistent_dc_state_is_stationary():
    """From the DC operating point (capacitors open, the default v_c(0)) with no
    load at t = 0 and t = h, nothing moves: v(h) = v(0) and i_l(h) = i_l(0);
    on an RLC grid with loads off until later, both levels are the supply."""
    net = pgsynth.config2(nx=7, ny=6)
    h = net.meta["h"]
    I = pwl.pwl_values(net.i_ptr, net.i_t, net.i_v, 0.0)
    Ih = pwl.pwl_values(net.i_ptr, net.i_t, net.i_v, h)
    net.i_v = net.i_v.copy()
    net.i_v[:] = np.where(np.repeat((I != 0) | (Ih != 0), np.diff(net.i_ptr)), 0.0, net.i_v)
    v0, v1, il1 = transient.paper_initial_conditions(net, h)
    np.testing.assert_allclose(v0, net.vdd[0], rtol=0, atol=1e-13)
    # i_c(0) is a KCL sum over up to ~40 S of conductance at ~1 V: rounding
    # 16 eps 40 A ~ 1.4e-13 A, which step 2 multiplies by h / C <= 200
    np.testing.assert_allclose(v1, v0, rtol=0, atol=5e-11)
    np.testing.assert_allclose(il1, 0.0, rtol=0, atol=1e-15)


def test_three_level_from_paper_initial_conditions_tracks_explicit_form():
    """Eq. 11 started from the two levels of Section IV-B equals the explicit
    form (Eq. 10) started from (v(h), i_l(h)) at t = h, step by step (direct
    solves: only rounding separates the two recurrences)."""
    net = pgsynth.config2(nx=6, ny=5)
    h = net.meta["h"]
    v0, v1, il1 = transient.paper_initial_conditions(net, h)
    V3 = [v for _, v in transient.simulate_three_level(net, h, 40, v0, v1)]
    VE, _ = transient.transient(net, h, 39, v0=v1, il0=il1, s0=1)
    np.testing.assert_allclose(np.stack(V3), VE[1:], rtol=0, atol=1e-11)


def _inductive_rlc():
    """A small RLC grid whose supply path is inductive: the pad resistors are
    weakened to 0.02 S (they keep the DC point defined) so that the pad
    inductors (h/L ~ 0.2-2 S) and the via inductors carry the dynamics."""
    net = pgsynth.config2(nx=6, ny=5)
    net.r_g = net.r_g.copy()
    net.r_g[np.asarray(net.r_b) < -1] = 0.02
    net.i_v = net.i_v.copy() * 20.0
    # every load starts its ramp 2 ps in, so the drops happen inside the short window
    net.i_t = net.i_t.copy()
    ptr = np.asarray(net.i_ptr)
    for e in range(len(ptr) - 1):
        net.i_t[ptr[e]:ptr[e + 1]] += 2e-12 - net.i_t[ptr[e]]
    return net


def _objective_difference(net_p, net_m, h, S, vref=1.0, margin=0.05):
    """J(net_p) - J(net_m) summed term by term over the two trajectories (no
    cancellation against the size of J)."""
    from oracle import adjoint
    Vp, _ = transient.transient(net_p, h, S)
    Vm, _ = transient.transient(net_m, h, S)
    sp = adjoint.softplus(vref - Vp[1:] - margin)
    sm = adjoint.softplus(vref - Vm[1:] - margin)
    return float(np.sum((sp - sm) * (sp + sm)))


def test_rlc_adjoint_matches_central_differences():
    """The oracle's RLC adjoint (explicit inductor currents, Eq. 10) against central
    finite differences of the forward objective, for inductors (vias and pad
    connections), resistors and capacitors, on a grid where the inductors matter
    (sum_e L_e |dJ/dL_e| is a sizeable fraction of sum_e g_e |dJ/dg_e|)."""
    from oracle import adjoint
    net = _inductive_rlc()
    h, S = net.meta["h"], 60
    J, dG, dC, dL = adjoint.gradients(net, h, S, with_l=True)
    assert J == pytest.approx(adjoint.objective(net, h, S), rel=1e-12)
    Lv = np.asarray(net.l_val)
    assert np.sum(Lv * np.abs(dL)) > 0.05 * np.sum(np.asarray(net.r_g) * np.abs(dG))
    rng = np.random.default_rng(11)
    pad_l = int(np.nonzero(np.asarray(net.l_b) < -1)[0][0])
    picks = [("l", int(k)) for k in rng.choice(len(net.l_val), 6, replace=False)] + [("l", pad_l)]
    picks += [("r", int(k)) for k in rng.choice(len(net.r_g), 4, replace=False)]
    picks += [("c", int(k)) for k in rng.choice(len(net.c_val), 4, replace=False)]
    field = {"l": "l_val", "r": "r_g", "c": "c_val"}
    grads = {"l": dL, "r": dG, "c": dC}
    for kind, k in picks:
        arr = getattr(net, field[kind])
        d = 1e-3 * arr[k]
        nets = []
        for sgn in (+1, -1):
            pert = arr.copy(); pert[k] += sgn * d
            nets.append(pgsynth.Netlist(**{**net.__dict__, field[kind]: pert}))
        fd = _objective_difference(nets[0], nets[1], h, S) / (2 * d)
        g = grads[kind][k]
        # central differences at 1e-3 relative: O(1e-6) truncation; the floor covers
        # parameters whose gradient is ~1e-6 of the largest of their kind
        assert g == pytest.approx(fd, rel=1e-4, abs=1e-6 * np.max(np.abs(grads[kind]))), (kind, k, g, fd)


def test_rlc_adjoint_scaling_identity():
    """g -> a g, C -> a C, L -> L / a maps v - Vdd to (v - Vdd)/a and leaves the
    inductor currents unchanged (Eq. 10 with one supply level), so
    sum g dJ/dg + sum C dJ/dC - sum L dJ/dL = sum 2 softplus(u) sigmoid(u) (v - Vdd)."""
    from oracle import adjoint
    net = _inductive_rlc()
    h, S = net.meta["h"], 60
    J, dG, dC, dL = adjoint.gradients(net, h, S, with_l=True)
    V, _ = transient.transient(net, h, S)
    u = 1.0 - V[1:] - 0.05
    rhs = float(np.sum(2.0 * adjoint.softplus(u) * adjoint.sigmoid(u) * (V[1:] - net.vdd[0])))
    lhs = float(np.dot(net.r_g, dG) + np.dot(net.c_val, dC) - np.dot(net.l_val, dL))
    assert abs(np.dot(net.l_val, dL)) > 1e-3 * abs(rhs)          # the inductor part is visible
    assert lhs == pytest.approx(rhs, rel=1e-9)
