"""The initial-condition procedure of Section IV-B (pg_initial_conditions) and
the three-level recurrence of Eq. 11 / Eq. 14 (PG_FORM_THREE_LEVEL) against the
oracle's literal versions (direct solves)."""
import numpy as np
import pytest

import pgsynth
from oracle import transient

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_V = 1e-6


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1409_7166_gb300 import binding
    return binding


def _state(B, g, net):
    v = np.zeros(net.n_nodes)
    il = np.zeros(max(len(net.l_val), 1))
    step = B.pg_get_state(g.handle, v, il if len(net.l_val) else None)
    return step, v, il[:len(net.l_val)]


def test_initial_conditions_rlc_default_vc(B):
    net = pgsynth.config2(nx=40, ny=33)
    h = net.meta["h"]
    il0 = np.random.default_rng(1).uniform(-1e-4, 1e-4, len(net.l_val))
    v0o, v1o, il1o = transient.paper_initial_conditions(net, h, il0=il0)
    with B.Grid(net, precision=0) as g:
        B.pg_initial_conditions(g.handle, h, il0=il0)
        step, v, il = _state(B, g, net)
    assert step == 1
    assert np.max(np.abs(v - v1o)) <= TOL_V
    assert np.max(np.abs(il - il1o)) <= 1e-3 * np.max(np.abs(il1o))


def test_initial_conditions_every_node_capped_is_exact(B):
    """Every node carries a capacitor: both DC analyses are fully fixed, so the
    levels are the given v_c(0) and its forward update, computed exactly."""
    net = pgsynth.config0(nx=23, ny=19)
    h = net.meta["h"]
    vc0 = 1.0 - 0.03 * np.random.default_rng(2).random(len(net.c_val))
    v0o, v1o, _ = transient.paper_initial_conditions(net, h, vc0=vc0)
    with B.Grid(net, precision=0) as g:
        B.pg_initial_conditions(g.handle, h, vc0=vc0)
        step, v, _ = _state(B, g, net)
    assert step == 1
    # i_c is a KCL sum of a few conductances (<= 8 S at ~1 V): rounding ~16 eps 8, times h / C <= 1000
    assert np.max(np.abs(v - v1o)) <= 1e-11


def test_initial_conditions_rlc_given_vc(B):
    net = pgsynth.config2(nx=31, ny=27)
    h = net.meta["h"]
    vc0 = 1.0 - 0.02 * np.random.default_rng(3).random(len(net.c_val))
    v0o, v1o, il1o = transient.paper_initial_conditions(net, h, vc0=vc0)
    with B.Grid(net, precision=0) as g:
        B.pg_initial_conditions(g.handle, h, vc0=vc0)
        step, v, il = _state(B, g, net)
    assert np.max(np.abs(v - v1o)) <= TOL_V
    assert np.max(np.abs(il - il1o)) <= 1e-3 * max(np.max(np.abs(il1o)), 1e-9)


@pytest.mark.parametrize("precision", [0, 1])
def test_three_level_rlc_matches_oracle(B, precision):
    net = pgsynth.config2(nx=40, ny=33)
    h, S = net.meta["h"], 300
    v0o, v1o, _ = transient.paper_initial_conditions(net, h)
    Vo = np.stack([v for _, v in transient.simulate_three_level(net, h, S + 1, v0o, v1o)])
    with B.Grid(net, precision=precision, form=B.PG_FORM_THREE_LEVEL) as g:
        B.pg_set_stream(g.handle, torch.cuda.current_stream().cuda_stream)
        B.pg_initial_conditions(g.handle, h)
        V = torch.empty((S, net.n_nodes), dtype=torch.float64, device="cuda")
        st = B.pg_transient(g.handle, h, S, v_all=V)
        err = float(np.max(np.abs(V.cpu().numpy() - Vo)))
    assert st.failed_step == -1 and np.isnan(st.err_bound)
    assert err <= TOL_V, f"max |v - v_oracle| = {err:.3e} V"


def test_three_level_rc_matches_oracle(B):
    net = pgsynth.config0(nx=37, ny=29)
    h, S = net.meta["h"], 100
    vc0 = 1.0 - 0.01 * np.random.default_rng(4).random(len(net.c_val))
    v0o, v1o, _ = transient.paper_initial_conditions(net, h, vc0=vc0)
    Vo = np.stack([v for _, v in transient.simulate_three_level(net, h, S + 1, v0o, v1o)])
    with B.Grid(net, precision=0, form=B.PG_FORM_THREE_LEVEL, tol=1e-8) as g:
        B.pg_initial_conditions(g.handle, h, vc0=vc0)
        V = np.zeros((S, net.n_nodes))
        B.pg_transient(g.handle, h, S, v_all=V)
    assert np.max(np.abs(V - Vo)) <= TOL_V


def test_three_level_from_dc_point_takes_one_be_step_first(B):
    """From a single level (the DC point) the first step is a backward-Euler
    step, then Eq. 11 runs on (v(0), v(1)): equal to the oracle's explicit first
    step followed by its three-level recurrence."""
    net = pgsynth.config2(nx=33, ny=28)
    h, S = net.meta["h"], 200
    V1, IL1 = transient.transient(net, h, 1)
    Vo = np.stack([V1[1]] + [v for _, v in transient.simulate_three_level(net, h, S, V1[0], V1[1])])
    with B.Grid(net, precision=0, form=B.PG_FORM_THREE_LEVEL) as g:
        V = np.zeros((S, net.n_nodes))
        B.pg_transient(g.handle, h, S, v_all=V)
    assert np.max(np.abs(V - Vo)) <= TOL_V


def test_three_level_keeps_no_currents_and_rejects_unknown_form(B):
    net = pgsynth.config2(nx=12, ny=10)
    h = net.meta["h"]
    with B.Grid(net, form=B.PG_FORM_THREE_LEVEL) as g:
        with pytest.raises(B.PGError):
            B.pg_transient(g.handle, h, 5, il_all=np.zeros((5, len(net.l_val))))
        st = B.pg_transient(g.handle, h, 5)
        assert st.steps_done == 5
    with pytest.raises(B.PGError):
        B.Grid(net, form=7)
