"""Load scenarios of one grid relaxed together (pg_transient_scenarios).

Every scenario is one right-hand side of the same backward-Euler system
(Eq. 2); the launch reads each coefficient once for all of them.  Each
scenario must match the FP64 oracle's direct solves of its own netlist, node
by node and step by step: with the point sweeps in both precisions and with
the lattice column-block tiles, for scenario counts that do not fill the last
group of four; its worst-drop waveform must equal that of the
copy-per-scenario batch.  Grids this entry point does not serve are refused
with PG_ERR_UNSUPPORTED.
"""
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


def _scenarios(net, n, seed):
    """n load patterns on the grid's breakpoints: each source's peak scaled by its own
    factor in [0, 2) (scenario 0 is the grid's own loads)."""
    rng = np.random.default_rng(seed)
    out = [np.asarray(net.i_v, dtype=np.float64)]
    for _ in range(n - 1):
        f = rng.uniform(0.0, 2.0, len(net.i_a))
        out.append(np.asarray(net.i_v) * np.repeat(f, np.diff(net.i_ptr)))
    return out


def _with_loads(net, iv):
    import copy
    m = copy.copy(net)
    m.i_v = iv
    return m


@pytest.mark.parametrize("solve", ["fp64_point", "mixed_point", "mixed_lattice"])
@pytest.mark.parametrize("recipe,n_scen", [("config0_37x29", 6), ("config1_21x17x3", 5), ("config0_20x18", 1),
                                           ("config1_43x39x3", 9)])
def test_every_scenario_matches_the_oracle(B, recipe, n_scen, solve):
    """Point sweeps (FP64 or FP32 with FP64 correction) and, on grids built for the
    lattice inner solve, its column-block tiles with four scenarios per region; the
    43 x 39 x 3 recipe spans several tiles with a ragged last row and column."""
    net = {"config0_37x29": lambda: pgsynth.config0(nx=37, ny=29),
           "config1_21x17x3": lambda: pgsynth.config1(nx=21, ny=17),
           "config0_20x18": lambda: pgsynth.config0(nx=20, ny=18),
           "config1_43x39x3": lambda: pgsynth.config1(nx=43, ny=39)}[recipe]()
    h, S = net.meta["h"], 30
    loads = _scenarios(net, n_scen, seed=n_scen)
    iv = torch.tensor(np.stack(loads), device="cuda")
    opts = {"fp64_point": dict(precision=0, lattice_sweeps=-1), "mixed_point": dict(precision=1, lattice_sweeps=-1),
            "mixed_lattice": dict(precision=1)}[solve]
    precision = opts["precision"]
    with B.Grid(net, **opts) as g:
        B.pg_set_stream(g.handle, torch.cuda.current_stream().cuda_stream)
        V = torch.empty((S, n_scen, net.n_nodes), dtype=torch.float64, device="cuda")
        vmin = torch.empty((S, n_scen), dtype=torch.float64, device="cuda")
        st = B.pg_transient_scenarios(g.handle, h, S, iv, v_all=V, vmin=vmin)
        torch.cuda.synchronize()
        V, vmin = V.cpu().numpy(), vmin.cpu().numpy()
    assert st.steps_done == S and st.failed_step == -1 and st.total_sweeps > 0
    assert (st.lattice_sweeps > 0) == (solve == "mixed_lattice")
    worst = 0.0
    for k in range(n_scen):
        Vo, _ = transient.transient(_with_loads(net, loads[k]), h, S)
        err = float(np.max(np.abs(V[:, k] - Vo[1:])))
        worst = max(worst, err)
        assert err <= TOL_V, f"scenario {k}: max |v - v_oracle| = {err:.3e} V"
        assert err <= st.err_bound + 1e-11
        np.testing.assert_array_equal(vmin[:, k], V[:, k].min(axis=1))
    assert st.err_bound <= 0.9 * TOL_V * (1 + 1e-9)
    print(f"{recipe}, {n_scen} scenarios, {solve}: max error {worst:.2e} V, "
          f"bound {st.err_bound:.2e} V, {st.total_sweeps} sweeps")


def test_shared_scenarios_match_the_copies(B):
    """The same nine scenarios as nine copies of the grid in one launch (each copy its own
    sub-circuit) and as nine right-hand sides of one grid: the same worst-drop waveforms."""
    from paper_1409_7166_gb300 import batch
    net = pgsynth.config0(nx=31, ny=27)
    h, S = net.meta["h"], 40
    loads = _scenarios(net, 9, seed=3)
    shared = batch.solve_scenarios_shared(net, loads, h, S, precision=1)
    shared_lat = batch.solve_scenarios_shared(net, loads, h, S, precision=1, lattice_sweeps=0)
    copies = batch.solve_scenarios(net, loads, h, S, precision=1)
    assert shared.shape == copies.shape == (S, 9)
    np.testing.assert_allclose(shared, copies, rtol=0, atol=2 * TOL_V)
    np.testing.assert_allclose(shared_lat, copies, rtol=0, atol=2 * TOL_V)


def test_unsupported_grids_are_refused(B):
    iv = torch.zeros((2, 1), dtype=torch.float64, device="cuda")
    rlc = pgsynth.config2(nx=12, ny=10)
    with B.Grid(rlc, lattice_sweeps=-1) as g:
        iv = torch.tensor(np.stack([rlc.i_v, rlc.i_v]), device="cuda")
        with pytest.raises(B.PGError) as e:
            B.pg_transient_scenarios(g.handle, rlc.meta["h"], 3, iv)
        assert e.value.name == "PG_ERR_UNSUPPORTED"
    rc = pgsynth.config1(nx=12, ny=10)
    with B.Grid(rc, precision=1, tile_rows=66) as g:        # the lattice solve on 66-row regions
        iv = torch.tensor(np.stack([rc.i_v]), device="cuda")
        with pytest.raises(B.PGError) as e:
            B.pg_transient_scenarios(g.handle, rc.meta["h"], 3, iv)
        assert e.value.name == "PG_ERR_UNSUPPORTED"
    with B.Grid(rc, precision=0, lattice_sweeps=3) as g:    # FP64 on the lattice inner solve
        assert B.pg_transient(g.handle, rc.meta["h"], 1).lattice_sweeps == 3
        B.pg_reset(g.handle)
        iv = torch.tensor(np.stack([rc.i_v]), device="cuda")
        with pytest.raises(B.PGError) as e:
            B.pg_transient_scenarios(g.handle, rc.meta["h"], 3, iv)
        assert e.value.name == "PG_ERR_UNSUPPORTED"
    with B.Grid(rc, precision=1, lattice_sweeps=-1) as g:  # loads on at t = 0: no v = Vdd start
        bad = np.asarray(rc.i_v).copy()
        bad[rc.i_ptr[0]] = 1e-3
        with pytest.raises(B.PGError) as e:
            B.pg_transient_scenarios(g.handle, rc.meta["h"], 3, torch.tensor(bad[None, :], device="cuda"))
        assert e.value.name == "PG_ERR_UNSUPPORTED"
