"""The batched workload on the GPU: per-component worst drop (pg_output.comp_vmin)
and the sharded driver (one rank here) against the oracle, each grid solved on
its own by direct solves (independent sub-circuits, Fig. 1)."""
import numpy as np
import pytest

import pgsynth
from oracle import transient
from paper_1409_7166_gb300 import batch

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


@pytest.mark.parametrize("precision", [0, 1])
def test_component_minima_match_full_field(B, precision):
    parts = [p for _, p in pgsynth.config3_parts(n_grids=6, side_lo=12, side_hi=45, seed=8)]
    net = batch.concat(parts)
    h, S = 10e-12, 40
    with B.Grid(net, precision=precision) as g:
        B.pg_set_stream(g.handle, torch.cuda.current_stream().cuda_stream)
        nc, comp = B.pg_grid_components(g.handle, net.n_nodes)
        assert nc == len(parts)
        assert np.array_equal(comp, np.repeat(np.arange(nc), [p.n_nodes for p in parts]))
        V = torch.empty((S, net.n_nodes), dtype=torch.float64, device="cuda")
        CV = torch.empty((S, nc), dtype=torch.float64, device="cuda")
        B.pg_transient(g.handle, h, S, v_all=V, comp_vmin=CV)
        V, CV = V.cpu().numpy(), CV.cpu().numpy()
    off = 0
    for j, p in enumerate(parts):
        assert np.array_equal(CV[:, j], V[:, off:off + p.n_nodes].min(axis=1))
        off += p.n_nodes


def test_sharded_driver_matches_oracle_per_grid(B):
    parts = [p for _, p in pgsynth.config3_parts(n_grids=5, side_lo=16, side_hi=40, seed=2)]
    h, S = 10e-12, 50
    res = batch.solve_sharded(parts, h, S, precision=1)
    for j, p in enumerate(parts):
        Vo, _ = transient.transient(p, h, S)
        err = float(np.max(np.abs(res[:, j] - Vo[1:].min(axis=1))))
        assert err <= TOL_V, f"grid {j}: {err:.3e} V"


@pytest.mark.parametrize("precision", [0, 1])
def test_load_scenarios_in_one_launch(B, precision):
    """Several load scenarios of one grid in one launch: each scenario's worst-drop
    waveform equals the oracle's for that scenario alone."""
    net = pgsynth.config0(nx=23, ny=19)
    h, S = net.meta["h"], 40
    rng = np.random.default_rng(21)
    n_src = len(net.i_ptr) - 1
    scen = [net.i_v * np.repeat(rng.uniform(0.2, 3.0, n_src), np.diff(net.i_ptr)) for _ in range(5)]
    res = batch.solve_scenarios(net, scen, h, S, precision=precision)
    assert res.shape == (S, 5)
    for j, iv in enumerate(scen):
        Vo, _ = transient.transient(pgsynth.Netlist(**{**net.__dict__, "i_v": iv}), h, S)
        err = float(np.max(np.abs(res[:, j] - Vo[1:].min(axis=1))))
        assert err <= TOL_V, f"scenario {j}: {err:.3e} V"
