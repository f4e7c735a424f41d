"""pg_autotune: the option search returns one of its candidates, and a grid
built with the chosen options still meets the 1e-6 V parity bar against the
oracle (every candidate runs under the same certified stopping rule, so tuning
may change only the time, never the accuracy)."""
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


def _parity(B, net, h, nsteps, opts):
    Vo, _ = transient.transient(net, h, nsteps)
    with B.Grid(net, **opts) as g:
        B.pg_set_stream(g.handle, torch.cuda.current_stream().cuda_stream)
        V = torch.empty((nsteps, net.n_nodes), dtype=torch.float64, device="cuda")
        st = B.pg_transient(g.handle, h, nsteps, v_all=V)
        err = float(np.max(np.abs(V.cpu().numpy() - Vo[1:])))
    assert st.failed_step == -1
    assert err <= TOL_V, f"max |v - v_oracle| = {err:.3e} V with {opts}"
    return st


@pytest.mark.parametrize("case", ["lattice3_mixed", "mesh_fp64", "batch_mixed"])
def test_autotune_choice_is_exact(B, case):
    if case == "lattice3_mixed":
        net, prec = pgsynth.config1(nx=97, ny=61), 1
    elif case == "mesh_fp64":
        net, prec = pgsynth.config0(nx=45, ny=38), 0
    else:
        net, prec = pgsynth.config3(n_grids=5, side_lo=16, side_hi=40, seed=2), 1
    h = net.meta["h"]
    best, ms = B.pg_autotune(net, h, 20, stream=torch.cuda.current_stream().cuda_stream, precision=prec)
    opts = B.options_dict(best)
    assert ms > 0.0 and opts["precision"] == prec
    assert opts["blocks_per_sm"] in (0, 1)
    assert opts["jacobi"] in (0, 1)
    assert opts["tile_rows"] in (0, 34, 66) and opts["colouring"] in (0, 2)
    if opts["colouring"] == 2:
        assert opts["lattice_sweeps"] <= 0            # a point-sweep order
    if opts["jacobi"]:
        assert opts["lattice_sweeps"] == -1
    elif prec == 1:
        assert opts["lattice_sweeps"] in (-1, 1, 2, 3)
        assert opts["inner_reduction"] in (1e-3, 1e-2, 1e-1)
    else:
        assert opts["lattice_sweeps"] == 0 and opts["inner_reduction"] == 0.0   # by grid class
    assert opts["omega"] == 0.0 or 1.0 < opts["omega"] < 2.0
    st = _parity(B, net, h, 50, opts)
    if opts["omega"] > 0.0:
        assert st.omega == opts["omega"]
