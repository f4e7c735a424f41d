"""pg_transient_async: the persistent transient as stream-ordered work captured
once into a CUDA graph and replayed for several load scenarios (new PWL
waveforms through pg_update_sources between replays).

Each replay must equal, bit for bit, the synchronous pg_transient of the same
scenario (same kernel, same state, same parameters), and the oracle's direct
solves of that scenario to 1e-6 V (Eq. 2, every node, every step).
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


def _scenarios(net, k):
    """k load patterns on the same breakpoints: every source rescaled by its own
    factor in [0.2, 1.5] (zero stays zero, so every load is still off at t = 0)."""
    n_src = len(net.i_ptr) - 1
    out = [net.i_v]
    for s in range(1, k):
        f = np.random.default_rng(100 + s).uniform(0.2, 1.5, n_src)
        out.append(net.i_v * np.repeat(f, np.diff(net.i_ptr)))
    return out


@pytest.mark.parametrize("precision", [0, 1])
def test_graph_replay_of_batched_grids(B, precision):
    net = pgsynth.config3(n_grids=5, side_lo=16, side_hi=40, seed=2)
    h, S, n = net.meta["h"], 60, net.n_nodes
    dev = "cuda"
    with B.Grid(net, precision=precision) as g:
        B.pg_set_stream(g.handle, torch.cuda.current_stream().cuda_stream)
        B.pg_transient(g.handle, h, 0)                      # assemble h before capturing
        V = torch.empty((S, n), dtype=torch.float64, device=dev)
        vmin = torch.empty(S, dtype=torch.float64, device=dev)
        rec = torch.zeros(B.PG_ASYNC_STATS_BYTES, dtype=torch.uint8, device=dev)
        graph = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream()
        with torch.cuda.graph(graph, stream=side):
            B.pg_set_stream(g.handle, side.cuda_stream)
            B.pg_transient_async(g.handle, h, S, v_all=V, vmin=vmin, dstats=rec)
        B.pg_set_stream(g.handle, torch.cuda.current_stream().cuda_stream)
        for iv in _scenarios(net, 3):
            B.pg_update_sources(g.handle, i_v=iv)
            graph.replay()
            torch.cuda.synchronize()
            rc, st = B.pg_async_stats(g.handle, rec)
            assert rc == 0 and st.steps_done == S and st.failed_step == -1
            assert st.max_step_bound <= st.step_tol * 1.0000001
            Vg = V.clone()
            B.pg_reset(g.handle)
            V2 = torch.empty_like(V)
            st2 = B.pg_transient(g.handle, h, S, v_all=V2)
            assert torch.equal(Vg, V2) and st2.total_sweeps == st.total_sweeps
            assert torch.equal(vmin, V2.min(dim=1).values)
            Vo, _ = transient.transient(pgsynth.Netlist(**{**net.__dict__, "i_v": iv}), h, S)
            err = float(np.max(np.abs(Vg.cpu().numpy() - Vo[1:])))
            assert err <= TOL_V, f"max |v - v_oracle| = {err:.3e} V"


def test_async_from_given_state(B):
    """v0 given on the device: the launch starts from it at step 0, exactly like
    pg_set_state followed by pg_transient, and matches the oracle's transient
    from the same state."""
    net = pgsynth.config0(nx=30, ny=24)
    h, n, S = net.meta["h"], net.n_nodes, 30
    ref = 1.0 - 0.01 * np.random.default_rng(3).random(n)
    with B.Grid(net, precision=1) as g:
        B.pg_set_stream(g.handle, torch.cuda.current_stream().cuda_stream)
        v0 = torch.tensor(ref, device="cuda")
        V = torch.empty((S, n), dtype=torch.float64, device="cuda")
        rec = torch.zeros(B.PG_ASYNC_STATS_BYTES, dtype=torch.uint8, device="cuda")
        B.pg_transient_async(g.handle, h, S, v0=v0, v_all=V, dstats=rec)
        rc, st = B.pg_async_stats(g.handle, rec)
        assert rc == 0 and st.steps_done == S
        B.pg_set_state(g.handle, v0)
        V2 = torch.empty_like(V)
        B.pg_transient(g.handle, h, S, v_all=V2)
        assert torch.equal(V, V2)
    Vo, _ = transient.transient(net, h, S, v0=ref)
    assert np.max(np.abs(V.cpu().numpy() - Vo[1:])) <= TOL_V


def test_async_rejects_host_buffers(B):
    """Host memory is refused before anything is enqueued: by the binding, and by
    the library's own pointer check for callers of the C ABI."""
    import ctypes as C
    net = pgsynth.config0(nx=12, ny=10)
    h = net.meta["h"]
    host = np.zeros((5, net.n_nodes))
    with B.Grid(net) as g:
        with pytest.raises(TypeError):
            B.pg_transient_async(g.handle, h, 5, v_all=host)
        out = B.pg_output()
        out.on_host = 0
        out.v_all = C.c_void_p(host.ctypes.data)
        rc = B.lib().pg_transient_async(g.handle, float(h), 5, None, C.byref(out), None)
        assert rc == B.PG_ERR_INVALID_ARG
        rc = B.lib().pg_transient_async(g.handle, float(h), 0, None, None, None)
        assert rc == B.PG_ERR_INVALID_ARG
