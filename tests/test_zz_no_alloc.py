"""pg_solve_noalloc: the solve entry point for callers that cannot allocate
device memory (memory reserved up front by another allocator or capped, or
loops that must not allocate).  It must give the same answer as pg_solve,
call after call, while keeping all its scratch in the library's fixed array.

This file is collected last on purpose, and passes both on its own in a fresh
process and after the rest of the suite.
"""
import numpy as np
import pytest

import pgsynth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_X = 1e-9     # the solve tolerance used in the parity tests (V)


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1409_7166_gb300 import binding
    return binding


@pytest.mark.parametrize("precision", [0, 1])
def test_noalloc_matches_pg_solve_twice(B, precision):
    net = pgsynth.config1(nx=75, ny=53)          # 11,925 nodes, 3 layers, ragged slices
    h = net.meta["h"]
    rng = np.random.default_rng(17)
    with B.Grid(net, precision=precision) as g:
        B.pg_set_stream(g.handle, torch.cuda.current_stream().cuda_stream)
        for trial in range(2):
            b = torch.tensor(rng.uniform(-1e-3, 1e-3, net.n_nodes), device="cuda")
            x_ref = torch.empty_like(b)
            B.pg_solve(g.handle, h, b, x_ref, TOL_X)
            for call in range(2):                  # two calls in a row share the scratch array
                x = torch.full_like(b, float("nan"))
                st = B.pg_solve_noalloc(g.handle, h, b, x, TOL_X)
                torch.cuda.synchronize()
                diff = float((x - x_ref).abs().max())
                assert diff <= 2 * TOL_X, f"trial {trial} call {call}: |x - x_ref| = {diff:.3e}"
                assert st.failed_step == -1 and st.total_sweeps > 0


def test_noalloc_allocates_nothing_and_serves_two_grids(B):
    """After grid creation (which sets up the fixed array) and one warm-up call, further
    calls must leave the device's free memory unchanged: they take no new allocation of
    any kind.  Two grids, solved alternately, both read and write the same array and must
    each still match their own pg_solve; the statistics must be pg_solve's."""
    nets = [pgsynth.config1(nx=61, ny=47), pgsynth.config0(nx=83, ny=71)]
    rng = np.random.default_rng(5)
    grids = [B.Grid(n, precision=p) for n, p in zip(nets, (1, 0))]
    try:
        stream = torch.cuda.current_stream().cuda_stream
        cases = []
        for g, net in zip(grids, nets):
            B.pg_set_stream(g.handle, stream)
            h = net.meta["h"]
            b = torch.tensor(rng.uniform(-1e-3, 1e-3, net.n_nodes), device="cuda")
            x_ref, x = torch.empty_like(b), torch.empty_like(b)
            st_ref = B.pg_solve(g.handle, h, b, x_ref, TOL_X)
            B.pg_solve_noalloc(g.handle, h, b, x, TOL_X)            # warm-up
            cases.append((g, h, b, x_ref, x, st_ref))
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for rep in range(3):
            for g, h, b, x_ref, x, st_ref in cases:
                x.fill_(float("nan"))
                st = B.pg_solve_noalloc(g.handle, h, b, x, TOL_X)
                torch.cuda.synchronize()
                diff = float((x - x_ref).abs().max())
                assert diff <= 2 * TOL_X, f"rep {rep}: |x - x_ref| = {diff:.3e}"
                for k in ("kappa", "kacc", "step_tol", "omega", "lattice_sweeps"):
                    assert getattr(st, k) == getattr(st_ref, k), k
                assert st.failed_step == -1
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] >= free0, "pg_solve_noalloc changed the free device memory"
    finally:
        for g in grids:
            g.close()


def test_noalloc_rejects_unassembled_h_and_oversize(B):
    net = pgsynth.config0(nx=20, ny=20)
    with B.Grid(net) as g:
        b = torch.zeros(net.n_nodes, dtype=torch.float64, device="cuda")
        x = torch.empty_like(b)
        with pytest.raises(B.PGError) as e:
            B.pg_solve_noalloc(g.handle, net.meta["h"], b, x, 1e-9)   # h never assembled
        assert e.value.name == "PG_ERR_INVALID_ARG"
    big = pgsynth.config0(nx=1000, ny=900)                            # 900k nodes > FP64 limit
    with B.Grid(big) as g:
        b = torch.zeros(big.n_nodes, dtype=torch.float64, device="cuda")
        x = torch.empty_like(b)
        B.pg_solve(g.handle, big.meta["h"], b, x, 1e-9)
        with pytest.raises(B.PGError) as e:
            B.pg_solve_noalloc(g.handle, big.meta["h"], b, x, 1e-9)
        assert e.value.name == "PG_ERR_INVALID_ARG" and "maximum" in str(e.value)
