"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Every comparison is element by element against the oracle's direct-solve
trajectory on the same seeded netlist.  The tolerance is the contract's
1e-6 V max-abs on node voltages; the library's own certified bound must also
be below it.
"""
import numpy as np
import pytest

import pgsynth
from pgsynth import GROUND, make_netlist, source_terminal as S
from oracle import bounds, transient

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


def run_gpu(B, net, h, nsteps, precision, **opts):
    with B.Grid(net, precision=precision, **opts) as g:
        B.pg_set_stream(g.handle, torch.cuda.current_stream().cuda_stream)
        V = torch.empty((nsteps, net.n_nodes), dtype=torch.float64, device="cuda")
        nl = len(net.l_val)
        IL = torch.empty((nsteps, max(nl, 1)), dtype=torch.float64, device="cuda") if nl else None
        vmin = torch.empty(nsteps, dtype=torch.float64, device="cuda")
        vnode = torch.empty(nsteps, dtype=torch.int32, device="cuda")
        st = B.pg_transient(g.handle, h, nsteps, v_all=V, il_all=IL, vmin=vmin, vmin_node=vnode)
        torch.cuda.synchronize()
        return (V.cpu().numpy(), None if IL is None else IL.cpu().numpy(), vmin.cpu().numpy(),
                vnode.cpu().numpy(), st)


def check_against_oracle(B, net, h, nsteps, precision, **opts):
    Vo, ILo = transient.transient(net, h, nsteps)
    V, IL, vmin, vnode, st = run_gpu(B, net, h, nsteps, precision, **opts)
    err = np.max(np.abs(V - Vo[1:]))
    assert err <= TOL_V, f"max |v - v_oracle| = {err:.3e} V"
    if IL is not None:
        il_err = np.max(np.abs(IL - ILo[1:]))
        assert il_err <= 1e-3 * max(np.max(np.abs(ILo)), 1e-6), f"inductor current error {il_err:.3e} A"
    # per-step worst drop: the value matches; the node attains the minimum of the GPU field
    np.testing.assert_allclose(vmin, Vo[1:].min(axis=1), rtol=0, atol=TOL_V)
    assert np.all(V[np.arange(nsteps), vnode] == vmin)
    assert st.steps_done == nsteps and st.failed_step == -1
    assert st.max_step_bound <= st.step_tol * 1.0000001
    if np.isfinite(st.err_bound):
        # the certificate bounds the actual error (the oracle's direct solves: ~1e-12 V)
        assert err <= st.err_bound + 1e-11, (err, st.err_bound)
        assert st.kacc * st.max_step_bound <= st.err_bound * 1.0000001 <= 0.9 * TOL_V * 1.0000002
    return err, st


@pytest.mark.parametrize("precision", [0, 1])
def test_config0_full_size(B, precision):
    """RC 100x100 mesh, 100 steps of 10 ps: every node, every step."""
    net = pgsynth.config0()
    err, st = check_against_oracle(B, net, net.meta["h"], net.meta["nsteps"], precision)
    assert st.err_bound <= TOL_V


def test_config1_recipe_ragged(B):
    """3-layer recipe at 97x61x3 (odd sides: colours of unequal size, ragged last slice),
    FP32 sweeps with FP64 defect correction."""
    net = pgsynth.config1(nx=97, ny=61)
    check_against_oracle(B, net, net.meta["h"], 60, 1)


def test_config2_recipe_rlc(B):
    """RLC recipe (R||L vias and pads) at 40x33x2, FP64, 300 steps of 2 ps."""
    net = pgsynth.config2(nx=40, ny=33)
    check_against_oracle(B, net, net.meta["h"], 300, 0)


def test_config3_recipe_batched(B):
    """Several independent grids of uneven size in one netlist (components)."""
    net = pgsynth.config3(n_grids=5, side_lo=17, side_hi=45)
    check_against_oracle(B, net, net.meta["h"], 40, 1)


def test_non_bipartite_multicolour(B):
    """A triangulated mesh is not 2-colourable: the greedy multicolour path."""
    n = 12
    ids = np.arange(n * n).reshape(n, n)
    rng = np.random.default_rng(5)
    R = []
    for y in range(n):
        for x in range(n):
            if x + 1 < n: R.append((ids[y, x], ids[y, x + 1], rng.uniform(0.5, 2)))
            if y + 1 < n: R.append((ids[y, x], ids[y + 1, x], rng.uniform(0.5, 2)))
            if x + 1 < n and y + 1 < n: R.append((ids[y, x], ids[y + 1, x + 1], rng.uniform(0.5, 2)))
    R += [(ids[0, 0], S(0), 10.0), (ids[n - 1, n - 1], S(0), 10.0)]
    C = [(int(i), GROUND, rng.uniform(10e-15, 100e-15)) for i in range(n * n)]
    I = [(int(i), GROUND, [0.0, 30e-12, 90e-12], [0.0, rng.uniform(0, 1e-3), 0.0])
         for i in rng.choice(n * n, 30, replace=False)]
    net = make_netlist(n * n, [1.0], R=R, C=C, I=I)
    info_net = net
    err, st = check_against_oracle(B, info_net, 10e-12, 20, 0)
    with B.Grid(net) as g:
        assert g.info["n_colours"] >= 3


def test_nontrivial_dc_initial_condition(B):
    """Resistors to ground and loads already on at t = 0: the DC operating point
    (capacitors open) is solved on the device before the first step."""
    net = pgsynth.config0(nx=23, ny=19)
    extra = np.arange(0, net.n_nodes, 37, dtype=np.int32)
    net.r_a = np.concatenate([net.r_a, extra])
    net.r_b = np.concatenate([net.r_b, np.full(extra.size, GROUND, np.int32)])
    net.r_g = np.concatenate([net.r_g, np.full(extra.size, 0.05)])
    net.i_v = net.i_v.copy()
    net.i_v[0::3] = 2e-4                      # every load starts at 0.2 mA
    check_against_oracle(B, net, net.meta["h"], 30, 0)


def test_single_node_closed_form(B):
    """One node (a slice of one real node and 127 padding nodes): the exact
    discrete decay v_k - Vdd = (v0 - Vdd)(1 + h G0/C)^-k."""
    C0, g0, h = 50e-15, 10.0, 1e-15
    net = make_netlist(1, [1.0], R=[(0, S(0), g0)], C=[(0, GROUND, C0)])
    with B.Grid(net) as g:
        B.pg_set_state(g.handle, np.array([0.5]))
        V = np.zeros((40, 1))
        B.pg_transient(g.handle, h, 40, v_all=V)
    k = np.arange(1, 41)
    np.testing.assert_allclose(V[:, 0], 1.0 - 0.5 * (1 + h * g0 / C0) ** (-k), rtol=0, atol=TOL_V)


def test_zero_load_is_exactly_vdd(B):
    net = pgsynth.config1(nx=40, ny=24)
    net.i_v[:] = 0.0
    V, _, _, _, st = run_gpu(B, net, net.meta["h"], 10, 1)
    assert np.all(V == 1.0) and st.total_sweeps == 0


def test_bounds_are_upper_bounds(B):
    """kappa >= ||M^-1 D||_inf and q >= ||M^-1 C/h||_inf (oracle, exact)."""
    net = pgsynth.config0(nx=40, ny=30)
    h = net.meta["h"]
    _, _, _, _, st = run_gpu(B, net, h, 2, 0)
    kx = bounds.scaled_minv_inf_norm(net, h)
    qx = bounds.step_gain(net, h)
    ax = bounds.accumulation_gain(net, h)
    assert kx <= st.kappa <= kx * 1.01
    assert qx <= st.q <= qx + 0.01
    assert ax <= st.kacc <= ax + 0.01
    assert st.kacc <= 1.0 / (1.0 - st.q)


def test_resume_equals_one_run(B):
    """get/set state: 20 + 20 steps from a saved state equal 40 steps at once."""
    net = pgsynth.config0(nx=30, ny=26)
    h = net.meta["h"]
    V1, _, _, _, _ = run_gpu(B, net, h, 40, 0)
    with B.Grid(net) as g:
        B.pg_transient(g.handle, h, 20)
        v = np.zeros(net.n_nodes)
        step = B.pg_get_state(g.handle, v)
        assert step == 20
    with B.Grid(net) as g2:
        B.pg_set_state(g2.handle, v, step=20)   # extrapolation restarts from V(s-1)
        V2 = np.zeros((20, net.n_nodes))
        B.pg_transient(g2.handle, h, 20, v_all=V2)
    np.testing.assert_allclose(V2, V1[20:], rtol=0, atol=TOL_V)


def test_step_lockstep_and_solve(B):
    net = pgsynth.config0(nx=21, ny=18)
    h = net.meta["h"]
    Vo, _ = transient.transient(net, h, 5)
    with B.Grid(net) as g:
        out = torch.empty(net.n_nodes, dtype=torch.float64, device="cuda")
        for s in range(1, 6):
            B.pg_step(g.handle, h, out)
            torch.cuda.synchronize()
            assert np.max(np.abs(out.cpu().numpy() - Vo[s])) <= TOL_V
        # pg_solve: M x = b against a direct solve
        from oracle.matrices import nodal_matrices
        M = nodal_matrices(net).system_matrix(h)
        b = np.random.default_rng(0).uniform(-1e-3, 1e-3, net.n_nodes)
        x_ref = transient.DirectSolver(M).solve(b)
        bt = torch.tensor(b, device="cuda")
        xt = torch.empty_like(bt)
        B.pg_solve(g.handle, h, bt, xt, 1e-9)
        torch.cuda.synchronize()
        assert np.max(np.abs(xt.cpu().numpy() - x_ref)) <= 1e-9


def test_update_sources_new_scenario(B):
    net = pgsynth.config0(nx=26, ny=22)
    h = net.meta["h"]
    net2 = pgsynth.config0(nx=26, ny=22, seed=11)
    net2.i_a = net.i_a; net2.i_b = net.i_b; net2.i_ptr = net.i_ptr   # same load sites, new waveforms
    scen = pgsynth.Netlist(**{**net.__dict__, "i_t": net2.i_t, "i_v": net2.i_v})
    Vo, _ = transient.transient(scen, h, 25)
    with B.Grid(net) as g:
        B.pg_transient(g.handle, h, 10)
        B.pg_update_sources(g.handle, net2.i_t, net2.i_v)
        B.pg_reset(g.handle)
        V = np.zeros((25, net.n_nodes))
        B.pg_transient(g.handle, h, 25, v_all=V)
    assert np.max(np.abs(V - Vo[1:])) <= TOL_V


def _jump_waveforms(net, h, seed):
    """Five-point waveforms on the recipe's load sites: a zero-length segment (a jump) at
    the rise and another at the fall, every breakpoint on an exact step time k h."""
    rng = np.random.default_rng(seed)
    m = len(net.i_ptr) - 1
    ptr = np.arange(0, 5 * m + 1, 5, dtype=np.int64)
    t = np.empty(5 * m)
    v = np.empty(5 * m)
    for e in range(m):
        peak = float(np.max(np.abs(net.i_v[net.i_ptr[e]:net.i_ptr[e + 1]]))) * rng.uniform(0.5, 1.5)
        ka = int(rng.integers(1, 60))
        kb = ka + int(rng.integers(1, 8))
        kc = kb + int(rng.integers(1, 8))
        t[5 * e:5 * e + 5] = [ka * h, ka * h, kb * h, kc * h, kc * h]
        v[5 * e:5 * e + 5] = [0.0, peak, 0.5 * peak, 0.3 * peak, 0.0]
    return pgsynth.Netlist(**{**net.__dict__, "i_ptr": ptr, "i_t": t, "i_v": v})


@pytest.mark.parametrize("precision", [1, 0])
def test_pwl_jumps_and_breakpoints_on_step_times(B, precision):
    """Breakpoints hit exactly by step times and zero-length segments: the held value on
    each side of a jump follows the PWL reading of Section II-A on both sides (left value
    at the jump's time, the next segment just after)."""
    net = _jump_waveforms(pgsynth.config1(nx=43, ny=39), pgsynth.config1().meta["h"], 5)
    check_against_oracle(B, net, net.meta["h"], 90, precision)


def test_update_sources_new_breakpoints(B):
    """New breakpoint times and values through pg_update_sources: the device evaluation
    (segment cursors, time keys, slopes) follows the new waveforms from the next run."""
    base = pgsynth.config1(nx=43, ny=39)
    h = base.meta["h"]
    net1, net2 = _jump_waveforms(base, h, 5), _jump_waveforms(base, h, 6)
    Vo, _ = transient.transient(net2, h, 90)
    with B.Grid(net1, precision=1) as g:
        B.pg_transient(g.handle, h, 40)              # cursors advanced on the first waveforms
        B.pg_update_sources(g.handle, net2.i_t, net2.i_v)
        B.pg_reset(g.handle)
        V = np.zeros((90, net2.n_nodes))
        B.pg_transient(g.handle, h, 90, v_all=V)
    assert np.max(np.abs(V - Vo[1:])) <= TOL_V


def test_not_converged_and_timeout_are_reported(B):
    net = pgsynth.config0(nx=30, ny=30)
    h = net.meta["h"]
    with B.Grid(net, max_sweeps=2) as g:
        rc, st = B.pg_transient_status(g.handle, h, 50)
        assert B.STATUS[rc] == "PG_ERR_NOT_CONVERGED"
        assert st.failed_step >= 1
    # a block that never arrives at the first barrier: the others give up after the limit
    with B.Grid(net, debug_flags=B.PG_DEBUG_SKIP_ARRIVAL, barrier_timeout_s=0.05) as g:
        rc, st = B.pg_transient_status(g.handle, h, 5)
        assert B.STATUS[rc] == "PG_ERR_TIMEOUT"
    # the context is still usable afterwards
    check_against_oracle(B, pgsynth.config0(nx=12, ny=12), h, 5, 0)


@pytest.mark.parametrize("shape,k", [((97, 61, 3), 2), ((96, 64, 3), 2), ((96, 64, 3), 1), ((64, 48, 1), 2),
                                     ((40, 36, 2), 3)])
def test_lattice_block_inner_solve(B, shape, k):
    """The shared-memory column-block red-black inner solve (lattice grids, mixed
    precision): odd sides use 4-byte region copies, multiples of 4 the 16-byte path;
    1, 2 and 3 layers; k sweeps per device barrier."""
    nx, ny, nl = shape
    net = pgsynth.config1(nx=nx, ny=ny, nl=nl) if nl > 1 else pgsynth.config0(nx=nx, ny=ny)
    with B.Grid(net, precision=1, lattice_sweeps=k) as g:
        assert g.info["n_nodes"] == nx * ny * nl
    check_against_oracle(B, net, net.meta["h"], 40, 1, lattice_sweeps=k)


def test_batched_lattices_skip_converged_grids(B):
    """A batch of lattices (1 and 2 layers) where some grids carry no load: those
    converge at once and their tiles are skipped while the others iterate; every
    node still matches the oracle.  Also checks the lattice inner solve is the one
    that ran."""
    net = pgsynth.config3(n_grids=7, side_lo=20, side_hi=52, seed=2)
    parts = pgsynth.config3_parts(n_grids=7, side_lo=20, side_hi=52, seed=2)
    net.i_v = net.i_v.copy()
    ptr = net.i_ptr
    for k in (1, 4):                                  # silence every load of grids 1 and 4
        off, p = parts[k]
        sel = (net.i_a >= off) & (net.i_a < off + p.n_nodes)
        for e in np.nonzero(sel)[0]:
            net.i_v[ptr[e]:ptr[e + 1]] = 0.0
    assert any(p.lattice[2] == 2 for _, p in parts) and any(p.lattice[2] == 1 for _, p in parts)
    err, st = check_against_oracle(B, net, net.meta["h"], 50, 1)
    assert st.lattice_sweeps == 3          # the automatic choice for lattices like these


@pytest.mark.parametrize("precision", [0, 1])
def test_damped_jacobi_inner_sweeps(B, precision):
    """The damped-Jacobi inner sweep (every node from the previous iterate) reaches
    the same certified solution as the coloured SOR, with more sweeps."""
    net = pgsynth.config0(nx=33, ny=27)
    h = net.meta["h"]
    err, st_j = check_against_oracle(B, net, h, 30, precision, jacobi=1)
    _, st_s = check_against_oracle(B, net, h, 30, precision)
    assert st_j.omega == 1.0 and st_j.total_sweeps > st_s.total_sweeps
    # damping
    err, st_d = check_against_oracle(B, net, h, 10, precision, jacobi=1, omega=0.8)
    assert st_d.omega == 0.8


@pytest.mark.parametrize("precision", [0, 1])
def test_grid_without_capacitors(B, precision):
    """No capacitors: M = G + G0 and every step is a DC solve at the step's loads
    (q = 0, accumulation gain 1)."""
    net = pgsynth.config0(nx=19, ny=14)
    for k in ("c_a", "c_b"):
        setattr(net, k, np.zeros(0, np.int32))
    net.c_val = np.zeros(0)
    err, st = check_against_oracle(B, net, net.meta["h"], 25, precision)
    assert st.q == 0.0 and st.kacc == 1.0


def test_lattices_smaller_than_a_tile(B):
    """Lattice inner solve on lattices smaller than one tile's interior (26 x 26
    columns for k = 2), alone and batched with a larger one."""
    from paper_1409_7166_gb300 import batch
    tiny = pgsynth.config1(nx=5, ny=3)
    check_against_oracle(B, tiny, tiny.meta["h"], 20, 1, lattice_sweeps=2)
    parts = [pgsynth.config1(nx=5, ny=3), pgsynth.config1(nx=30, ny=27), pgsynth.config1(nx=2, ny=7)]
    net = batch.concat(parts)
    Vo, _ = transient.transient(net, tiny.meta["h"], 20)
    V, _, _, _, st = run_gpu(B, net, tiny.meta["h"], 20, 1, lattice_sweeps=2)
    assert st.lattice_sweeps == 2
    assert np.max(np.abs(V - Vo[1:])) <= TOL_V


@pytest.mark.parametrize("precision", [0, 1])
def test_load_aware_warm_start(B, precision):
    """warm_start = 2 damps the extrapolation once the loads have been constant for two
    steps.  It only moves the starting point, so parity holds.  The 3-layer recipe's loads
    all finish within 1.2 ns (240 steps of 5 ps), so 300 steps include a quiet stretch.
    There the damped start saves sweeps on the mixed-precision lattice path and costs a
    few per cent on this small grid's FP64 point path; the sweep ratio is printed and
    held within 5 %.  A run split over launches takes the same decisions (they depend on
    absolute time only)."""
    net = pgsynth.config1(nx=40, ny=30)
    h, S = net.meta["h"], 300
    err2, st2 = check_against_oracle(B, net, h, S, precision, warm_start=2)
    _, st1 = check_against_oracle(B, net, h, S, precision, warm_start=1)
    print(f"sweeps: warm_start 1 {st1.total_sweeps}, warm_start 2 {st2.total_sweeps} "
          f"(ratio {st2.total_sweeps / st1.total_sweeps:.4f})")
    assert st2.total_sweeps <= 1.05 * st1.total_sweeps
    with B.Grid(net, precision=precision, warm_start=2) as g:
        B.pg_set_stream(g.handle, torch.cuda.current_stream().cuda_stream)
        one = torch.empty(S, dtype=torch.float64, device="cuda")
        B.pg_transient(g.handle, h, S, vmin=one)
        B.pg_reset(g.handle)
        parts = []
        for a in range(0, S, 70):
            k = min(70, S - a)
            v = torch.empty(k, dtype=torch.float64, device="cuda")
            B.pg_transient(g.handle, h, k, vmin=v)
            parts.append(v)
        torch.cuda.synchronize()
        assert torch.equal(torch.cat(parts), one)


def test_full_step_start_after_many_outer_passes(B):
    """The incremental step start carries the previous step's final residual, whose rounding
    drift grows with every outer pass; a step that needed more than four passes is followed
    by a full recompute.  Weak inner solves (inner_reduction 0.5) force such steps: the run
    still matches the oracle, and a run split over launches (which carries the pass count)
    repeats the single launch bit for bit."""
    net = pgsynth.config1(nx=43, ny=39)
    h, S = net.meta["h"], 80
    _, st = check_against_oracle(B, net, h, S, 1, inner_reduction=0.5)
    assert st.max_outer_step > 4, st.max_outer_step
    with B.Grid(net, precision=1, inner_reduction=0.5) as g:
        B.pg_set_stream(g.handle, torch.cuda.current_stream().cuda_stream)
        one = torch.empty(S, dtype=torch.float64, device="cuda")
        B.pg_transient(g.handle, h, S, vmin=one)
        B.pg_reset(g.handle)
        parts = []
        for a in range(0, S, 9):
            k = min(9, S - a)
            v = torch.empty(k, dtype=torch.float64, device="cuda")
            B.pg_transient(g.handle, h, k, vmin=v)
            parts.append(v)
        torch.cuda.synchronize()
        assert torch.equal(torch.cat(parts), one)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("recipe", ["config0_37x29", "config1_33x27x3", "config2_24x19x2"])
def test_four_colour_order(B, recipe, precision):
    """PG_COLOUR_FOUR sweeps the neighbour-list path in four colours ((x + l) mod 2 +
    2 (y mod 2)), a Gauss-Seidel order other than red-black (Section IV-A leaves the order
    open; Theorem 1 covers any order).  The fixed point is the same: parity with the oracle
    holds on odd-sided RC, 3-layer and RLC recipes, and the grid reports four colours."""
    net = {"config0_37x29": lambda: pgsynth.config0(nx=37, ny=29),
           "config1_33x27x3": lambda: pgsynth.config1(nx=33, ny=27),
           "config2_24x19x2": lambda: pgsynth.config2(nx=24, ny=19)}[recipe]()
    with B.Grid(net, precision=precision, colouring=B.PG_COLOUR_FOUR, lattice_sweeps=-1) as g:
        assert g.info["n_colours"] == 4
    _, st4 = check_against_oracle(B, net, net.meta["h"], 40, precision, colouring=B.PG_COLOUR_FOUR,
                                  lattice_sweeps=-1)
    _, st2 = check_against_oracle(B, net, net.meta["h"], 40, precision, lattice_sweeps=-1)
    print(f"{recipe} precision {precision}: sweeps four-colour {st4.total_sweeps}, red-black {st2.total_sweeps}")


@pytest.mark.parametrize("recipe,k", [("config1_97x141x3", 3), ("config2_70x75x2", 2), ("config0_83x150", 3)])
def test_tall_lattice_regions(B, recipe, k):
    """tile_rows = 66: the lattice inner solve on 34-column by 66-row regions (one block per
    SM for 2-3 layers).  The same iteration as 34-row regions (the host replay shows the
    interior equals k global block sweeps for both), so parity with the oracle holds on
    ragged 3-layer, RLC and single-layer recipes."""
    net = {"config1_97x141x3": lambda: pgsynth.config1(nx=97, ny=141),
           "config2_70x75x2": lambda: pgsynth.config2(nx=70, ny=75),
           "config0_83x150": lambda: pgsynth.config0(nx=83, ny=150)}[recipe]()
    _, st = check_against_oracle(B, net, net.meta["h"], 30, 1, tile_rows=66, lattice_sweeps=k)
    assert st.lattice_sweeps == k
    _, st34 = check_against_oracle(B, net, net.meta["h"], 30, 1, tile_rows=34, lattice_sweeps=k)
    print(f"{recipe}: sweeps 66-row {st.total_sweeps} ({st.device_ms:.2f} ms), 34-row {st34.total_sweeps} "
          f"({st34.device_ms:.2f} ms)")


def test_tall_regions_on_a_batch(B):
    """A batch of uneven lattices (1-2 layers, odd offsets: 4-byte staging for most) on
    66-row regions: every grid of the batch against its own oracle solve."""
    net = pgsynth.config3(n_grids=6, side_lo=20, side_hi=90)
    parts = pgsynth.config3_parts(n_grids=6, side_lo=20, side_hi=90)
    h, S = net.meta["h"], 25
    V, _, _, _, st = run_gpu(B, net, h, S, 1, tile_rows=66)
    assert st.failed_step == -1 and st.lattice_sweeps > 0
    for off, part in parts:
        Vo, _ = transient.transient(part, h, S)
        err = np.max(np.abs(V[:, off:off + part.n_nodes] - Vo[1:]))
        assert err <= TOL_V, f"grid at {off} {part.lattice}: {err:.3e} V"
