"""Parity at the full sizes of the workloads, in the launch configuration the
benchmark uses (one persistent launch per transient, mixed precision for the
RC grids).

* RC 1024x1024x3, 1000 steps: too large for the oracle's direct solver, so the
  oracle certifies the GPU trajectory instead.  For every step it evaluates,
  from its own incidence-matrix assembly and PWL evaluation, the FP64 residual
  of the backward-Euler equation (Eq. 2) at the GPU's voltages.  With the
  stored, verified upper bounds of ``kappa = ||M^-1 D||`` and of the
  accumulation gain ``1 + ||G^-1 (C/h) 1||`` (tests/golden/fullsize_bounds.json,
  written by make_fullsize_bounds.py from the oracle alone) this bounds the
  distance of every step to the exact BE trajectory; the bound must be below
  1e-6 V.  The chunked run used for the check must equal the single
  1000-step launch the benchmark times, bit for bit.
* RLC 512x512x2: element-by-element against the oracle's direct solves, every
  node and inductor current of all 2000 steps, in lockstep chunks.
* 256 batched grids: every grid is an independent sub-circuit (Fig. 1), so the
  oracle solves sampled grids exactly on their own and compares every node of
  them, every step of all 500 (read through the probe output): the largest
  single-layer and two-layer grids and three small ones.  The batch's
  accumulated certified bound is asserted too.
* RC 2048x2048, 500 steps (the adjoint workload): the forward trajectory is
  certified like the 1024x1024x3 one; the gradients of pg_adjoint (no
  counterpart in the paper) are checked at full size by properties that hold at
  any size: an exact scaling identity over all parameters, a tangent-linear
  (forward-mode) dot-product test along a capacitor direction, a central
  difference along a random resistor direction, bit-identical checkpoint replay;
  and one parameter at a time, 50 random resistors and 50 random capacitors,
  against central differences of the exact recurrence around the GPU's
  trajectory (windowed direct solves on the host), each within 1e-4.
"""
import json
import os

import numpy as np
import pytest

import pgsynth
from oracle import matrices, pwl, transient

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_V = 1e-6
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fullsize_bounds.json")


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1409_7166_gb300 import binding
    return binding


def _certify_rc(B, net, bounds, chunk=50):
    """Certified max error of the GPU trajectory (mixed precision) over all steps."""
    h, nsteps = net.meta["h"], net.meta["nsteps"]
    mats = matrices.nodal_matrices(net)
    M = mats.system_matrix(h).tocsr()
    Mdiag = M.diagonal()
    Ch = mats.C.diagonal() / h
    src = -(mats.G_s @ mats.vd)
    absrow = abs(M) @ np.ones(net.n_nodes)
    eps = 2.0 ** -52
    with B.Grid(net, precision=B.PG_PREC_MIXED) as g:
        B.pg_set_stream(g.handle, torch.cuda.current_stream().cuda_stream)
        # reference: the benchmark's launch, 1000 steps at once, worst-drop waveform only
        vmin_one = torch.empty(nsteps, dtype=torch.float64, device="cuda")
        B.pg_transient(g.handle, h, nsteps, vmin=vmin_one)
        vmin_one = vmin_one.cpu().numpy()
        B.pg_reset(g.handle)
        B.pg_transient(g.handle, h, 0)                 # DC point (step 0)
        v_prev = np.zeros(net.n_nodes)
        assert B.pg_get_state(g.handle, v_prev) == 0
        # step 0 is the exact DC point: zero load at t = 0 and one supply level
        r0 = -(mats.G @ v_prev) + src - mats.A_i.T @ pwl.pwl_values(net.i_ptr, net.i_t, net.i_v, 0.0)
        assert np.all(v_prev == 1.0) and np.max(np.abs(r0)) < 1e-12
        V = torch.empty((chunk, net.n_nodes), dtype=torch.float64, device="cuda")
        vmin = torch.empty(chunk, dtype=torch.float64, device="cuda")
        worst_step, s = 0.0, 0
        vmin_chunks = []
        while s < nsteps:
            k = min(chunk, nsteps - s)
            B.pg_transient(g.handle, h, k, v_all=V[:k], vmin=vmin[:k])
            Vh = V[:k].cpu().numpy()
            vmin_chunks.append(vmin[:k].cpu().numpy())
            for j in range(k):
                t = (s + j + 1) * h
                b = Ch * v_prev + src - mats.A_i.T @ pwl.pwl_values(net.i_ptr, net.i_t, net.i_v, t)
                r = b - M @ Vh[j]
                R = np.max(np.abs(r) / Mdiag)
                # rounding of this FP64 residual evaluation (at most 16 terms per row)
                R += 2 * 16 * eps * np.max((absrow * np.abs(Vh[j]) + np.abs(b)) / Mdiag)
                worst_step = max(worst_step, bounds["kappa_upper"] * R)
                v_prev = Vh[j]
            s += k
    # the chunked run repeats the single launch exactly (same iteration, same state)
    assert np.array_equal(np.concatenate(vmin_chunks), vmin_one)
    return bounds["gain_upper"] * worst_step, worst_step


@pytest.mark.skipif(not os.path.exists(GOLDEN), reason="run tests/golden/make_fullsize_bounds.py")
def test_config1_full_size_certified(B):
    net = pgsynth.config1()
    with open(GOLDEN) as f:
        bounds = json.load(f)["config1"]
    err, per_step = _certify_rc(B, net, bounds)
    print(f"config 1: per-step bound {per_step:.3e} V, accumulated bound {err:.3e} V")
    assert err <= TOL_V


def test_config2_full_size_rlc(B):
    """All 2000 steps of the RLC grid, every node and every inductor current, against the
    oracle's direct solves (explicit inductor currents, Eq. 10) in lockstep chunks of 100
    steps, so no more than one chunk of either waveform is held.  The loads switch until
    about step 530 (t0 up to 1 ns, edges up to 30 + 30 ps at 2 ps per step) and the LC
    ringing runs after that; both are compared.  RLC grids carry no accumulated
    certificate, so this is their full-size parity proof.  The chunked run must repeat a
    single 2000-step launch (the launch the benchmark times) bit for bit."""
    net = pgsynth.config2()
    h, S, chunk = net.meta["h"], net.meta["nsteps"], 100
    sim = transient.simulate(net, h, S)
    next(sim)                                          # the DC point (step 0)
    worst_v = worst_il = il_max = 0.0
    with B.Grid(net, precision=B.PG_PREC_FP64) as g:
        B.pg_set_stream(g.handle, torch.cuda.current_stream().cuda_stream)
        vmin_one = torch.empty(S, dtype=torch.float64, device="cuda")
        st = B.pg_transient(g.handle, h, S, vmin=vmin_one)
        assert st.failed_step == -1 and st.steps_done == S
        vmin_one = vmin_one.cpu().numpy()
        B.pg_reset(g.handle)
        V = torch.empty((chunk, net.n_nodes), dtype=torch.float64, device="cuda")
        IL = torch.empty((chunk, len(net.l_val)), dtype=torch.float64, device="cuda")
        vmin = torch.empty(chunk, dtype=torch.float64, device="cuda")
        parts, s = [], 0
        while s < S:
            k = min(chunk, S - s)
            st = B.pg_transient(g.handle, h, k, v_all=V[:k], il_all=IL[:k], vmin=vmin[:k])
            assert st.failed_step == -1 and st.steps_done == k
            Vh, ILh = V[:k].cpu().numpy(), IL[:k].cpu().numpy()
            parts.append(vmin[:k].cpu().numpy())
            for j in range(k):
                step, vo, ilo = next(sim)
                assert step == s + j + 1
                worst_v = max(worst_v, float(np.max(np.abs(Vh[j] - vo))))
                worst_il = max(worst_il, float(np.max(np.abs(ILh[j] - ilo))))
                il_max = max(il_max, float(np.max(np.abs(ilo))))
            s += k
    print(f"config 2, {S} steps: max |v - v_oracle| {worst_v:.3e} V, max |i_l - i_l,oracle| {worst_il:.3e} A "
          f"(max |i_l| {il_max:.3e} A)")
    assert worst_v <= TOL_V, f"max |v - v_oracle| = {worst_v:.3e} V"
    assert worst_il <= 1e-3 * il_max, f"inductor current error {worst_il:.3e} A"
    assert np.array_equal(np.concatenate(parts), vmin_one)


def test_config3_full_size_sampled_grids(B):
    """The 256-grid batch in one 500-step launch.  Compared node by node, every step, with
    the oracle's direct solve of each grid on its own (the grids are independent
    sub-circuits, Fig. 1): the batch's largest single-layer and largest two-layer grids,
    which converge slowest and leave the inner solve last, and three small grids drawn at
    random.  The batch's accumulated certified bound must meet the 0.9 tol the per-step
    target is set for."""
    net = pgsynth.config3()
    parts = pgsynth.config3_parts()
    h, nsteps = net.meta["h"], net.meta["nsteps"]
    rng = np.random.default_rng(33)
    small = [k for k, (_, p) in enumerate(parts) if p.n_nodes <= 40000]
    pick = set(rng.choice(small, size=3, replace=False).tolist())
    for nl in (1, 2):
        same = [k for k, (_, p) in enumerate(parts) if p.lattice[2] == nl]
        pick.add(max(same, key=lambda k: parts[k][1].n_nodes))
    pick = sorted(pick)
    probes = np.concatenate([np.arange(parts[k][0], parts[k][0] + parts[k][1].n_nodes) for k in pick])
    with B.Grid(net, precision=B.PG_PREC_MIXED) as g:
        B.pg_set_stream(g.handle, torch.cuda.current_stream().cuda_stream)
        pr = torch.tensor(probes, dtype=torch.int32, device="cuda")
        PV = torch.empty((nsteps, probes.size), dtype=torch.float64, device="cuda")
        st = B.pg_transient(g.handle, h, nsteps, probes=pr, probe_v=PV)
        PV = PV.cpu().numpy()
    assert st.failed_step == -1 and st.steps_done == nsteps
    print(f"config 3: accumulated bound {st.err_bound:.3e} V over {nsteps} steps")
    assert st.err_bound <= 0.9 * TOL_V * (1 + 1e-9)
    col = 0
    for k in pick:
        off, part = parts[k]
        Vo, _ = transient.transient(part, h, nsteps)
        got = PV[:, col:col + part.n_nodes]
        col += part.n_nodes
        err = float(np.max(np.abs(got - Vo[1:])))
        print(f"  grid {k} {part.lattice}: max error {err:.3e} V")
        assert err <= TOL_V, f"grid {k} ({part.lattice}): max error {err:.3e} V"


@pytest.mark.skipif(not os.path.exists(GOLDEN), reason="run tests/golden/make_fullsize_bounds.py")
def test_config4_full_size_certified(B):
    net = pgsynth.config4()
    with open(GOLDEN) as f:
        bounds = json.load(f)["config4"]
    err, per_step = _certify_rc(B, net, bounds)
    print(f"config 4: per-step bound {per_step:.3e} V, accumulated bound {err:.3e} V")
    assert err <= TOL_V


def _dJ_dv(V, vref, margin):
    u = vref - V - margin
    return -2.0 * torch.nn.functional.softplus(u, threshold=1e9) * torch.sigmoid(u)


def test_config4_full_size_adjoint(B):
    """Gradients of J = sum_s sum_i softplus(1 - v - 0.05)^2 over 500 steps of
    the 2048x2048 grid (checkpoints every 50 steps).

    * Scaling identity: multiplying every conductance and capacitance by a
      leaves M v = b invariant up to v - Vdd -> (v - Vdd)/a (the supply is the
      only source and the DC point is v = Vdd), so
      sum_e g_e dJ/dg_e + sum_k C_k dJ/dC_k = sum_{s,i} 2 sp(u) sig(u) (v - Vdd)
      exactly; both sides in FP64, equal to 1e-9 relative.
    * Tangent linear model along dC = K C w (w = 1 on the left half): with
      M dv_s = (C/h) dv_{s-1} - (dC/h)(v_s - v_{s-1}), dv_0 = 0, the directional
      derivative is sum_{s,i} dJ/dv_{s,i} dv_{s,i}.  Each solve is certified to
      tol_s; T = M^-1 C/h >= 0 carries the errors, so
      |error| <= kacc tol_s sum|dJ/dv|, the test's bound.
    * Central difference along a random-sign relative perturbation of every
      resistor (eps = 1e-3, per-term differences of J): relative 1e-4.
    """
    net = pgsynth.config4()
    h, S, n = net.meta["h"], net.meta["nsteps"], net.n_nodes
    vref, margin, vdd = 1.0, 0.05, float(net.vdd[0])
    dev = "cuda"
    with B.Grid(net, precision=B.PG_PREC_MIXED, tol=1e-9) as g:
        B.pg_set_stream(g.handle, torch.cuda.current_stream().cuda_stream)
        gG = torch.zeros(len(net.r_g), dtype=torch.float64, device=dev)
        gC = torch.zeros(len(net.c_val), dtype=torch.float64, device=dev)
        J, st = B.pg_adjoint(g.handle, h, S, vref=vref, margin=margin, ckpt_every=50, dJ_dG=gG, dJ_dC=gC)
        # the backward pass replays segments from checkpoints: their spacing changes nothing
        gG2, gC2 = torch.zeros_like(gG), torch.zeros_like(gC)
        J2, _ = B.pg_adjoint(g.handle, h, S, vref=vref, margin=margin, ckpt_every=125, dJ_dG=gG2, dJ_dC=gC2)
        assert J2 == J and torch.equal(gG, gG2) and torch.equal(gC, gC2)
        del gG2, gC2

        B.pg_reset(g.handle)
        V = torch.empty((S, n), dtype=torch.float64, device=dev)
        fst = B.pg_transient(g.handle, h, S, v_all=V)
        chunks = range(0, S, 25)
        Jv = sum(float((torch.nn.functional.softplus(vref - V[a:a + 25] - margin, threshold=1e9) ** 2).sum())
                 for a in chunks)
        assert Jv == pytest.approx(J, rel=1e-12)

        r_g = torch.tensor(net.r_g, device=dev)
        c_val = torch.tensor(net.c_val, device=dev)
        lhs = float((r_g * gG).sum()) + float((c_val * gC).sum())
        rhs = sum(float((-_dJ_dv(V[a:a + 25], vref, margin) * (V[a:a + 25] - vdd)).sum()) for a in chunks)
        assert lhs == pytest.approx(rhs, rel=1e-9), (lhs, rhs)

        # tangent linear model along a capacitor direction
        cnode = np.where(net.c_a >= 0, net.c_a, net.c_b)
        xs = (cnode % 2048) < 1024                       # left half of the grid
        K = 1e4
        dc = np.where(xs, K * net.c_val, 0.0)
        Ch = torch.tensor(np.bincount(cnode, net.c_val / h, minlength=n), device=dev)
        dCh = torch.tensor(np.bincount(cnode, dc / h, minlength=n), device=dev)
        tol_s = 1e-10
        dv = torch.zeros(n, dtype=torch.float64, device=dev)
        nxt = torch.empty_like(dv)
        v_prev = torch.full((n,), vdd, dtype=torch.float64, device=dev)   # DC point v_0 = Vdd
        tl, absw = 0.0, 0.0
        for s_ in range(S):
            b = Ch * dv - dCh * (V[s_] - v_prev)
            B.pg_solve(g.handle, h, b, nxt, tol_s)
            w = _dJ_dv(V[s_], vref, margin)
            tl += float((w * nxt).sum())
            absw += float(w.abs().sum())
            dv, nxt = nxt, dv
            v_prev = V[s_]
        ad = float((torch.tensor(dc, device=dev) * gC).sum())
        bound = st.kacc * tol_s * absw
        print(f"tangent linear {tl:.12e} adjoint {ad:.12e} bound {bound:.2e}")
        assert abs(tl - ad) <= bound + 1e-9 * abs(ad)
        del V, dv, nxt, v_prev

        # central difference along a random resistor direction, per-term J differences
        rng = np.random.default_rng(44)
        sgn = rng.choice([-1.0, 1.0], size=len(net.r_g))
        eps = 1e-3
        Vp = torch.empty((S, n), dtype=torch.float64, device=dev)
        Vm = torch.empty_like(Vp)
        for sign, Vx in ((1.0, Vp), (-1.0, Vm)):
            B.pg_update_values(g.handle, r_g=net.r_g * (1.0 + sign * eps * sgn))
            B.pg_reset(g.handle)
            B.pg_transient(g.handle, h, S, v_all=Vx)
        dJ = 0.0
        for a in chunks:
            sp_p = torch.nn.functional.softplus(vref - Vp[a:a + 25] - margin, threshold=1e9)
            sp_m = torch.nn.functional.softplus(vref - Vm[a:a + 25] - margin, threshold=1e9)
            dJ += float(((sp_p - sp_m) * (sp_p + sp_m)).sum())
        fd = dJ / (2.0 * eps)
        ad = float((torch.tensor(sgn * net.r_g, device=dev) * gG).sum())
        print(f"central difference {fd:.12e} adjoint {ad:.12e}")
        assert fd == pytest.approx(ad, rel=1e-4)


def test_config4_full_size_per_parameter_gradients(B):
    """dJ/dg of 50 random resistors and dJ/dC of 50 random capacitors of the 2048x2048 grid
    over all 500 steps, one parameter at a time, against central differences (eps = 1e-3
    of the parameter), each within 1e-4 relative.

    Central differences of the GPU transient itself cannot resolve one parameter: a 0.1 %
    change of one of 8.4M resistors moves J (about 1e9) by some 1e-7, below what the
    iterative solves' stopping decisions and rounding leave in a difference of two
    4.2M-node, 500-step runs.  So the differences are taken of the exact backward-Euler
    recurrence around the GPU's trajectory: the change dv of the trajectory solves
    (M + dM) dv_s = ((C + dC)/h) dv_(s-1) - dM v_s + (dC/h) v_(s-1) with direct solves on a
    257 x 257 box around the parameter (the pads confine its influence), and J's change is
    formed per term without cancellation (window_fd.py; pinned against the oracle's exact
    adjoint, with the box's truncation measured below 1e-6, in test_window_fd_host.py).
    The per-parameter solves run in a pool of host processes."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import window_fd

    net = pgsynth.config4()
    h, S, n = net.meta["h"], net.meta["nsteps"], net.n_nodes
    vref, margin, vdd = 1.0, 0.05, float(net.vdd[0])
    rel_eps, R, tol_rel = 1e-3, 128, 1e-4
    rng = np.random.default_rng(100)
    seg = np.where((net.r_a >= 0) & (net.r_b >= 0))[0]
    cnode = np.where(net.c_a >= 0, net.c_a, net.c_b)
    params = [("r", int(e), (int(net.r_a[e]), int(net.r_b[e])), float(net.r_g[e]))
              for e in rng.choice(seg, size=50, replace=False)]
    params += [("c", int(k), (int(cnode[k]),), float(net.c_val[k]))
               for k in rng.choice(len(net.c_val), size=50, replace=False)]
    mats = matrices.nodal_matrices(net)
    M = mats.system_matrix(h).tocsr()
    ch = mats.C.diagonal() / h
    dev = "cuda"
    with B.Grid(net, precision=B.PG_PREC_MIXED, tol=1e-9) as g:
        B.pg_set_stream(g.handle, torch.cuda.current_stream().cuda_stream)
        gG = torch.zeros(len(net.r_g), dtype=torch.float64, device=dev)
        gC = torch.zeros(len(net.c_val), dtype=torch.float64, device=dev)
        B.pg_adjoint(g.handle, h, S, vref=vref, margin=margin, ckpt_every=50, dJ_dG=gG, dJ_dC=gC)
        gG, gC = gG.cpu().numpy(), gC.cpu().numpy()
        B.pg_reset(g.handle)
        V = torch.empty((S, n), dtype=torch.float64, device=dev)
        B.pg_transient(g.handle, h, S, v_all=V)
        torch.cuda.synchronize()

        workers = max(1, min(16, len(os.sched_getaffinity(0))))
        worst = {"r": 0.0, "c": 0.0}
        rels = {"r": [], "c": []}
        with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as pool:
            pending = {}

            def drain(limit):
                while len(pending) > limit:
                    done, _ = cf.wait(list(pending), return_when=cf.FIRST_COMPLETED)
                    for f in done:
                        kind, idx, p = pending.pop(f)
                        fd = f.result() * p
                        ad = p * (gG[idx] if kind == "r" else gC[idx])
                        rel = abs(fd - ad) / abs(ad)
                        worst[kind] = max(worst[kind], rel)
                        rels[kind].append(rel)
                        assert rel <= tol_rel, (f"{'resistor' if kind == 'r' else 'capacitor'} {idx}: central "
                                                f"difference {fd:.9e}, adjoint {ad:.9e} (p dJ/dp, rel {rel:.2e})")

            for kind, idx, term, p in params:
                win, Mw, chw, loc = window_fd.parameter_window(M, ch, net.lattice, kind, term, R)
                Vw = V[:, torch.from_numpy(win).to(dev)].cpu().numpy()
                f = pool.submit(window_fd.central_difference, Mw, chw, Vw, np.full(len(win), vdd), kind, loc,
                                rel_eps * p, h, vref, margin)
                pending[f] = (kind, idx, p)
                drain(2 * workers)
            drain(0)
        print(f"per-parameter central differences: 50 resistors worst {worst['r']:.2e} (median "
              f"{np.median(rels['r']):.2e}), 50 capacitors worst {worst['c']:.2e} (median {np.median(rels['c']):.2e}) "
              f"relative ({workers} host processes)")
