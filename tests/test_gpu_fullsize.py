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
* RLC 512x512x2: element-by-element against the oracle's direct solves for the
  first 400 steps (the loads' active window), then the remaining steps must
  run without a failure.
* 256 batched grids: every grid is an independent sub-circuit (Fig. 1), so the
  oracle solves sampled grids exactly on their own and compares every node of
  them, every step (read through the probe output).
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
    net = pgsynth.config2()
    h, n_check = net.meta["h"], 400
    Vo, ILo = transient.transient(net, h, n_check)
    with B.Grid(net, precision=B.PG_PREC_FP64) as g:
        B.pg_set_stream(g.handle, torch.cuda.current_stream().cuda_stream)
        V = torch.empty((n_check, net.n_nodes), dtype=torch.float64, device="cuda")
        IL = torch.empty((n_check, len(net.l_val)), dtype=torch.float64, device="cuda")
        B.pg_transient(g.handle, h, n_check, v_all=V, il_all=IL)
        err = float(np.max(np.abs(V.cpu().numpy() - Vo[1:])))
        il_err = float(np.max(np.abs(IL.cpu().numpy() - ILo[1:])))
        assert err <= TOL_V, f"max |v - v_oracle| = {err:.3e} V"
        assert il_err <= 1e-3 * np.max(np.abs(ILo)), f"inductor current error {il_err:.3e} A"
        st = B.pg_transient(g.handle, h, net.meta["nsteps"] - n_check)
        assert st.failed_step == -1 and st.steps_done == net.meta["nsteps"] - n_check


def test_config3_full_size_sampled_grids(B):
    net = pgsynth.config3()
    parts = pgsynth.config3_parts()
    h, nsteps = net.meta["h"], 120
    rng = np.random.default_rng(33)
    small = [k for k, (_, p) in enumerate(parts) if p.n_nodes <= 40000]
    pick = sorted(rng.choice(small, size=3, replace=False).tolist())
    probes = np.concatenate([np.arange(parts[k][0], parts[k][0] + parts[k][1].n_nodes) for k in pick])
    with B.Grid(net, precision=B.PG_PREC_MIXED) as g:
        B.pg_set_stream(g.handle, torch.cuda.current_stream().cuda_stream)
        pr = torch.tensor(probes, dtype=torch.int32, device="cuda")
        PV = torch.empty((nsteps, probes.size), dtype=torch.float64, device="cuda")
        st = B.pg_transient(g.handle, h, nsteps, probes=pr, probe_v=PV)
        PV = PV.cpu().numpy()
    assert st.failed_step == -1
    col = 0
    for k in pick:
        off, part = parts[k]
        Vo, _ = transient.transient(part, h, nsteps)
        got = PV[:, col:col + part.n_nodes]
        col += part.n_nodes
        err = float(np.max(np.abs(got - Vo[1:])))
        assert err <= TOL_V, f"grid {k} ({part.lattice}): max error {err:.3e} V"
