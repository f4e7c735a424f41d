"""pg_adjoint (discrete adjoint of the BE RC and RLC transient, not in the paper)
against the oracle's exact adjoint, plus pg_update_values and the
torch.autograd.Function wrapper.

Gradient tolerance: |g - g_ref| <= 1e-4 max(|g_ref|, 1e-3 max|g_ref|) (relative
1e-4 with a floor for near-zero entries).  The forward tolerance is tightened
to 1e-9 V here so that the comparison measures the adjoint, not the forward
solver's 1e-6 V budget (a segment gradient multiplies voltage differences of a
few mV).
"""
import numpy as np
import pytest

import pgsynth
from pgsynth import GROUND
from oracle import adjoint as oadj, transient

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1409_7166_gb300 import binding
    return binding


def _close(g, ref, rel=1e-4):
    floor = 1e-3 * np.max(np.abs(ref))
    bad = np.abs(g - ref) > rel * np.maximum(np.abs(ref), floor)
    return int(np.sum(bad)), float(np.max(np.abs(g - ref) / np.maximum(np.abs(ref), floor)))


def _heavy(net, factor=40.0):
    net.i_v = net.i_v * factor          # drops of tens of mV, so the objective has a gradient
    return net


@pytest.mark.parametrize("precision", [0, 1])
def test_adjoint_matches_oracle(B, precision):
    net = _heavy(pgsynth.config0(nx=37, ny=29))
    h, S = net.meta["h"], 80
    J0, dG0, dC0 = oadj.gradients(net, h, S)
    with B.Grid(net, precision=precision, tol=1e-9) as g:
        gG = np.zeros(len(net.r_g)); gC = np.zeros(len(net.c_val))
        J, st = B.pg_adjoint(g.handle, h, S, ckpt_every=25, dJ_dG=gG, dJ_dC=gC)
    assert J == pytest.approx(J0, rel=1e-8)
    nbad, worst = _close(gG, dG0)
    assert nbad == 0, f"dJ/dG: {nbad} entries off, worst {worst:.2e}"
    nbad, worst = _close(gC, dC0)
    assert nbad == 0, f"dJ/dC: {nbad} entries off, worst {worst:.2e}"


def test_adjoint_with_dc_point_term(B):
    """A resistor to ground and loads on at t = 0: the DC point depends on G and
    its adjoint term enters dJ/dG."""
    net = _heavy(pgsynth.config0(nx=15, ny=13))
    extra = np.arange(3, net.n_nodes, 41, dtype=np.int32)
    net.r_a = np.concatenate([net.r_a, extra])
    net.r_b = np.concatenate([net.r_b, np.full(extra.size, GROUND, np.int32)])
    net.r_g = np.concatenate([net.r_g, np.full(extra.size, 0.3)])
    net.i_v = net.i_v.copy(); net.i_v[0::3] = 4e-3
    h, S = net.meta["h"], 30
    J0, dG0, dC0 = oadj.gradients(net, h, S)
    with B.Grid(net, tol=1e-9) as g:
        gG = np.zeros(len(net.r_g)); gC = np.zeros(len(net.c_val))
        J, _ = B.pg_adjoint(g.handle, h, S, ckpt_every=7, dJ_dG=gG, dJ_dC=gC)
    assert J == pytest.approx(J0, rel=1e-8)
    assert _close(gG, dG0)[0] == 0 and _close(gC, dC0)[0] == 0


def test_update_values_equals_new_grid(B):
    net = pgsynth.config0(nx=31, ny=22)
    h = net.meta["h"]
    rng = np.random.default_rng(8)
    r2 = net.r_g * rng.uniform(0.8, 1.25, net.r_g.size)
    c2 = net.c_val * rng.uniform(0.8, 1.25, net.c_val.size)
    net2 = pgsynth.Netlist(**{**net.__dict__, "r_g": r2, "c_val": c2})
    Vo, _ = transient.transient(net2, h, 20)
    with B.Grid(net) as g:
        B.pg_transient(g.handle, h, 5)
        B.pg_update_values(g.handle, r_g=r2, c_val=c2)
        B.pg_reset(g.handle)
        V = np.zeros((20, net.n_nodes))
        B.pg_transient(g.handle, h, 20, v_all=V)
    assert np.max(np.abs(V - Vo[1:])) <= 1e-6


def test_autograd_function(B):
    from paper_1409_7166_gb300.autograd import IRDropObjective
    net = _heavy(pgsynth.config0(nx=21, ny=17))
    h, S = net.meta["h"], 40
    J0, dG0, dC0 = oadj.gradients(net, h, S)
    with B.Grid(net, tol=1e-9) as g:
        r = torch.tensor(net.r_g, device="cuda", requires_grad=True)
        c = torch.tensor(net.c_val, device="cuda", requires_grad=True)
        J = IRDropObjective.apply(g, r, c, h, S)
        (2.0 * J).backward()
    assert float(J.detach()) == pytest.approx(J0, rel=1e-8)
    assert _close(r.grad.cpu().numpy() / 2.0, dG0)[0] == 0
    assert _close(c.grad.cpu().numpy() / 2.0, dC0)[0] == 0


def _inductive_rlc(nx, ny):
    """config-2 recipe with an inductive supply path (pad resistors 0.02 S) and every
    load starting 2 ps in, so that dJ/dL is a sizeable part of the gradient."""
    net = pgsynth.config2(nx=nx, ny=ny)
    net.r_g = net.r_g.copy()
    net.r_g[np.asarray(net.r_b) < -1] = 0.02
    net.i_v = net.i_v.copy() * 20.0
    net.i_t = net.i_t.copy()
    ptr = np.asarray(net.i_ptr)
    for e in range(len(ptr) - 1):
        net.i_t[ptr[e]:ptr[e + 1]] += 2e-12 - net.i_t[ptr[e]]
    return net


@pytest.mark.parametrize("precision", [0, 1])
def test_rlc_adjoint_matches_oracle(B, precision):
    net = _inductive_rlc(19, 15)
    h, S = net.meta["h"], 60
    J0, dG0, dC0, dL0 = oadj.gradients(net, h, S, with_l=True)
    # default tol: the per-step target of a grid with inductors is 1e-4 tol, which with this
    # grid's kappa (about 630) is close to what FP64 residuals can certify
    with B.Grid(net, precision=precision) as g:
        gG = np.zeros(len(net.r_g)); gC = np.zeros(len(net.c_val)); gL = np.zeros(len(net.l_val))
        J, st = B.pg_adjoint(g.handle, h, S, ckpt_every=17, dJ_dG=gG, dJ_dC=gC, dJ_dL=gL)
    assert J == pytest.approx(J0, rel=1e-8)
    for name, got, ref in (("dJ/dG", gG, dG0), ("dJ/dC", gC, dC0), ("dJ/dL", gL, dL0)):
        nbad, worst = _close(got, ref)
        assert nbad == 0, f"{name}: {nbad} entries off, worst {worst:.2e}"


def test_autograd_function_rlc(B):
    from paper_1409_7166_gb300.autograd import IRDropObjective
    net = _inductive_rlc(13, 11)
    h, S = net.meta["h"], 40
    J0, dG0, dC0, dL0 = oadj.gradients(net, h, S, with_l=True)
    with B.Grid(net) as g:
        r = torch.tensor(net.r_g, device="cuda", requires_grad=True)
        c = torch.tensor(net.c_val, device="cuda", requires_grad=True)
        lv = torch.tensor(net.l_val, device="cuda", requires_grad=True)
        J = IRDropObjective.apply(g, r, c, h, S, 1.0, 0.05, 50, lv)
        J.backward()
    assert float(J.detach()) == pytest.approx(J0, rel=1e-8)
    assert _close(r.grad.cpu().numpy(), dG0)[0] == 0
    assert _close(c.grad.cpu().numpy(), dC0)[0] == 0
    assert _close(lv.grad.cpu().numpy(), dL0)[0] == 0
