"""Seeded synthetic power-grid netlists.

This module only draws inputs: element lists, terminals and piecewise-linear
(PWL) load-current breakpoints.  It holds none of the analysis arithmetic
(no matrix assembly, no PWL evaluation, no solve), so that the CPU oracle and
the CUDA path can both consume the same netlist without sharing any of the
method's code.

Netlist model (Section III of the paper, Eq. 4-6)
-------------------------------------------------
* ``n_nodes`` trivial nodes, numbered ``0 .. n_nodes-1``.
* ``p = len(vdd)`` source nodes: positive terminals of ideal voltage sources
  whose negative terminal is ground (topological assumption 1).
* A branch terminal is an ``int32``: ``t >= 0`` is a trivial node, ``-1`` is
  ground, and ``-2-k`` is source node ``k``.  Splitting terminals this way is
  the paper's split of the incidence matrix into the modified incidence ``A``
  (trivial nodes, Eq. 4) and the source incidence ``A_s`` (Eq. 5).
* Branch groups follow Eq. 6: resistors (conductance ``r_g`` in S),
  capacitors (``c_val`` in F), inductors (``l_val`` in H) and current
  sources.  Every branch is oriented ``a -> b`` (``a`` is the branch source
  with incidence +1, ``b`` the sink with -1).
* A current source drives its PWL current from ``a`` to ``b`` through the
  source, so a load that draws ``I(t)`` from node ``k`` is ``a = k,
  b = ground``.  Breakpoints are stored CSR-style: source ``e`` owns
  ``i_t[i_ptr[e]:i_ptr[e+1]]`` / ``i_v[...]``.
* ``lattice = (nx, ny, nl)`` is an optional structural hint: node
  ``(x, y, l)`` has id ``(l*ny + y)*nx + x``.  Nothing depends on it for
  correctness.

Workload recipes
----------------
``config0`` .. ``config4`` are the five seeded workloads of the build
(RC 100x100 mesh, RC 1024x1024x3, RLC 512x512x2, 256 batched RC grids, RC
2048x2048 for the adjoint).  Each takes ``seed`` and optional reduced sizes
so tests can draw the same recipe at a size the oracle finishes in seconds.
Units are SI throughout.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional, Tuple

import numpy as np

GROUND = -1


def source_terminal(k: int) -> int:
    """Terminal code of source node ``k``."""
    return -2 - int(k)


@dataclass
class Netlist:
    n_nodes: int
    vdd: np.ndarray
    r_a: np.ndarray
    r_b: np.ndarray
    r_g: np.ndarray
    c_a: np.ndarray
    c_b: np.ndarray
    c_val: np.ndarray
    l_a: np.ndarray
    l_b: np.ndarray
    l_val: np.ndarray
    i_a: np.ndarray
    i_b: np.ndarray
    i_ptr: np.ndarray
    i_t: np.ndarray
    i_v: np.ndarray
    lattice: Optional[Tuple[int, int, int]] = None
    name: str = ""
    # independent lattices side by side: (first node id, nx, ny, nl) each
    lattices: Optional[list] = None
    meta: dict = field(default_factory=dict)

    @property
    def n_sources(self) -> int:
        return int(self.vdd.shape[0])

    def counts(self) -> dict:
        return dict(n=self.n_nodes, p=self.n_sources, R=len(self.r_g),
                    C=len(self.c_val), L=len(self.l_val), I=len(self.i_a))

    def nbytes(self) -> int:
        return sum(getattr(self, k).nbytes for k in (
            "vdd", "r_a", "r_b", "r_g", "c_a", "c_b", "c_val", "l_a", "l_b",
            "l_val", "i_a", "i_b", "i_ptr", "i_t", "i_v"))


def _i32(x):
    return np.ascontiguousarray(x, dtype=np.int32)


def _f64(x):
    return np.ascontiguousarray(x, dtype=np.float64)


def make_netlist(n_nodes, vdd, R=(), C=(), L=(), I=(), lattice=None, name=""):
    """Build a :class:`Netlist` from small Python lists (tests, hand circuits).

    ``R``/``C``/``L``: iterables of ``(a, b, value)``.  ``I``: iterables of
    ``(a, b, t_points, i_points)``.
    """
    R = list(R); C = list(C); L = list(L); I = list(I)
    ptr = [0]
    ts, vs = [], []
    for (_, _, t, v) in I:
        assert len(t) == len(v) and len(t) >= 1
        ts.extend(t); vs.extend(v); ptr.append(len(ts))
    return Netlist(
        n_nodes=int(n_nodes), vdd=_f64(np.atleast_1d(np.asarray(vdd, dtype=np.float64))),
        r_a=_i32([e[0] for e in R]), r_b=_i32([e[1] for e in R]), r_g=_f64([e[2] for e in R]),
        c_a=_i32([e[0] for e in C]), c_b=_i32([e[1] for e in C]), c_val=_f64([e[2] for e in C]),
        l_a=_i32([e[0] for e in L]), l_b=_i32([e[1] for e in L]), l_val=_f64([e[2] for e in L]),
        i_a=_i32([e[0] for e in I]), i_b=_i32([e[1] for e in I]),
        i_ptr=np.asarray(ptr, dtype=np.int64), i_t=_f64(ts), i_v=_f64(vs),
        lattice=lattice, name=name)


# ---------------------------------------------------------------------------
# lattice recipe
# ---------------------------------------------------------------------------

@dataclass
class LatticeSpec:
    nx: int
    ny: int
    nl: int
    g_layer: tuple            # ("uniform", lo, hi) | ("lognormal", mu, sigma)
    g_via: tuple = ("uniform", 5.0, 20.0)
    l_via: Optional[tuple] = None      # inductance of via (in parallel with the via R)
    pad_layer: int = -1                # -1 = top layer
    pad_pitch: int = 10
    g0: float = 10.0
    l_pad: Optional[tuple] = None      # inductance of pad (in parallel with G0)
    vdd: float = 1.0
    cap_layers: Tuple[int, ...] = (0,)
    cap: tuple = ("uniform", 10e-15, 100e-15)
    load_layer: int = 0
    load_frac: float = 0.2
    ipk: tuple = ("uniform", 0.0, 1e-3)
    tr: tuple = ("uniform", 20e-12, 100e-12)
    tf: tuple = ("uniform", 20e-12, 100e-12)
    t0: tuple = ("uniform", 0.0, 1e-9)


def _draw(rng, dist, size):
    kind = dist[0]
    if kind == "uniform":
        return rng.uniform(dist[1], dist[2], size)
    if kind == "lognormal":
        return rng.lognormal(dist[1], dist[2], size)
    raise ValueError(f"unknown distribution {dist!r}")


def lattice_netlist(spec: LatticeSpec, rng: np.random.Generator, node_offset: int = 0,
                    source_index: int = 0, name: str = "") -> Netlist:
    """Draw one multi-layer lattice grid.

    Draw order (fixed, so a seed names one netlist): per layer x-segments,
    per layer y-segments, vias, via inductors, pad inductors, caps, load
    node choice, then per load Ipk, tr, tf, t0.
    """
    nx, ny, nl = spec.nx, spec.ny, spec.nl
    npl = nx * ny
    n = npl * nl
    ids = np.arange(n, dtype=np.int64).reshape(nl, ny, nx) + node_offset

    ra, rb, rg = [], [], []
    for l in range(nl):
        a = ids[l, :, :-1].ravel(); b = ids[l, :, 1:].ravel()
        ra.append(a); rb.append(b); rg.append(_draw(rng, spec.g_layer, a.size))
    for l in range(nl):
        a = ids[l, :-1, :].ravel(); b = ids[l, 1:, :].ravel()
        ra.append(a); rb.append(b); rg.append(_draw(rng, spec.g_layer, a.size))
    la, lb, lv = [], [], []
    if nl > 1:
        a = ids[:-1].ravel(); b = ids[1:].ravel()
        ra.append(a); rb.append(b); rg.append(_draw(rng, spec.g_via, a.size))
        if spec.l_via is not None:
            la.append(a); lb.append(b); lv.append(_draw(rng, spec.l_via, a.size))
    pl = spec.pad_layer if spec.pad_layer >= 0 else nl - 1
    pads = ids[pl, ::spec.pad_pitch, ::spec.pad_pitch].ravel()
    src = source_terminal(source_index)
    ra.append(pads); rb.append(np.full(pads.size, src)); rg.append(np.full(pads.size, spec.g0))
    if spec.l_pad is not None:
        la.append(pads); lb.append(np.full(pads.size, src)); lv.append(_draw(rng, spec.l_pad, pads.size))

    ca, cv = [], []
    for l in spec.cap_layers:
        a = ids[l].ravel()
        ca.append(a); cv.append(_draw(rng, spec.cap, a.size))

    nload = int(round(spec.load_frac * npl))
    cand = ids[spec.load_layer].ravel()
    pick = np.sort(rng.choice(npl, size=nload, replace=False))
    loads = cand[pick]
    ipk = _draw(rng, spec.ipk, nload)
    tr = _draw(rng, spec.tr, nload)
    tf = _draw(rng, spec.tf, nload)
    t0 = _draw(rng, spec.t0, nload)
    # triangular PWL: 0 at t0, Ipk at t0+tr, 0 at t0+tr+tf
    i_t = np.stack([t0, t0 + tr, t0 + tr + tf], axis=1).ravel()
    i_v = np.stack([np.zeros(nload), ipk, np.zeros(nload)], axis=1).ravel()

    cat = lambda xs, dt: (np.concatenate(xs).astype(dt) if xs else np.zeros(0, dt))
    nl_ = Netlist(
        n_nodes=n, vdd=np.array([spec.vdd]),
        r_a=cat(ra, np.int32), r_b=cat(rb, np.int32), r_g=cat(rg, np.float64),
        c_a=cat(ca, np.int32), c_b=np.full(sum(x.size for x in ca), GROUND, np.int32),
        c_val=cat(cv, np.float64),
        l_a=cat(la, np.int32), l_b=cat(lb, np.int32), l_val=cat(lv, np.float64),
        i_a=loads.astype(np.int32), i_b=np.full(nload, GROUND, np.int32),
        i_ptr=np.arange(0, 3 * nload + 1, 3, dtype=np.int64), i_t=i_t, i_v=i_v,
        lattice=(nx, ny, nl), name=name)
    return nl_


def concat_netlists(parts, name=""):
    """Place independent grids side by side (node ids already offset).

    All parts share the same source nodes.  The result is one netlist whose
    connected components are the parts (the paper's independent sub-circuits,
    Fig. 1).
    """
    def cat(k, dt):
        return np.concatenate([getattr(p, k) for p in parts]).astype(dt)
    ptr = [np.zeros(1, np.int64)]
    off = 0
    for p in parts:
        ptr.append(p.i_ptr[1:] + off)
        off += int(p.i_ptr[-1])
    return Netlist(
        n_nodes=sum(p.n_nodes for p in parts), vdd=parts[0].vdd.copy(),
        r_a=cat("r_a", np.int32), r_b=cat("r_b", np.int32), r_g=cat("r_g", np.float64),
        c_a=cat("c_a", np.int32), c_b=cat("c_b", np.int32), c_val=cat("c_val", np.float64),
        l_a=cat("l_a", np.int32), l_b=cat("l_b", np.int32), l_val=cat("l_val", np.float64),
        i_a=cat("i_a", np.int32), i_b=cat("i_b", np.int32),
        i_ptr=np.concatenate(ptr), i_t=cat("i_t", np.float64), i_v=cat("i_v", np.float64),
        lattice=None, name=name)


# ---------------------------------------------------------------------------
# the five workloads (time step h and step count travel in .meta)
# ---------------------------------------------------------------------------

def config0(seed: int = 0, nx: int = 100, ny: int = 100) -> Netlist:
    """RC single-layer mesh, 100x100: g U[0.5,2] S, C U[10,100] fF on every
    node, G0 = 10 S pads to Vdd = 1 V every 10th node both ways, 20 % of the
    nodes draw triangular PWL loads (Ipk U[0,1] mA, tr/tf U[20,100] ps, t0
    U[0,1] ns).  h = 10 ps, 100 steps, FP64."""
    spec = LatticeSpec(nx=nx, ny=ny, nl=1, g_layer=("uniform", 0.5, 2.0), pad_pitch=10,
                       cap_layers=(0,), cap=("uniform", 10e-15, 100e-15), load_frac=0.2)
    nl = lattice_netlist(spec, np.random.Generator(np.random.PCG64(seed)),
                         name=f"rc_mesh_{nx}x{ny}")
    nl.meta = dict(h=10e-12, nsteps=100, precision="fp64")
    return nl


def config1(seed: int = 1, nx: int = 1024, ny: int = 1024, nl: int = 3) -> Netlist:
    """RC 3-layer grid 1024x1024x3: in-layer g lognormal(0, 0.3) S, vias
    U[5,20] S, pads on the top layer every 32 nodes, decaps U[10,200] fF on
    the bottom layer, 30 % of bottom-layer nodes load as in config 0.
    h = 5 ps, 1000 steps, FP32 sweeps with FP64 residual/defect correction."""
    spec = LatticeSpec(nx=nx, ny=ny, nl=nl, g_layer=("lognormal", 0.0, 0.3),
                       g_via=("uniform", 5.0, 20.0), pad_pitch=32,
                       cap_layers=(0,), cap=("uniform", 10e-15, 200e-15), load_frac=0.3)
    net = lattice_netlist(spec, np.random.Generator(np.random.PCG64(seed)),
                          name=f"rc_grid_{nx}x{ny}x{nl}")
    net.meta = dict(h=5e-12, nsteps=1000, precision="mixed")
    return net


def config2(seed: int = 2, nx: int = 512, ny: int = 512, nl: int = 2) -> Netlist:
    """RLC 2-layer grid 512x512x2: every via is R U[5,20] S in parallel with
    L U[1,10] pH, every pad (top layer, every 16 nodes) is G0 = 10 S in
    parallel with L U[1,10] pH; R and C as config 1; 40 % of the bottom layer
    loads with 10-30 ps edges.  h = 2 ps, 2000 steps, FP64."""
    spec = LatticeSpec(nx=nx, ny=ny, nl=nl, g_layer=("lognormal", 0.0, 0.3),
                       g_via=("uniform", 5.0, 20.0), l_via=("uniform", 1e-12, 10e-12),
                       pad_pitch=16, l_pad=("uniform", 1e-12, 10e-12),
                       cap_layers=(0,), cap=("uniform", 10e-15, 200e-15), load_frac=0.4,
                       tr=("uniform", 10e-12, 30e-12), tf=("uniform", 10e-12, 30e-12))
    net = lattice_netlist(spec, np.random.Generator(np.random.PCG64(seed)),
                          name=f"rlc_grid_{nx}x{ny}x{nl}")
    net.meta = dict(h=2e-12, nsteps=2000, precision="fp64")
    return net


def config3_parts(seed: int = 3, n_grids: int = 256, side_lo: int = 64, side_hi: int = 512):
    """The independent grids of :func:`config3`, each as its own netlist with node
    ids starting at 0, plus the node offset at which it sits in the batch."""
    root = np.random.SeedSequence(seed)
    top = np.random.Generator(np.random.PCG64(root))
    sides = top.integers(side_lo, side_hi + 1, size=n_grids)
    layers = top.integers(1, 3, size=n_grids)
    children = root.spawn(n_grids)
    parts, off = [], 0
    for k in range(n_grids):
        s, nlk = int(sides[k]), int(layers[k])
        spec = LatticeSpec(nx=s, ny=s, nl=nlk, g_layer=("uniform", 0.5, 2.0),
                           g_via=("uniform", 5.0, 20.0), pad_pitch=10,
                           cap_layers=(0,), cap=("uniform", 10e-15, 100e-15), load_frac=0.2)
        part = lattice_netlist(spec, np.random.Generator(np.random.PCG64(children[k])))
        parts.append((off, part))
        off += part.n_nodes
    return parts


def config3_part(k: int, seed: int = 3, n_grids: int = 256, side_lo: int = 64, side_hi: int = 512):
    """Grid ``k`` of :func:`config3` alone, as ``(node offset in the batch, netlist)``:
    the same draws as :func:`config3_parts` without generating the other grids."""
    root = np.random.SeedSequence(seed)
    top = np.random.Generator(np.random.PCG64(root))
    sides = top.integers(side_lo, side_hi + 1, size=n_grids)
    layers = top.integers(1, 3, size=n_grids)
    children = root.spawn(n_grids)
    off = int(np.sum(sides[:k].astype(np.int64) ** 2 * layers[:k]))
    spec = LatticeSpec(nx=int(sides[k]), ny=int(sides[k]), nl=int(layers[k]), g_layer=("uniform", 0.5, 2.0),
                       g_via=("uniform", 5.0, 20.0), pad_pitch=10,
                       cap_layers=(0,), cap=("uniform", 10e-15, 100e-15), load_frac=0.2)
    return off, lattice_netlist(spec, np.random.Generator(np.random.PCG64(children[k])))


def config3_shapes(seed: int = 3, n_grids: int = 256, side_lo: int = 64, side_hi: int = 512):
    """(side, layers) of every grid of :func:`config3`, without generating them."""
    top = np.random.Generator(np.random.PCG64(np.random.SeedSequence(seed)))
    sides = top.integers(side_lo, side_hi + 1, size=n_grids)
    layers = top.integers(1, 3, size=n_grids)
    return [(int(a), int(b)) for a, b in zip(sides, layers)]


def config3(seed: int = 3, n_grids: int = 256, side_lo: int = 64, side_hi: int = 512) -> Netlist:
    """256 independent RC grids of uneven size (side U{64..512}, 1-2 layers),
    each drawn like config 0 from its own child seed; 2-layer grids get vias
    U[5,20] S with pads on the top layer and caps/loads on the bottom layer.
    h = 10 ps, 500 steps, FP32 sweeps with FP64 refinement."""
    parts = config3_parts(seed, n_grids, side_lo, side_hi)
    shifted = []
    for off, p in parts:
        sh = lambda t: np.where(t >= 0, t + off, t).astype(np.int32)
        shifted.append(Netlist(**{**p.__dict__, "r_a": sh(p.r_a), "r_b": sh(p.r_b), "c_a": sh(p.c_a),
                                  "c_b": sh(p.c_b), "l_a": sh(p.l_a), "l_b": sh(p.l_b),
                                  "i_a": sh(p.i_a), "i_b": sh(p.i_b)}))
    net = concat_netlists(shifted, name=f"batched_{n_grids}_rc_grids")
    net.lattices = [(off, *p.lattice) for off, p in parts]
    net.meta = dict(h=10e-12, nsteps=500, precision="mixed",
                    grid_sizes=[p.n_nodes for _, p in parts],
                    grid_shapes=[p.lattice for _, p in parts],
                    grid_offsets=[off for off, _ in parts])
    return net


def config4(seed: int = 4, nx: int = 2048, ny: int = 2048) -> Netlist:
    """RC single-layer 2048x2048 drawn like config 0 (adjoint workload):
    500 steps at h = 10 ps, FP32 sweeps with FP64 accumulation."""
    spec = LatticeSpec(nx=nx, ny=ny, nl=1, g_layer=("uniform", 0.5, 2.0), pad_pitch=10,
                       cap_layers=(0,), cap=("uniform", 10e-15, 100e-15), load_frac=0.2)
    net = lattice_netlist(spec, np.random.Generator(np.random.PCG64(seed)),
                          name=f"rc_mesh_{nx}x{ny}")
    net.meta = dict(h=10e-12, nsteps=500, precision="mixed")
    return net


CONFIGS = {0: config0, 1: config1, 2: config2, 3: config3, 4: config4}
