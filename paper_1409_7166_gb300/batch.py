"""Many independent grids: one batch per GPU, the batch split across ranks.

Grids that share no element are independent sub-circuits (Section III-B,
Fig. 1): the system matrix is block diagonal and every block is solved on its
own.  One GPU solves its grids as one netlist in one persistent launch (the
library splits components and iterates them together, skipping lattices that
have converged).  Several ranks split the grids by longest-processing-time
(LPT) on an estimated cost; nothing is exchanged while the transients run, and
the per-grid worst-drop waveforms are gathered on rank 0 at the end.

This module is host logic only (partitioning, node renumbering, the gather);
every step of the transient runs in the library's kernels.
"""
from __future__ import annotations

import heapq
from types import SimpleNamespace
from typing import Callable, Dict, List, Optional, Sequence

import numpy as np

_FIELDS_I32 = ("r_a", "r_b", "c_a", "c_b", "l_a", "l_b", "i_a", "i_b")
_FIELDS_F64 = ("r_g", "c_val", "l_val", "i_t", "i_v")


def grid_cost(net) -> float:
    """Relative cost of one grid's transient: nodes x the sweeps a step needs.

    Red-black SOR with Young's omega needs O(side) sweeps for a lattice of
    side `side` (the spectral gap of the Jacobi matrix shrinks like 1/side^2,
    and optimal SOR converts it to 1/side), so the cost grows like n * side.
    Without a lattice description, side is taken as sqrt(n).
    """
    lat = getattr(net, "lattice", None)
    side = float(max(lat[0], lat[1])) if lat else float(np.sqrt(max(net.n_nodes, 1)))
    return float(net.n_nodes) * side


def lpt_partition(costs: Sequence[float], n_ranks: int) -> List[List[int]]:
    """Assign items to ranks, largest cost first, each to the least-loaded rank
    (ties go to the lower rank; equal costs keep their index order).  Returns
    each rank's item indices in increasing order."""
    if n_ranks < 1:
        raise ValueError("n_ranks must be >= 1")
    order = sorted(range(len(costs)), key=lambda k: (-float(costs[k]), k))
    heap = [(0.0, r) for r in range(n_ranks)]
    out: List[List[int]] = [[] for _ in range(n_ranks)]
    for k in order:
        load, r = heapq.heappop(heap)
        out[r].append(k)
        heapq.heappush(heap, (load + float(costs[k]), r))
    return [sorted(ks) for ks in out]


def concat(grids: Sequence) -> SimpleNamespace:
    """One netlist holding the given grids side by side.

    Node ids of grid j are shifted by the node count of grids 0..j-1; ground
    and source terminals (negative ids) keep their meaning, so all grids must
    use the same source list.  Each grid that describes itself as one lattice
    contributes a lattice entry (first id, nx, ny, nl), which lets the library
    run its column-block inner solve on every grid of the batch.
    """
    if not grids:
        raise ValueError("no grids")
    vdd = np.asarray(grids[0].vdd, dtype=np.float64)
    for gr in grids[1:]:
        if not np.array_equal(np.asarray(gr.vdd, dtype=np.float64), vdd):
            raise ValueError("all grids of a batch must share the source list")
    fields: Dict[str, list] = {k: [] for k in _FIELDS_I32 + _FIELDS_F64}
    ptr, lattices = [np.zeros(1, np.int64)], []
    off, pw = 0, 0
    all_lattice = True
    for gr in grids:
        for k in _FIELDS_I32:
            a = np.asarray(getattr(gr, k), dtype=np.int32)
            fields[k].append(np.where(a >= 0, a + off, a).astype(np.int32))
        for k in _FIELDS_F64:
            fields[k].append(np.asarray(getattr(gr, k), dtype=np.float64))
        ip = np.asarray(gr.i_ptr, dtype=np.int64)
        ptr.append(ip[1:] + pw)
        pw += int(ip[-1])
        lat = getattr(gr, "lattice", None)
        if lat:
            lattices.append((off, int(lat[0]), int(lat[1]), int(lat[2])))
        else:
            all_lattice = False
        off += int(gr.n_nodes)
    out = SimpleNamespace(n_nodes=off, n_sources=int(vdd.shape[0]), vdd=vdd.copy(), i_ptr=np.concatenate(ptr),
                          lattice=None, lattices=lattices if all_lattice else None, name=f"batch_of_{len(grids)}")
    for k, parts in fields.items():
        setattr(out, k, np.concatenate(parts))
    return out


def solve_grids_gpu(grids: Sequence, h: float, nsteps: int, device: Optional[int] = None,
                    **options) -> np.ndarray:
    """Worst-drop waveform of every grid: ``[nsteps, len(grids)]`` (smallest node
    voltage of grid j after each step), from one persistent launch on this
    process's GPU."""
    import torch

    from . import binding as B

    net = concat(grids)
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
    with torch.cuda.device(dev), B.Grid(net, **options) as g:
        B.pg_set_stream(g.handle, torch.cuda.current_stream().cuda_stream)
        n_comp, _ = B.pg_grid_components(g.handle)
        if n_comp != len(grids):
            raise ValueError(f"the grids are not independent: {n_comp} components for {len(grids)} grids")
        out = torch.empty((nsteps, n_comp), dtype=torch.float64, device=dev)
        B.pg_transient(g.handle, h, nsteps, comp_vmin=out)
        return out.cpu().numpy()


def scenario_copies(net, load_values: Sequence) -> List[SimpleNamespace]:
    """Copies of ``net`` that differ only in their load values: copy j draws the PWL
    currents ``load_values[j]`` (same breakpoints as ``net.i_t``, same length as
    ``net.i_v``).  Solved together (:func:`solve_grids_gpu`), the scenarios share one
    persistent launch and its device barriers; each copy keeps its own weights."""
    fields = ("n_nodes", "vdd", "r_a", "r_b", "r_g", "c_a", "c_b", "c_val", "l_a", "l_b", "l_val",
              "i_a", "i_b", "i_ptr", "i_t")
    base = {k: getattr(net, k) for k in fields}
    out = []
    for iv in load_values:
        iv = np.asarray(iv, dtype=np.float64)
        if iv.shape != np.asarray(net.i_v).shape:
            raise ValueError("every scenario needs one value per PWL breakpoint")
        out.append(SimpleNamespace(**base, i_v=iv, lattice=getattr(net, "lattice", None)))
    return out


def solve_scenarios(net, load_values: Sequence, h: float, nsteps: int, **options) -> np.ndarray:
    """Worst-drop waveform of every load scenario of ``net``: ``[nsteps, len(load_values)]``,
    all scenarios in one persistent launch on this process's GPU."""
    return solve_grids_gpu(scenario_copies(net, load_values), h, nsteps, **options)


def solve_scenarios_shared(net, load_values: Sequence, h: float, nsteps: int, device: Optional[int] = None,
                           **options) -> np.ndarray:
    """Like :func:`solve_scenarios`, but the scenarios share one copy of the grid: one
    launch of ``pg_transient_scenarios`` relaxes every right-hand side together, each
    coefficient read once for all of them.  Needs an RC grid; ``options`` as for
    :class:`binding.Grid` (the lattice inner solve where the grid's options choose it).
    Returns ``[nsteps, len(load_values)]``."""
    import torch

    from . import binding as B

    dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
    iv = torch.tensor(np.stack([np.asarray(v, dtype=np.float64) for v in load_values]), device=dev)
    with torch.cuda.device(dev):
        with B.Grid(net, **options) as g:
            B.pg_set_stream(g.handle, torch.cuda.current_stream(dev).cuda_stream)
            vmin = torch.empty((nsteps, len(load_values)), dtype=torch.float64, device=dev)
            B.pg_transient_scenarios(g.handle, h, nsteps, iv, vmin=vmin)
            torch.cuda.synchronize(dev)
            return vmin.cpu().numpy()


def solve_sharded(grids: Sequence, h: float, nsteps: int,
                  solver: Optional[Callable[[Sequence, float, int], np.ndarray]] = None,
                  costs: Optional[Sequence[float]] = None, **options) -> Optional[np.ndarray]:
    """Split ``grids`` over the ranks of the default process group (one rank
    when torch.distributed is not initialised), solve each rank's share with
    ``solver`` (default :func:`solve_grids_gpu` with ``options``) and gather
    the worst-drop waveforms on rank 0.  Returns ``[nsteps, len(grids)]`` in the
    caller's grid order on rank 0 and None elsewhere.  No collective runs while
    the transients run: the only exchange is the final gather."""
    import torch.distributed as dist

    active = dist.is_available() and dist.is_initialized()
    rank = dist.get_rank() if active else 0
    world = dist.get_world_size() if active else 1
    costs = [grid_cost(gr) for gr in grids] if costs is None else list(costs)
    shares = lpt_partition(costs, world)
    mine = shares[rank]
    if solver is None:
        def solver(gs, hh, ns):
            return solve_grids_gpu(gs, hh, ns, **options)
    local = solver([grids[k] for k in mine], h, nsteps) if mine else np.zeros((nsteps, 0))
    if not active:
        res = np.empty((nsteps, len(grids)))
        res[:, mine] = local
        return res
    gathered = [None] * world if rank == 0 else None
    dist.gather_object((mine, np.asarray(local)), gathered, dst=0)
    if rank != 0:
        return None
    res = np.full((nsteps, len(grids)), np.nan)
    for ks, vals in gathered:
        if ks:
            res[:, ks] = vals
    return res
