"""Host logic of the batched, sharded workload (CPU only): the LPT split, the
netlist concatenation, and the rank-0 gather over a real 2-rank gloo group.

The per-rank solver here is the oracle, so these tests pin the partition and
gather logic, not the kernels (the GPU path of the same function is in
tests/test_gpu_batch.py).
"""
import itertools
import os
import socket

import numpy as np
import pytest

import pgsynth
from oracle import transient
from paper_1409_7166_gb300 import batch


def _brute_makespan(costs, m):
    best = float("inf")
    for assign in itertools.product(range(m), repeat=len(costs)):
        loads = [0.0] * m
        for c, r in zip(costs, assign):
            loads[r] += c
        best = min(best, max(loads))
    return best


@pytest.mark.parametrize("seed", range(6))
def test_lpt_partition_is_a_partition_within_graham_bound(seed):
    rng = np.random.default_rng(seed)
    n, m = int(rng.integers(3, 9)), int(rng.integers(2, 4))
    costs = rng.uniform(1.0, 10.0, n)
    shares = batch.lpt_partition(costs, m)
    assert sorted(k for s in shares for k in s) == list(range(n))
    makespan = max(sum(costs[k] for k in s) for s in shares)
    # Graham: LPT is within 4/3 - 1/(3m) of the optimum
    assert makespan <= (4.0 / 3.0 - 1.0 / (3 * m)) * _brute_makespan(costs, m) + 1e-9


def test_lpt_ties_and_degenerate_cases():
    assert batch.lpt_partition([1.0, 1.0, 1.0, 1.0], 2) == [[0, 2], [1, 3]]
    assert batch.lpt_partition([5.0], 3) == [[0], [], []]
    assert batch.lpt_partition([], 2) == [[], []]
    with pytest.raises(ValueError):
        batch.lpt_partition([1.0], 0)


def _grids(k=4, seed=2):
    return [p for _, p in pgsynth.config3_parts(n_grids=k, side_lo=6, side_hi=11, seed=seed)]


def _oracle_worst(grids, h, nsteps):
    """Per-grid worst drop of the concatenated share, from the oracle's direct solves."""
    net = batch.concat(grids)
    V, _ = transient.transient(net, h, nsteps)
    out, off = np.empty((nsteps, len(grids))), 0
    for j, gr in enumerate(grids):
        out[:, j] = V[1:, off:off + gr.n_nodes].min(axis=1)
        off += gr.n_nodes
    return out


def test_concat_keeps_grids_independent():
    grids = _grids()
    net = batch.concat(grids)
    assert net.n_nodes == sum(g.n_nodes for g in grids)
    assert [l[0] for l in net.lattices] == list(np.cumsum([0] + [g.n_nodes for g in grids[:-1]]))
    h, S = 10e-12, 15
    V, _ = transient.transient(net, h, S)
    off = 0
    for gr in grids:            # the batch's trajectory restricted to a grid is that grid's own (Fig. 1)
        Vg, _ = transient.transient(gr, h, S)
        assert np.max(np.abs(V[:, off:off + gr.n_nodes] - Vg)) <= 1e-12
        off += gr.n_nodes


def test_solve_sharded_single_process():
    grids = _grids(5, seed=4)
    h, S = 10e-12, 12
    res = batch.solve_sharded(grids, h, S, solver=_oracle_worst)
    ref = _oracle_worst(grids, h, S)
    assert np.max(np.abs(res - ref)) <= 1e-12


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        grids = _grids(7, seed=5)
        res = batch.solve_sharded(grids, 10e-12, 12, solver=_oracle_worst)
        if rank == 0:
            np.save(out_path, res)
        else:
            assert res is None
    finally:
        dist.destroy_process_group()


def test_solve_sharded_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    out = str(tmp_path / "res.npy")
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, start_method="spawn", join=True)
    grids = _grids(7, seed=5)
    ref = _oracle_worst(grids, 10e-12, 12)
    res = np.load(out)
    assert not np.isnan(res).any()
    assert np.max(np.abs(res - ref)) <= 1e-12
    # each rank solved its LPT share only
    shares = batch.lpt_partition([batch.grid_cost(g) for g in grids], 2)
    assert all(shares) and sorted(shares[0] + shares[1]) == list(range(7))
