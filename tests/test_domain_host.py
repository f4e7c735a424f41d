"""Row-block domain decomposition of one lattice grid over gloo ranks on the CPU.

With a one-row halo exchanged after every colour half-sweep, the red-black
iteration decomposed over 2 or 3 ranks must make exactly the updates of the
undecomposed one (Eq. 16-17 read only a node's neighbours, and red-black order
puts the two colours in separate half-sweeps).  The test checks four things:
- the result is bit-identical to the undecomposed run;
- the sweep count is the same;
- the solution is the direct solution of the nodal system;
- the halo rows hold the neighbours' boundary rows.
The block half-sweep here is a plain numpy restatement of Eq. 17 on a lattice
with random per-edge conductances.
"""
import os
import socket

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla
import torch

from paper_1409_7166_gb300 import domain

NX, NY, NL = 9, 11, 3          # ragged row blocks: 6+5 on 2 ranks, 4+4+3 on 3
OMEGA, TOL, MAX_SWEEPS = 1.4, 1e-13, 4000


def _problem(seed=4):
    rng = np.random.default_rng(seed)
    gx = rng.uniform(0.5, 2.0, (NL, NY, NX)); gx[:, :, -1] = 0.0   # edge (x, x+1)
    gy = rng.uniform(0.5, 2.0, (NL, NY, NX)); gy[:, -1, :] = 0.0   # edge (y, y+1)
    gz = rng.uniform(1.0, 5.0, (NL, NY, NX)); gz[-1] = 0.0         # via (l, l+1)
    g0 = rng.uniform(0.2, 0.6, (NL, NY, NX))   # C/h plus pad conductance
    b = rng.uniform(0.0, 1.0, (NL, NY, NX))
    return gx, gy, gz, g0, b


def _diagonal(gx, gy, gz, g0):
    D = g0 + gx + gy + gz
    D[:, :, 1:] += gx[:, :, :-1]
    D[:, 1:, :] += gy[:, :-1, :]
    D[1:] += gz[:-1]
    return D


def _half_sweep_for(P, y0, rows):
    """Eq. 17 on the rows [y0, y0 + rows) of the lattice, halos at local rows 0 and rows + 1."""
    gx, gy, gz, g0, b = P
    sl = slice(y0, y0 + rows)
    D = _diagonal(gx, gy, gz, g0)[:, sl]
    bb = b[:, sl]
    w_e = gx[:, sl]
    w_w = np.zeros_like(w_e); w_w[:, :, 1:] = gx[:, sl, :-1]
    w_n = gy[:, sl]
    w_s = np.zeros_like(w_n)
    w_s[:, 1:] = gy[:, y0:y0 + rows - 1]
    if y0 > 0:
        w_s[:, 0] = gy[:, y0 - 1]
    w_u = gz[:, sl]
    w_d = np.zeros_like(w_u); w_d[1:] = gz[:-1, sl]
    l, y, x = np.meshgrid(np.arange(NL), np.arange(y0, y0 + rows), np.arange(NX), indexing="ij")
    parity = (l + y + x) % 2

    def half_sweep(xl, colour, y0_):
        assert y0_ == y0
        X = xl.numpy()
        c = X[:, 1:rows + 1, :]
        xw = np.zeros_like(c); xw[:, :, 1:] = c[:, :, :-1]
        xe = np.zeros_like(c); xe[:, :, :-1] = c[:, :, 1:]
        xd = np.zeros_like(c); xd[1:] = c[:-1]
        xu = np.zeros_like(c); xu[:-1] = c[1:]
        s = bb + w_w * xw + w_e * xe + w_s * X[:, 0:rows, :] + w_n * X[:, 2:rows + 2, :] + w_d * xd + w_u * xu
        new = c + OMEGA * (s / D - c)
        m = parity == colour
        upd = np.max(np.abs(new[m] - c[m])) if m.any() else 0.0
        c[m] = new[m]
        return float(upd)

    return half_sweep


def _run(P, rank, world):
    halo = domain.HaloExchange(NX, NY, NL, rank, world)
    x = torch.zeros(halo.local_shape(), dtype=torch.float64)
    sweeps, est = domain.red_black_sor(x, halo, _half_sweep_for(P, halo.y0, halo.rows),
                                       MAX_SWEEPS, TOL, check_every=4)
    return x, halo, sweeps, est


def _direct(P):
    gx, gy, gz, g0, b = P
    n = NL * NY * NX
    idx = np.arange(n).reshape(NL, NY, NX)
    rows, cols, vals = [], [], []
    for w, a, c in ((gx[:, :, :-1], idx[:, :, :-1], idx[:, :, 1:]),
                    (gy[:, :-1, :], idx[:, :-1, :], idx[:, 1:, :]),
                    (gz[:-1], idx[:-1], idx[1:])):
        rows += [a.ravel(), c.ravel()]; cols += [c.ravel(), a.ravel()]; vals += [-w.ravel(), -w.ravel()]
    rows.append(idx.ravel()); cols.append(idx.ravel()); vals.append(_diagonal(gx, gy, gz, g0).ravel())
    M = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    return spla.spsolve(M.tocsc(), b.ravel()).reshape(NL, NY, NX)


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
        halo = domain.HaloExchange(NX, NY, NL, rank, world)
        # halo contents: fill own rows with their global row index
        probe = torch.full(halo.local_shape(), -1.0, dtype=torch.float64)
        probe[:, 1:halo.rows + 1, :] = torch.arange(halo.y0, halo.y1, dtype=torch.float64).view(1, -1, 1)
        halo.exchange(probe)
        below = float(probe[0, 0, 0]) if halo.below is not None else None
        above = float(probe[0, halo.rows + 1, 0]) if halo.above is not None else None
        uniform = bool((probe[:, 0] == probe[0, 0, 0]).all() and (probe[:, -1] == probe[0, -1, 0]).all())
        x, halo, sweeps, est = _run(_problem(), rank, world)
        full = domain.gather_rows(x, halo)
        info = torch.tensor([halo.y0, halo.y1, -2 if below is None else below,
                             -2 if above is None else above, float(uniform), sweeps, est], dtype=torch.float64)
        parts = [None] * world if rank == 0 else None
        dist.gather_object(info, parts, dst=0)
        if rank == 0:
            np.savez(out_path, full=full.numpy(), info=torch.stack(parts).numpy())
    finally:
        dist.destroy_process_group()


def test_row_blocks_partition():
    for ny in (1, 2, 7, 11, 1024):
        for world in range(1, min(ny, 9) + 1):
            blocks = domain.row_blocks(ny, world)
            assert blocks[0][0] == 0 and blocks[-1][1] == ny
            assert all(a[1] == b[0] for a, b in zip(blocks, blocks[1:]))
            sizes = [y1 - y0 for y0, y1 in blocks]
            assert min(sizes) >= 1 and max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        domain.row_blocks(3, 4)
    with pytest.raises(ValueError):
        domain.row_blocks(3, 0)


def test_single_domain_red_black_reaches_the_direct_solution():
    P = _problem()
    x, halo, sweeps, est = _run(P, 0, 1)
    assert est <= TOL and sweeps < MAX_SWEEPS
    ref = _direct(P)
    assert np.max(np.abs(x[:, 1:NY + 1].numpy() - ref)) <= 1e-10
    # the outer halos of the undecomposed grid are never written
    assert not x[:, 0].any() and not x[:, NY + 1].any()


@pytest.mark.parametrize("world", [2, 3])
def test_decomposed_red_black_is_bit_identical(tmp_path, world):
    import torch.multiprocessing as mp
    out = str(tmp_path / "dd.npz")
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn", join=True)
    got = np.load(out)
    P = _problem()
    x1, _, sweeps1, est1 = _run(P, 0, 1)
    assert np.array_equal(got["full"], x1[:, 1:NY + 1].numpy())
    info = got["info"]
    for r, (y0, y1, below, above, uniform, sweeps, est) in enumerate(info):
        assert (y0, y1) == domain.row_blocks(NY, world)[r]
        assert below == (y0 - 1 if r > 0 else -2)
        assert above == (y1 if r < world - 1 else -2)
        assert uniform == 1.0
        assert sweeps == sweeps1 and est == est1
