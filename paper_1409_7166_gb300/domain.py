"""Row-block domain decomposition of one lattice grid across ranks.

The node update of Eq. 16-17 reads only the node's own value and its
neighbours', so one red-black half-sweep over a block of lattice rows needs,
from the other colour, only the row just below and the row just above the
block.  The grid (nodes (x, y, l), all layers of a column kept together, so the
vias stay inside a block) is cut along y into contiguous row blocks, one per
rank:
- every rank updates its rows of the current colour;
- it sends its first and last rows to the neighbouring ranks;
- it receives their boundary rows into its halo rows before the next half-sweep.

The global red-black order is unchanged, so the decomposed iteration performs
exactly the same updates as the undecomposed one.  Every `check_every` sweeps
the ranks agree on the stopping test through a max all-reduce of their
residual estimate.

This module is the host side of that schedule: the partition, the halo
exchange (torch.distributed point-to-point; gloo on the CPU, NCCL for device
tensors), and the sweep loop.  The half-sweep over a block is supplied by the
caller; on the GPU it is the library's ``pg_block_half_sweep``.  Several blocks
of one grid can also be held in one process (``split_blocks``,
``LocalHaloExchange``, ``red_black_sor_blocks``), their halos refreshed by
device copies.
"""
from __future__ import annotations

from typing import Callable, List, Optional, Tuple

import torch


def row_blocks(ny: int, world: int) -> List[Tuple[int, int]]:
    """Contiguous row ranges ``[y0, y1)`` covering ``0..ny``, sizes differing by at most 1."""
    if world < 1 or ny < world:
        raise ValueError("need at least one row per rank")
    base, extra = divmod(ny, world)
    out, y = [], 0
    for r in range(world):
        h = base + (1 if r < extra else 0)
        out.append((y, y + h))
        y += h
    return out


class HaloExchange:
    """Halo rows of one rank's block.

    The local array has shape ``[nl, rows + 2, nx]``: row 0 is the halo below
    the block (the last row of rank - 1), row ``rows + 1`` the halo above (the
    first row of rank + 1), and rows ``1..rows`` are the rank's own.  At the
    outer edges of the grid the halos stay zero and are never read as
    neighbours, because those nodes have no neighbour across the edge.
    """

    def __init__(self, nx: int, ny: int, nl: int, rank: int, world: int, group=None):
        self.nx, self.ny, self.nl = nx, ny, nl
        self.rank, self.world, self.group = rank, world, group
        self.y0, self.y1 = row_blocks(ny, world)[rank]
        self.rows = self.y1 - self.y0
        self.below = rank - 1 if rank > 0 else None
        self.above = rank + 1 if rank + 1 < world else None

    def local_shape(self) -> Tuple[int, int, int]:
        return (self.nl, self.rows + 2, self.nx)

    def exchange(self, x: torch.Tensor) -> None:
        """Send the block's boundary rows and receive the neighbours' into the halos."""
        import torch.distributed as dist
        reqs, recvs = [], []
        if self.below is not None:
            send = x[:, 1, :].contiguous()
            recv = torch.empty_like(send)
            reqs.append(dist.isend(send, self.below, group=self.group))
            reqs.append(dist.irecv(recv, self.below, group=self.group))
            recvs.append((0, recv))
        if self.above is not None:
            send = x[:, self.rows, :].contiguous()
            recv = torch.empty_like(send)
            reqs.append(dist.isend(send, self.above, group=self.group))
            reqs.append(dist.irecv(recv, self.above, group=self.group))
            recvs.append((self.rows + 1, recv))
        for r in reqs:
            r.wait()
        for row, recv in recvs:
            x[:, row, :] = recv

    def max_all(self, value: float) -> float:
        """Max of a scalar over all ranks (the stopping test every rank must agree on)."""
        if self.world == 1:
            return float(value)
        import torch.distributed as dist
        t = torch.tensor([float(value)], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX, group=self.group)
        return float(t.item())


def red_black_sor(x: torch.Tensor, halo: HaloExchange,
                  half_sweep: Callable[[torch.Tensor, int, int], float],
                  max_sweeps: int, tol: float, check_every: int = 4) -> Tuple[int, float]:
    """Red-black SOR on one rank's block with halo exchange after each half-sweep.

    ``half_sweep(x, colour, y0)`` updates the block's nodes of one colour (the
    parity of x + y + l, with y the global row ``y0 + local row - 1``) in place,
    reading halo rows for the neighbours across the block edges.  It returns
    the largest update it made.  Every ``check_every`` sweeps the ranks take the
    max of their largest update over the last sweep.  They stop together once it
    is at most ``tol``, or after ``max_sweeps``.  Returns ``(sweeps, last
    global max update)``.
    """
    halo.exchange(x)
    est = float("inf")
    for k in range(1, max_sweeps + 1):
        m = 0.0
        for colour in (0, 1):
            m = max(m, half_sweep(x, colour, halo.y0))
            halo.exchange(x)
        if k % check_every == 0 or k == max_sweeps:
            est = halo.max_all(m)
            if est <= tol:
                return k, est
    return max_sweeps, est


def gather_rows(x: torch.Tensor, halo: HaloExchange, root: int = 0) -> Optional[torch.Tensor]:
    """The full ``[nl, ny, nx]`` field on ``root`` (None elsewhere)."""
    own = x[:, 1:halo.rows + 1, :].contiguous()
    if halo.world == 1:
        return own
    import torch.distributed as dist
    parts = [None] * halo.world if halo.rank == root else None
    dist.gather_object(own, parts, dst=root, group=halo.group)
    if halo.rank != root:
        return None
    return torch.cat(parts, dim=1)


# ---------------------------------------------------------------------------
# several row blocks of one grid in one process (device tensors)
# ---------------------------------------------------------------------------

def split_blocks(w_e: torch.Tensor, w_n: torch.Tensor, w_u: torch.Tensor, inv_d: torch.Tensor,
                 rhs: torch.Tensor, world: int) -> List[dict]:
    """Cut full-grid coefficient arrays, each ``[nl, ny, nx]``, into ``world`` row blocks.

    ``w_e``: conductance (x, y, l)-(x + 1, y, l), zero on the last column; ``w_n``:
    (x, y, l)-(x, y + 1, l), zero on the last row; ``w_u``: (x, y, l)-(x, y, l + 1), zero
    on the top layer; ``inv_d``: 1 / D (Eq. 14); ``rhs``: the right-hand side.  Each block
    gets the layout of ``pg_row_block``: its rows of every layer, the north couplings of
    its rows plus the one from the row below it (``[nl, rows + 1, nx]``), and a zero
    iterate with one halo row on each side (``[nl, rows + 2, nx]``)."""
    nl, ny, nx = w_e.shape
    out = []
    for (y0, y1) in row_blocks(ny, world):
        rows = y1 - y0
        wn = torch.zeros((nl, rows + 1, nx), dtype=w_n.dtype, device=w_n.device)
        if y0 > 0:
            wn[:, 0] = w_n[:, y0 - 1]
        wn[:, 1:] = w_n[:, y0:y1]
        out.append(dict(nx=nx, rows=rows, nl=nl, y0=y0,
                        w_e=w_e[:, y0:y1].contiguous(), w_n=wn, w_u=w_u[:, y0:y1].contiguous(),
                        inv_d=inv_d[:, y0:y1].contiguous(), rhs=rhs[:, y0:y1].contiguous(),
                        x=torch.zeros((nl, rows + 2, nx), dtype=rhs.dtype, device=rhs.device)))
    return out


class LocalHaloExchange:
    """The halo exchange between row blocks held in one process: after a half-sweep,
    each block's first and last rows are copied into the halos of the blocks below
    and above it (device-to-device copies on the current stream)."""

    def __init__(self, blocks: List[dict]):
        self.blocks = blocks

    def exchange(self) -> None:
        for lo, hi in zip(self.blocks[:-1], self.blocks[1:]):
            lo["x"][:, lo["rows"] + 1].copy_(hi["x"][:, 1])
            hi["x"][:, 0].copy_(lo["x"][:, lo["rows"]])


def red_black_sor_blocks(blocks: List[dict], half_sweep: Callable[[dict, int, torch.Tensor], None],
                         max_sweeps: int, tol: float, check_every: int = 4) -> Tuple[int, float]:
    """Red-black SOR over every block of one process, in the schedule of
    :func:`red_black_sor`: per colour, every block's half-sweep, then the halo exchange;
    every ``check_every`` sweeps the largest update of the last sweep over all blocks
    decides the stop.  ``half_sweep(block, colour, max_update)`` max-merges its largest
    update into the device scalar ``max_update``."""
    halo = LocalHaloExchange(blocks)
    dev = blocks[0]["x"].device
    mx = torch.zeros(1, dtype=torch.float64, device=dev)
    est = float("inf")
    halo.exchange()
    for k in range(1, max_sweeps + 1):
        mx.zero_()
        for colour in (0, 1):
            for blk in blocks:
                half_sweep(blk, colour, mx)
            halo.exchange()
        if k % check_every == 0 or k == max_sweeps:
            est = float(mx.item())
            if est <= tol:
                return k, est
    return max_sweeps, est


def gather_blocks(blocks: List[dict]) -> torch.Tensor:
    """The full ``[nl, ny, nx]`` field from the blocks' own rows."""
    return torch.cat([b["x"][:, 1:b["rows"] + 1] for b in blocks], dim=1)
