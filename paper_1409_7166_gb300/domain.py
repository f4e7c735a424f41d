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
caller.
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
