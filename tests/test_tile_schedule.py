"""The ghost-zone tile schedule of the lattice inner solve, modelled on the host.

The FP32 lattice solve (block red-black SOR over (x, y) columns, Eq. 16-17 with
the via couplings inside the column blocks) runs k exact sweeps per device
barrier.  Each tile does this:
- it loads a region of 34 columns by 34 or 66 rows;
- it applies 2k half-sweeps;
- it stores its (34 - 4k) x (rows - 4k) interior.
Half-sweep hs updates only the columns farther than hs from the region edge.
The columns are assigned as in the kernel: each half-warp row has 16 column
pairs, every thread takes one pair in two rows (34-row regions) or four rows
(66-row regions) per half-sweep, and the half-warps take adjacent rows.

Rows are staged from the 16-byte boundary at or below the region's first
column.  A batch of lattices is one flat tile range: each tile's lattice comes
from a binary search over the first-tile table.  A lattice that has already
converged is skipped, and its correction is zeroed on the first round.

This model replays that index arithmetic in FP64 and checks four things:
- every shared-memory index stays inside the staged rows;
- on widths that are a multiple of 4, every 16-byte piece is wholly inside or wholly outside the lattice;
- every column is stored by exactly one tile, and the stored interior equals k
  global red-black block sweeps exactly, with the same operations in the same
  order;
- in a batch, lattices at any offset behave like that independently (16-byte
  staging where the offset and the width allow it, 4-byte otherwise), and
  skipped lattices end with a zero correction.
"""
import numpy as np
import pytest

SIDE = 34          # region width in columns
W = 36             # shared-memory row stride (the region plus a lead of 0 or 2 columns)
THREADS = 256


def _column_update(f, m, p, u, NL):
    """Thomas elimination of one column block with precomputed factors."""
    for l in range(1, NL):
        f[l] = m[l] * f[l - 1] + f[l]
    x = [0.0] * NL
    x[NL - 1] = f[NL - 1] * p[NL - 1]
    for l in range(NL - 2, -1, -1):
        x[l] = (u[l] * x[l + 1] + f[l]) * p[l]
    return x


def tile_apply(off, nx, ny, NL, k, tile, srcs, dnew, stored, omega, rows=SIDE):
    """One tile of the lattice at global offset ``off``; ``srcs`` are the flat global
    arrays (d, r, wE, wN, wU, m, 1/pivot) and ``dnew`` the flat output."""
    H = 2 * k
    T, TY = SIDE - 2 * H, rows - 2 * H
    J = (rows - 2) // 16
    tiles_x = -(-nx // T)
    plane = nx * ny
    x0, y0 = (tile % tiles_x) * T - H, (tile // tiles_x) * TY - H
    assert x0 % 2 == 0
    lead = x0 & 3
    xa = x0 - lead
    assert xa % 4 == 0 and lead in (0, 2)
    sm = np.zeros((7, NL, rows * W))
    if nx % 4 == 0 and off % 4 == 0:
        chunks = W // 4
        pieces = rows * chunks
        for q in range(pieces * 7):
            a, pos = divmod(q, pieces)
            ry, c4 = pos // chunks, 4 * (pos % chunks)
            xx, yy = xa + c4, y0 + ry
            inside = 0 <= yy < ny and 0 <= xx < nx
            assert inside == (0 <= yy < ny and 0 <= xx + 3 < nx)
            sa = ry * W + c4
            assert 0 <= sa and sa + 3 < rows * W
            if inside:
                for l in range(NL):
                    o = off + yy * nx + xx + l * plane
                    assert o % 4 == 0                       # a 16-byte aligned source
                    sm[a, l, sa:sa + 4] = srcs[a][o:o + 4]
    else:
        for q in range(rows * W):
            ry, c = divmod(q, W)
            xx, yy = xa + c, y0 + ry
            if 0 <= yy < ny and 0 <= xx < nx:
                for a in range(7):
                    for l in range(NL):
                        sm[a, l, q] = srcs[a][off + yy * nx + xx + l * plane]
    sd, sr, se, sn, su, smm, sp = sm
    for hs in range(2 * k):
        touched = set()
        for t in range(THREADS):
            lane, warp = t & 31, t >> 5
            pair, rsub = lane & 15, lane >> 4
            for j in range(J):
                ry = 1 + 2 * (warp + 8 * j) + rsub
                y = y0 + ry
                cx = 1 + 2 * pair + ((hs + x0 + 1 + y) & 1)
                x = x0 + cx
                assert (x + y) % 2 == hs % 2               # this half-sweep's colour
                edge = min(cx, ry, SIDE - 1 - cx, rows - 1 - ry)
                if edge <= hs or not (0 <= x < nx and 0 <= y < ny):
                    continue
                a0 = ry * W + cx + lead
                assert 1 <= cx <= SIDE - 2 and 1 <= ry <= rows - 2 and cx + lead + 1 < W
                assert a0 not in touched
                touched.add(a0)
                f = [sr[l, a0] + se[l, a0] * sd[l, a0 + 1] + se[l, a0 - 1] * sd[l, a0 - 1]
                     + sn[l, a0] * sd[l, a0 + W] + sn[l, a0 - W] * sd[l, a0 - W]
                     for l in range(NL)]
                xv = _column_update(f, smm[:, a0], sp[:, a0], su[:, a0], NL)
                for l in range(NL):
                    dv = sd[l, a0]
                    sd[l, a0] = omega * (xv[l] - dv) + dv
    for q in range(T * TY):
        iy, ix = divmod(q, T)
        x, y = x0 + H + ix, y0 + H + iy
        if x >= nx or y >= ny:
            continue
        for l in range(NL):
            o = off + l * plane + y * nx + x
            dnew[o] = sd[l, (H + iy) * W + H + ix + lead]
            stored[o] += 1


def lattice_round(lats, k, srcs, omega, converged=(), first=True, rows=SIDE):
    """One round over every lattice of a batch, as the kernel schedules it: a flat
    tile index, its lattice found by binary search over the first-tile table, and
    converged lattices skipped (their correction zeroed on the first round)."""
    T, TY = SIDE - 4 * k, rows - 4 * k
    tile0 = [0]
    for (off, nx, ny, nl) in lats:
        tile0.append(tile0[-1] + (-(-nx // T)) * (-(-ny // TY)))
    dnew = np.full_like(srcs[0], np.nan)
    stored = np.zeros(srcs[0].size, int)
    for t in range(tile0[-1]):
        lo, hi = 0, len(lats)
        while hi - lo > 1:
            mid = (lo + hi) >> 1
            if tile0[mid] <= t:
                lo = mid
            else:
                hi = mid
        assert tile0[lo] <= t < tile0[lo + 1]
        off, nx, ny, nl = lats[lo]
        tile = t - tile0[lo]
        if lo in converged:
            if first:
                tiles_x = -(-nx // T)
                tx0, ty0 = (tile % tiles_x) * T, (tile // tiles_x) * TY
                for q in range(T * TY):
                    x, y = tx0 + q % T, ty0 + q // T
                    if x < nx and y < ny:
                        for l in range(nl):
                            o = off + l * nx * ny + y * nx + x
                            dnew[o] = 0.0
                            stored[o] += 1
            continue
        tile_apply(off, nx, ny, nl, k, tile, srcs, dnew, stored, omega, rows)
    assert (stored == 1).all(), "every node of the batch written exactly once"
    return dnew


def tile_round(nx, ny, NL, k, arrs, dold, omega, rows=SIDE):
    srcs = [dold.ravel()] + [a.ravel() for a in arrs]
    return lattice_round([(0, nx, ny, NL)], k, srcs, omega, rows=rows).reshape(dold.shape)


def global_sweeps(nx, ny, NL, k, arrs, d, omega):
    r, wE, wN, wU, m, p = arrs
    d = d.copy()
    for hs in range(2 * k):
        new = d.copy()
        for y in range(ny):
            for x in range(nx):
                if (x + y) % 2 != hs % 2:
                    continue
                f = []
                for l in range(NL):
                    s = r[l, y, x]
                    s += wE[l, y, x] * (d[l, y, x + 1] if x + 1 < nx else 0.0)
                    s += wE[l, y, x - 1] * d[l, y, x - 1] if x > 0 else 0.0
                    s += wN[l, y, x] * (d[l, y + 1, x] if y + 1 < ny else 0.0)
                    s += wN[l, y - 1, x] * d[l, y - 1, x] if y > 0 else 0.0
                    f.append(s)
                xv = _column_update(f, m[:, y, x], p[:, y, x], wU[:, y, x], NL)
                for l in range(NL):
                    new[l, y, x] = omega * (xv[l] - d[l, y, x]) + d[l, y, x]
        d = new
    return d


@pytest.mark.parametrize("nx,ny,NL,k", [(32, 28, 3, 2), (61, 37, 2, 2), (52, 60, 1, 1),
                                        (27, 27, 3, 3), (8, 6, 2, 2), (72, 34, 3, 2),
                                        (70, 30, 2, 2), (48, 40, 1, 3)])
def test_tile_round_is_k_global_block_sweeps(nx, ny, NL, k):
    rng = np.random.default_rng(nx * 1000 + ny)
    arrs = [rng.uniform(-1, 1, (NL, ny, nx))] + [rng.uniform(0.05, 0.2, (NL, ny, nx)) for _ in range(5)]
    d = rng.uniform(-1, 1, (NL, ny, nx))
    got = tile_round(nx, ny, NL, k, arrs, d, 1.3)
    want = global_sweeps(nx, ny, NL, k, arrs, d, 1.3)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("nx,ny,NL,k", [(32, 130, 3, 2), (61, 75, 2, 3), (44, 70, 1, 1), (8, 6, 2, 2),
                                        (36, 140, 3, 3)])
def test_tall_tile_round_is_k_global_block_sweeps(nx, ny, NL, k):
    """66-row regions (four rows per thread per half-sweep): the same sweeps, exactly."""
    rng = np.random.default_rng(nx * 1000 + ny + 7)
    arrs = [rng.uniform(-1, 1, (NL, ny, nx))] + [rng.uniform(0.05, 0.2, (NL, ny, nx)) for _ in range(5)]
    d = rng.uniform(-1, 1, (NL, ny, nx))
    got = tile_round(nx, ny, NL, k, arrs, d, 1.3, rows=66)
    want = global_sweeps(nx, ny, NL, k, arrs, d, 1.3)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("lats_shape,k,converged", [
    ([(5, 3, 3), (30, 27, 3), (2, 7, 1)], 2, ()),          # odd offsets: 4-byte staging
    ([(8, 4, 1), (12, 8, 2), (36, 20, 3)], 2, ()),         # offsets and widths multiples of 4
    ([(8, 4, 1), (12, 8, 2), (36, 20, 3)], 3, (1,)),       # a converged lattice is skipped
    ([(26, 26, 2), (27, 5, 1)], 1, (0,)),
])
def test_batched_round(lats_shape, k, converged):
    rng = np.random.default_rng(len(lats_shape) * 10 + k)
    lats, off = [], 0
    for (nx, ny, nl) in lats_shape:
        lats.append((off, nx, ny, nl))
        off += nx * ny * nl
    N = off
    d = rng.uniform(-1, 1, N)
    arrs = [rng.uniform(-1, 1, N)] + [rng.uniform(0.05, 0.2, N) for _ in range(5)]
    got = lattice_round(lats, k, [d] + arrs, 1.3, converged=converged)
    for L, (o, nx, ny, nl) in enumerate(lats):
        sl = slice(o, o + nx * ny * nl)
        if L in converged:
            assert not got[sl].any()
            continue
        shape = (nl, ny, nx)
        want = global_sweeps(nx, ny, nl, k, [a[sl].reshape(shape) for a in arrs], d[sl].reshape(shape), 1.3)
        assert np.array_equal(got[sl].reshape(shape), want), f"lattice {L}"



@pytest.mark.parametrize("tiles,blocks", [(2209, 304), (5, 8), (1, 1), (16, 3), (100, 152)])
def test_tile_claims_cover_every_round_once(tiles, blocks):
    """The kernel hands a round's tiles out from one launch-wide counter: each block
    claims its first tile, then claims the next one while it works on the current one,
    and stops at its first claim at or past round_base + tiles, with round_base =
    n (tiles + blocks) for round n (modulo 2^32 like the counter).  Under any order in
    which the blocks' claims interleave, every tile of every round must be processed
    exactly once and the counter must stand at (n + 1)(tiles + blocks) after round n."""
    import random
    rnd = random.Random(tiles * 31 + blocks)
    ctr = 0
    for n in range(6):
        base = (n * (tiles + blocks)) % 2**32
        claim = {}
        for b in rnd.sample(range(blocks), blocks):          # first claims, in any order
            claim[b] = ctr % 2**32
            ctr += 1
        done, active = [], list(range(blocks))
        while active:
            b = rnd.choice(active)
            t = (claim[b] - base) % 2**32
            if t < tiles:
                claim[b] = ctr % 2**32
                ctr += 1
                done.append(t)
            else:
                active.remove(b)
        assert sorted(done) == list(range(tiles))
        assert ctr == (n + 1) * (tiles + blocks)
