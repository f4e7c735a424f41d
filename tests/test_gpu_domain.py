"""The device half of the row-block domain decomposition of one grid, on one GPU.

Several row blocks of one lattice are held in one process; each colour
half-sweep (Eq. 16-17) runs on every block through the C ABI
(``pg_block_half_sweep``), and the blocks' halo rows are refreshed by device
copies after it.  Red-black order puts the colours in separate half-sweeps, so
the decomposed iteration must make exactly the updates of the undecomposed one
(a single block with every row): the test checks that bit for bit on 2 and 3
ragged blocks, with the same sweep count, and that the halos hold the
neighbours' boundary rows.  The common fixed point is checked against direct
solves: of a lattice with random per-edge conductances, and of one
backward-Euler step of the 3-layer grid recipe assembled by the oracle (Eq. 2,
M = C/h + G + G0).  Only the transport between GPUs (NCCL point-to-point into
the same halo rows) is not exercised: a box here has one GPU.
"""
import numpy as np
import pytest

import pgsynth
from oracle import matrices, transient

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_V = 1e-6


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1409_7166_gb300 import binding
    return binding


def _lattice_coefficients(M, nx, ny, nl):
    """w_e, w_n, w_u, D of a lattice nodal matrix (node (x, y, l) = (l ny + y) nx + x)."""
    M = M.tocsr()
    n = nx * ny * nl
    ids = np.arange(n)
    x, y, l = ids % nx, (ids // nx) % ny, ids // (nx * ny)

    def off(d, ok):
        w = np.zeros(n)
        w[ok] = -np.asarray(M[ids[ok], ids[ok] + d]).ravel()
        return w.reshape(nl, ny, nx)

    return (off(1, x + 1 < nx), off(nx, y + 1 < ny), off(nx * ny, l + 1 < nl),
            M.diagonal().reshape(nl, ny, nx))


def _solve_blocks(B, coeffs, rhs, world, omega, tol=1e-14, max_sweeps=20000):
    from paper_1409_7166_gb300 import domain
    dev = torch.device("cuda")
    w_e, w_n, w_u, D = (torch.tensor(a, dtype=torch.float64, device=dev) for a in coeffs)
    blocks = domain.split_blocks(w_e, w_n, w_u, 1.0 / D, torch.tensor(rhs, dtype=torch.float64, device=dev),
                                 world)
    stream = torch.cuda.current_stream().cuda_stream

    def half(blk, colour, mx):
        B.pg_block_half_sweep(blk["nx"], blk["rows"], blk["nl"], blk["y0"], blk["w_e"], blk["w_n"], blk["w_u"],
                              blk["inv_d"], blk["rhs"], blk["x"], colour, omega, mx, stream)

    sweeps, est = domain.red_black_sor_blocks(blocks, half, max_sweeps, tol)
    torch.cuda.synchronize()
    for lo, hi in zip(blocks[:-1], blocks[1:]):
        assert torch.equal(lo["x"][:, lo["rows"] + 1], hi["x"][:, 1])
        assert torch.equal(hi["x"][:, 0], lo["x"][:, lo["rows"]])
    return domain.gather_blocks(blocks).cpu().numpy(), sweeps, est


def _check(B, coeffs, rhs, exact, omega, tol_fixed):
    ref, n1, _ = _solve_blocks(B, coeffs, rhs, 1, omega)
    err = float(np.max(np.abs(ref - exact)))
    assert err <= tol_fixed, f"undecomposed fixed point off by {err:.3e}"
    for world in (2, 3):
        got, nw, _ = _solve_blocks(B, coeffs, rhs, world, omega)
        assert nw == n1, f"{world} blocks: {nw} sweeps against {n1}"
        assert np.array_equal(got, ref), f"{world} blocks differ from one block"
    return err, n1


def test_decomposed_sweeps_random_lattice(B):
    """67 x 53 x 3 lattice, random conductances, a positive diagonal excess (C/h plus pads):
    rows split 27 + 26 and 18 + 18 + 17."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    nx, ny, nl = 67, 53, 3
    rng = np.random.default_rng(11)
    gx = rng.uniform(0.5, 2.0, (nl, ny, nx)); gx[:, :, -1] = 0.0
    gy = rng.uniform(0.5, 2.0, (nl, ny, nx)); gy[:, -1, :] = 0.0
    gz = rng.uniform(1.0, 5.0, (nl, ny, nx)); gz[-1] = 0.0
    g0 = rng.uniform(0.2, 0.6, (nl, ny, nx))
    rhs = rng.uniform(-1.0, 1.0, (nl, ny, nx))
    n = nx * ny * nl
    ids = np.arange(n)
    rows, cols, vals = [], [], []
    for d, w in ((1, gx), (nx, gy), (nx * ny, gz)):
        w = w.ravel()
        ok = w > 0
        rows += [ids[ok], ids[ok] + d]; cols += [ids[ok] + d, ids[ok]]; vals += [-w[ok], -w[ok]]
    W = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    M = W + sp.diags(g0.ravel() - np.asarray(W.sum(axis=1)).ravel())
    exact = spla.spsolve(M.tocsc(), rhs.ravel()).reshape(nl, ny, nx)
    err, sweeps = _check(B, _lattice_coefficients(M, nx, ny, nl), rhs, exact, 1.6, 1e-11)
    print(f"random lattice: {sweeps} sweeps, fixed point off by {err:.2e}")


def test_decomposed_sweeps_be_step_of_grid_recipe(B):
    """A backward-Euler system (Eq. 2) of the 3-layer RC recipe at 45 x 38 x 3, assembled
    by the oracle from the element lists: the DC point as the previous step and the loads
    at t = 1.2 ns (mid-switching).  The decomposed relaxation reaches the oracle's direct
    solve."""
    net = pgsynth.config1(nx=45, ny=38)
    nx, ny, nl = net.lattice
    h = net.meta["h"]
    mats = matrices.nodal_matrices(net)
    M = mats.system_matrix(h)
    v0 = transient.dc_operating_point(net, mats)
    t = 240 * h
    rhs = mats.C.diagonal() / h * v0 + transient.source_terms(mats, h) - transient.load_current(net, mats, t)
    exact = transient.DirectSolver(M).solve(rhs)
    err, sweeps = _check(B, _lattice_coefficients(M, nx, ny, nl), rhs.reshape(nl, ny, nx),
                         exact.reshape(nl, ny, nx), 1.9, 1e-3 * TOL_V)
    print(f"BE step of the 3-layer recipe: {sweeps} sweeps, off the oracle by {err:.2e} V")
