"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every entry point ``include/pg.h`` declares, and rejects netlists that break
the paper's topological assumptions (Section III-B) before touching CUDA."""
import os
import re
import subprocess

import numpy as np
import pytest

import pgsynth
from pgsynth import GROUND, make_netlist, source_terminal as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def B():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1409_7166_gb300 import binding
    return binding


def declared_functions():
    src = open(os.path.join(ROOT, "include", "pg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pg_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol(B):
    lib = B.lib()
    names = declared_functions()
    assert len(names) >= 14
    for name in names:
        assert hasattr(lib, name), f"libpg.so does not export {name}"
    nm = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (pg_\w+)", nm))
    assert set(names) <= exported
    assert set(B.EXPORTS) <= exported


def test_default_options_and_status_names(B):
    o = B.pg_default_options()
    assert (o.precision, o.tol, o.max_sweeps, o.warm_start, o.threads_per_block) == (0, 1e-6, 20000, -1, 256)
    for code, name in B.STATUS.items():
        assert B.lib().pg_status_str(code).decode() == name


def _create_status(B, net, **opt):
    try:
        h = B.pg_create_grid(net, B.pg_default_options(**opt))
    except B.PGError as e:
        return e.name
    B.pg_destroy(h)
    return "PG_OK"


def test_validation_rejects_bad_netlists(B):
    good = make_netlist(2, [1.0], R=[(0, S(0), 1.0), (0, 1, 2.0)], C=[(1, GROUND, 1e-15)])
    bad_index = make_netlist(2, [1.0], R=[(0, S(0), 1.0), (0, 5, 2.0)])
    bad_source = make_netlist(2, [1.0], R=[(0, S(3), 1.0), (0, 1, 2.0)])
    neg_g = make_netlist(2, [1.0], R=[(0, S(0), 1.0), (0, 1, -2.0)])
    self_loop = make_netlist(2, [1.0], R=[(0, S(0), 1.0), (1, 1, 2.0), (0, 1, 1.0)])
    pwl_back = make_netlist(2, [1.0], R=[(0, S(0), 1.0), (0, 1, 2.0)],
                            I=[(1, GROUND, [2.0, 1.0], [0.0, 1.0])])
    assert _create_status(B, bad_index) == "PG_ERR_INVALID_ARG"
    assert _create_status(B, bad_source) == "PG_ERR_INVALID_ARG"
    assert _create_status(B, neg_g) == "PG_ERR_INVALID_ARG"
    assert _create_status(B, self_loop) == "PG_ERR_INVALID_ARG"
    assert _create_status(B, pwl_back) == "PG_ERR_INVALID_ARG"
    assert _create_status(B, good, omega=2.0) == "PG_ERR_INVALID_ARG"      # Eq. 17 needs 0 < w < 2
    assert _create_status(B, good, precision=7) == "PG_ERR_INVALID_ARG"


def test_validation_topological_assumptions(B):
    # assumption 2: a node whose only branch is a current source
    only_isrc = make_netlist(2, [1.0], R=[(0, S(0), 1.0)], I=[(1, GROUND, [0.0], [1e-3])])
    assert _create_status(B, only_isrc) == "PG_ERR_FLOATING_NODE"
    # assumption 3 / Fig. 1: a sub-circuit with no path to a source or ground
    floating = make_netlist(4, [1.0], R=[(0, S(0), 1.0), (0, 1, 2.0), (2, 3, 1.0)],
                            C=[(2, GROUND, 1e-15)])
    assert _create_status(B, floating) == "PG_ERR_FLOATING_NODE"
    # node-to-node capacitors are outside the per-node form of Eq. 12
    coupling = make_netlist(2, [1.0], R=[(0, S(0), 1.0), (0, 1, 2.0)], C=[(0, 1, 1e-15)])
    assert _create_status(B, coupling) == "PG_ERR_UNSUPPORTED"


def test_valid_netlist_reaches_cuda(B):
    """A valid netlist passes validation; without a GPU the first CUDA call fails
    with PG_ERR_CUDA (there is no CPU fallback)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present: covered by the GPU tests")
    net = pgsynth.config0(nx=8, ny=8)
    assert _create_status(B, net) == "PG_ERR_CUDA"


def test_jacobi_option_validation():
    """Damped Jacobi accepts jacobi in {0, 1} and omega <= 1 only; checked on the
    host before any device work."""
    from paper_1409_7166_gb300 import binding as B
    net = pgsynth.config0(nx=6, ny=5)
    for bad in (dict(jacobi=2), dict(jacobi=1, omega=1.5)):
        with pytest.raises(B.PGError) as ei:
            B.pg_create_grid(net, B.pg_default_options(**bad))
        assert ei.value.status == B.PG_ERR_INVALID_ARG


def test_degenerate_netlists(B):
    """An empty netlist is invalid; a sub-circuit with no source at all, or a node
    held only by a capacitor, has no DC point (Lemma 1 needs a strictly dominant row
    in DC) and is rejected as floating."""
    assert _create_status(B, make_netlist(0, [1.0])) == "PG_ERR_INVALID_ARG"
    no_source = make_netlist(2, [], R=[(0, 1, 1.0)], C=[(0, GROUND, 1e-15), (1, GROUND, 1e-15)])
    assert _create_status(B, no_source) == "PG_ERR_FLOATING_NODE"
    cap_only = make_netlist(1, [1.0], C=[(0, GROUND, 1e-15)])
    assert _create_status(B, cap_only) == "PG_ERR_FLOATING_NODE"


def test_warm_start_option_validation():
    """warm_start takes -1 (automatic), 0 (previous value), 1 (linear extrapolation) or 2
    (load-aware damped extrapolation); anything else is rejected before any device work."""
    from paper_1409_7166_gb300 import binding as B
    net = pgsynth.config0(nx=6, ny=5)
    for bad in (-2, 3):
        with pytest.raises(B.PGError) as ei:
            B.pg_create_grid(net, B.pg_default_options(warm_start=bad))
        assert ei.value.status == B.PG_ERR_INVALID_ARG



def test_colouring_and_tile_rows_validation():
    """colouring takes PG_COLOUR_AUTO, _RED_BLACK or _FOUR and tile_rows 0, 34 or 66;
    anything else is rejected before any device work."""
    from paper_1409_7166_gb300 import binding as B
    net = pgsynth.config0(nx=6, ny=5)
    for bad in (dict(colouring=-1), dict(colouring=3), dict(tile_rows=33), dict(tile_rows=-34)):
        with pytest.raises(B.PGError) as ei:
            B.pg_create_grid(net, B.pg_default_options(**bad))
        assert ei.value.status == B.PG_ERR_INVALID_ARG
    o = B.pg_default_options()
    assert (o.colouring, o.tile_rows) == (B.PG_COLOUR_AUTO, 0)


def test_block_half_sweep_and_scenarios_validate_arguments():
    """pg_block_half_sweep refuses null arrays, empty blocks, colours other than 0 and 1 and
    omega outside (0, 2), and pg_transient_scenarios a null grid or no steps, all before
    touching the device (status PG_ERR_INVALID_ARG)."""
    import ctypes as C
    from paper_1409_7166_gb300 import binding as B
    L = B.lib()
    blk = B.pg_row_block()
    mx = C.c_double(0.0)
    assert L.pg_block_half_sweep(C.byref(blk), 0, 1.5, C.byref(mx), None) == B.PG_ERR_INVALID_ARG
    buf = (C.c_double * 64)()
    ptr = C.cast(buf, C.c_void_p)
    blk = B.pg_row_block(4, 2, 1, 0, ptr, ptr, ptr, ptr, ptr, ptr)
    for colour, omega in ((2, 1.5), (-1, 1.5), (0, 0.0), (1, 2.0)):
        assert L.pg_block_half_sweep(C.byref(blk), colour, omega, C.byref(mx), None) == B.PG_ERR_INVALID_ARG
    empty = B.pg_row_block(4, 0, 1, 0, ptr, ptr, ptr, ptr, ptr, ptr)
    assert L.pg_block_half_sweep(C.byref(empty), 0, 1.5, C.byref(mx), None) == B.PG_ERR_INVALID_ARG
    st = B.pg_run_stats()
    assert L.pg_transient_scenarios(None, 1e-12, 10, 2, ptr, None, C.byref(st)) == B.PG_ERR_INVALID_ARG
