"""ctypes binding of ``include/pg.h`` (argument marshalling only).

Every function here forwards to the entry point of the same name in
``_lib/libpg.so``; all computation happens in the library's CUDA kernels.
Device buffers may be PyTorch CUDA tensors (their ``data_ptr()`` is passed);
host buffers are NumPy arrays.  If the library is not built, :func:`lib`
raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

from .build import LIB

PG_GROUND = -1
STATUS = {0: "PG_OK", 1: "PG_ERR_INVALID_ARG", 2: "PG_ERR_FLOATING_NODE", 3: "PG_ERR_OOM",
          4: "PG_ERR_CUDA", 5: "PG_ERR_NOT_CONVERGED", 6: "PG_ERR_TIMEOUT", 7: "PG_ERR_UNSUPPORTED"}
(PG_OK, PG_ERR_INVALID_ARG, PG_ERR_FLOATING_NODE, PG_ERR_OOM, PG_ERR_CUDA, PG_ERR_NOT_CONVERGED,
 PG_ERR_TIMEOUT, PG_ERR_UNSUPPORTED) = range(8)
PG_PREC_FP64, PG_PREC_MIXED = 0, 1
PG_FORM_EXPLICIT, PG_FORM_THREE_LEVEL = 0, 1
PG_COLOUR_AUTO, PG_COLOUR_RED_BLACK, PG_COLOUR_FOUR = 0, 1, 2
PG_DEBUG_SKIP_ARRIVAL = 1

_i32p = C.POINTER(C.c_int32)
_i64p = C.POINTER(C.c_int64)
_f64p = C.POINTER(C.c_double)


class pg_netlist(C.Structure):
    _fields_ = [("n_nodes", C.c_int32), ("n_sources", C.c_int32), ("vdd", _f64p),
                ("n_r", C.c_int64), ("r_a", _i32p), ("r_b", _i32p), ("r_g", _f64p),
                ("n_c", C.c_int64), ("c_a", _i32p), ("c_b", _i32p), ("c_val", _f64p),
                ("n_l", C.c_int64), ("l_a", _i32p), ("l_b", _i32p), ("l_val", _f64p),
                ("n_i", C.c_int64), ("i_a", _i32p), ("i_b", _i32p), ("i_ptr", _i64p),
                ("i_t", _f64p), ("i_v", _f64p),
                ("lat_nx", C.c_int32), ("lat_ny", C.c_int32), ("lat_nl", C.c_int32),
                ("n_lat", C.c_int32), ("lat_desc", _i32p)]


class pg_options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("omega", C.c_double), ("tol", C.c_double),
                ("step_tol", C.c_double), ("max_sweeps", C.c_int32), ("warm_start", C.c_int32),
                ("inner_reduction", C.c_double), ("threads_per_block", C.c_int32),
                ("blocks_per_sm", C.c_int32), ("barrier_timeout_s", C.c_double),
                ("debug_flags", C.c_int32), ("lattice_sweeps", C.c_int32), ("jacobi", C.c_int32),
                ("form", C.c_int32), ("colouring", C.c_int32), ("tile_rows", C.c_int32)]


class pg_row_block(C.Structure):
    _fields_ = [("nx", C.c_int32), ("rows", C.c_int32), ("nl", C.c_int32), ("y0", C.c_int32),
                ("w_e", C.c_void_p), ("w_n", C.c_void_p), ("w_u", C.c_void_p), ("inv_d", C.c_void_p),
                ("rhs", C.c_void_p), ("x", C.c_void_p)]


class pg_scenario_output(C.Structure):
    _fields_ = [("on_host", C.c_int32), ("v_all", C.c_void_p), ("vmin", C.c_void_p)]


class pg_output(C.Structure):
    _fields_ = [("on_host", C.c_int32), ("v_all", C.c_void_p), ("il_all", C.c_void_p),
                ("vmin", C.c_void_p), ("vmin_node", C.c_void_p), ("n_probes", C.c_int32),
                ("probes", C.c_void_p), ("probe_v", C.c_void_p), ("comp_vmin", C.c_void_p)]


class pg_objective(C.Structure):
    _fields_ = [("kind", C.c_int32), ("vref", C.c_double), ("margin", C.c_double)]


class pg_run_stats(C.Structure):
    _fields_ = [("steps_done", C.c_int64), ("total_sweeps", C.c_int64), ("max_sweeps_step", C.c_int32),
                ("max_outer_step", C.c_int32), ("total_outer", C.c_int64), ("max_step_bound", C.c_double),
                ("err_bound", C.c_double), ("failed_step", C.c_int64), ("omega", C.c_double),
                ("rho_jacobi", C.c_double), ("kappa", C.c_double), ("q", C.c_double),
                ("step_tol", C.c_double), ("device_ms", C.c_double), ("kacc", C.c_double),
                ("lattice_sweeps", C.c_int32), ("phase_ms", C.c_double * 4)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["phase_ms"] = list(d["phase_ms"])
        return d


class PGError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        self.name = STATUS.get(status, str(status))
        super().__init__(f"{where}: {self.name}" + (f" ({detail})" if detail else ""))


_LIB = None
EXPORTS = ["pg_default_options", "pg_create_grid", "pg_destroy", "pg_status_str", "pg_last_error",
           "pg_set_stream", "pg_grid_info", "pg_set_state", "pg_get_state", "pg_reset",
           "pg_update_sources", "pg_transient", "pg_step", "pg_solve", "pg_solve_noalloc",
           "pg_update_values", "pg_adjoint"]


def lib(path: Optional[str] = None) -> C.CDLL:
    """Load ``libpg.so`` (raises if it has not been built)."""
    global _LIB
    if _LIB is not None and path is None:
        return _LIB
    p = path or LIB
    if not os.path.exists(p):
        raise RuntimeError(f"CUDA library not built: {p} is missing (run __graft_entry__.build())")
    L = C.CDLL(p)
    vp = C.c_void_p
    L.pg_default_options.argtypes = [C.POINTER(pg_options)]; L.pg_default_options.restype = None
    L.pg_create_grid.argtypes = [C.POINTER(pg_netlist), C.POINTER(pg_options), C.POINTER(vp)]
    L.pg_destroy.argtypes = [vp]; L.pg_destroy.restype = None
    L.pg_status_str.argtypes = [C.c_int]; L.pg_status_str.restype = C.c_char_p
    L.pg_last_error.argtypes = []; L.pg_last_error.restype = C.c_char_p
    L.pg_set_stream.argtypes = [vp, vp]
    L.pg_grid_info.argtypes = [vp, _i32p, _i32p, _i32p, _i32p]
    L.pg_set_state.argtypes = [vp, vp, vp, C.c_int64, C.c_int32]
    L.pg_grid_components.argtypes = [vp, _i32p, vp]
    L.pg_initial_conditions.argtypes = [vp, C.c_double, vp, vp, C.c_int32]
    L.pg_get_state.argtypes = [vp, vp, vp, _i64p, C.c_int32]
    L.pg_reset.argtypes = [vp]
    L.pg_update_sources.argtypes = [vp, vp, vp, C.c_int32]
    L.pg_transient.argtypes = [vp, C.c_double, C.c_int32, C.POINTER(pg_output), C.POINTER(pg_run_stats)]
    L.pg_step.argtypes = [vp, C.c_double, vp, C.POINTER(pg_run_stats)]
    L.pg_solve.argtypes = [vp, C.c_double, vp, vp, C.c_double, C.POINTER(pg_run_stats)]
    L.pg_solve_noalloc.argtypes = [vp, C.c_double, vp, vp, C.c_double, C.POINTER(pg_run_stats)]
    L.pg_update_values.argtypes = [vp, vp, vp, vp, C.c_int32]
    L.pg_adjoint.argtypes = [vp, C.c_double, C.c_int32, C.POINTER(pg_objective), C.c_int32, _f64p, vp, vp, vp,
                             C.c_int32, C.POINTER(pg_run_stats)]
    L.pg_transient_async.argtypes = [vp, C.c_double, C.c_int32, vp, C.POINTER(pg_output), vp]
    L.pg_async_stats.argtypes = [vp, vp, C.POINTER(pg_run_stats)]
    L.pg_autotune.argtypes = [C.POINTER(pg_netlist), C.POINTER(pg_options), C.c_double, C.c_int32, vp,
                              C.POINTER(pg_options), _f64p]
    L.pg_block_half_sweep.argtypes = [C.POINTER(pg_row_block), C.c_int32, C.c_double, vp, vp]
    L.pg_transient_scenarios.argtypes = [vp, C.c_double, C.c_int32, C.c_int32, vp, C.POINTER(pg_scenario_output),
                                         C.POINTER(pg_run_stats)]
    for name in ("pg_create_grid", "pg_set_stream", "pg_grid_info", "pg_set_state", "pg_get_state",
                 "pg_reset", "pg_update_sources", "pg_transient", "pg_step", "pg_solve", "pg_solve_noalloc",
                 "pg_update_values", "pg_adjoint", "pg_transient_async", "pg_async_stats", "pg_autotune", "pg_grid_components",
                 "pg_initial_conditions", "pg_block_half_sweep", "pg_transient_scenarios"):
        getattr(L, name).restype = C.c_int
    if path is None:
        _LIB = L
    return L


def _check(st: int, where: str):
    if st != 0:
        raise PGError(st, where, lib().pg_last_error().decode(errors="replace"))


def _ptr(x):
    """Address of a torch tensor or NumPy array (or None)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return C.c_void_p(x.data_ptr())
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return C.c_void_p(x.ctypes.data)
    raise TypeError(f"unsupported buffer {type(x)}")


def _on_host(*bufs) -> int:
    kinds = {hasattr(b, "data_ptr") and getattr(b, "is_cuda", False) for b in bufs if b is not None}
    if len(kinds) > 1:
        raise ValueError("mix of host and device buffers in one call")
    return 0 if kinds == {True} else 1


# ------------------------------------------------------------------ same-name wrappers

def pg_default_options(**over) -> pg_options:
    o = pg_options()
    lib().pg_default_options(C.byref(o))
    for k, v in over.items():
        setattr(o, k, v)
    return o


def _netlist(net):
    """Marshal a ``pgsynth.Netlist``-like object into a ``pg_netlist`` (plus the arrays it points into)."""
    keep = []

    def arr(a, dt):
        a = np.ascontiguousarray(a, dtype=dt)
        keep.append(a)
        return a.ctypes.data_as({np.int32: _i32p, np.int64: _i64p, np.float64: _f64p}[dt])

    nl = pg_netlist()
    nl.n_nodes = int(net.n_nodes); nl.n_sources = int(len(net.vdd)); nl.vdd = arr(net.vdd, np.float64)
    nl.n_r = len(net.r_g); nl.r_a = arr(net.r_a, np.int32); nl.r_b = arr(net.r_b, np.int32); nl.r_g = arr(net.r_g, np.float64)
    nl.n_c = len(net.c_val); nl.c_a = arr(net.c_a, np.int32); nl.c_b = arr(net.c_b, np.int32); nl.c_val = arr(net.c_val, np.float64)
    nl.n_l = len(net.l_val); nl.l_a = arr(net.l_a, np.int32); nl.l_b = arr(net.l_b, np.int32); nl.l_val = arr(net.l_val, np.float64)
    nl.n_i = len(net.i_a); nl.i_a = arr(net.i_a, np.int32); nl.i_b = arr(net.i_b, np.int32)
    nl.i_ptr = arr(net.i_ptr, np.int64); nl.i_t = arr(net.i_t, np.float64); nl.i_v = arr(net.i_v, np.float64)
    lat = getattr(net, "lattice", None) or (0, 0, 0)
    nl.lat_nx, nl.lat_ny, nl.lat_nl = (int(x) for x in lat)
    lats = getattr(net, "lattices", None)
    if lats:
        nl.n_lat = len(lats)
        nl.lat_desc = arr(np.asarray(lats, dtype=np.int32).reshape(-1), np.int32)
    return nl, keep


def pg_create_grid(net, opt: Optional[pg_options] = None):
    """Create a grid from a ``pgsynth.Netlist``-like object; returns an opaque handle."""
    nl, keep = _netlist(net)
    h = C.c_void_p()
    _check(lib().pg_create_grid(C.byref(nl), C.byref(opt) if opt is not None else None, C.byref(h)),
           "pg_create_grid")
    return h


def pg_destroy(h):
    lib().pg_destroy(h)


def pg_set_stream(h, stream_handle: int):
    _check(lib().pg_set_stream(h, C.c_void_p(stream_handle)), "pg_set_stream")


def pg_grid_info(h):
    n, nl, nc, npad = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
    _check(lib().pg_grid_info(h, C.byref(n), C.byref(nl), C.byref(nc), C.byref(npad)), "pg_grid_info")
    return dict(n_nodes=n.value, n_inductors=nl.value, n_colours=nc.value, n_padded=npad.value)


def pg_grid_components(h, n_nodes: Optional[int] = None):
    """``(n_components, comp_of)``; ``comp_of`` (node -> component) when ``n_nodes`` is given."""
    nc = C.c_int32()
    comp = None if n_nodes is None else np.zeros(int(n_nodes), dtype=np.int32)
    _check(lib().pg_grid_components(h, C.byref(nc), _ptr(comp)), "pg_grid_components")
    return nc.value, comp


def pg_initial_conditions(h, step_h: float, vc0=None, il0=None):
    """Section IV-B initial conditions: the grid's state becomes v(h) at step 1 (v(0) before it)."""
    _check(lib().pg_initial_conditions(h, float(step_h), _ptr(vc0), _ptr(il0), _on_host(vc0, il0)),
           "pg_initial_conditions")


def pg_set_state(h, v, il=None, step: int = 0):
    _check(lib().pg_set_state(h, _ptr(v), _ptr(il), int(step), _on_host(v, il)), "pg_set_state")


def pg_get_state(h, v, il=None):
    s = C.c_int64()
    _check(lib().pg_get_state(h, _ptr(v), _ptr(il), C.byref(s), _on_host(v, il)), "pg_get_state")
    return s.value


def pg_reset(h):
    _check(lib().pg_reset(h), "pg_reset")


def pg_update_sources(h, i_t=None, i_v=None):
    _check(lib().pg_update_sources(h, _ptr(i_t), _ptr(i_v), _on_host(i_t, i_v)), "pg_update_sources")


def pg_transient(h, step_h: float, nsteps: int, v_all=None, il_all=None, vmin=None, vmin_node=None,
                 probes=None, probe_v=None, comp_vmin=None) -> pg_run_stats:
    out = pg_output()
    out.on_host = _on_host(v_all, il_all, vmin, vmin_node, probes, probe_v, comp_vmin)
    out.v_all = _ptr(v_all); out.il_all = _ptr(il_all); out.vmin = _ptr(vmin)
    out.vmin_node = _ptr(vmin_node)
    out.n_probes = 0 if probes is None else int(len(probes))
    out.probes = _ptr(probes); out.probe_v = _ptr(probe_v)
    out.comp_vmin = _ptr(comp_vmin)
    st = pg_run_stats()
    _check(lib().pg_transient(h, float(step_h), int(nsteps), C.byref(out), C.byref(st)), "pg_transient")
    return st


def pg_transient_status(h, step_h: float, nsteps: int) -> tuple:
    """Like :func:`pg_transient` without outputs, returning ``(status, stats)`` instead of raising."""
    st = pg_run_stats()
    rc = lib().pg_transient(h, float(step_h), int(nsteps), None, C.byref(st))
    return rc, st


PG_ASYNC_STATS_BYTES = 128


def pg_transient_async(h, step_h: float, nsteps: int, v0=None, v_all=None, il_all=None, vmin=None,
                       vmin_node=None, comp_vmin=None, dstats=None):
    """Stream-ordered transient from step 0 (capturable into a CUDA graph); device buffers only."""
    for name, b in (("v0", v0), ("v_all", v_all), ("il_all", il_all), ("vmin", vmin),
                    ("vmin_node", vmin_node), ("comp_vmin", comp_vmin), ("dstats", dstats)):
        if b is not None and not (hasattr(b, "data_ptr") and getattr(b, "is_cuda", False)):
            raise TypeError(f"pg_transient_async: {name} must be a CUDA tensor")
    out = pg_output()
    out.on_host = 0
    out.v_all = _ptr(v_all); out.il_all = _ptr(il_all); out.vmin = _ptr(vmin)
    out.vmin_node = _ptr(vmin_node)
    out.comp_vmin = _ptr(comp_vmin)
    _check(lib().pg_transient_async(h, float(step_h), int(nsteps), _ptr(v0), C.byref(out), _ptr(dstats)),
           "pg_transient_async")


def pg_async_stats(h, dstats) -> tuple:
    """``(status, stats)`` of a record written by :func:`pg_transient_async`."""
    st = pg_run_stats()
    rc = lib().pg_async_stats(h, _ptr(dstats), C.byref(st))
    return rc, st


def pg_step(h, step_h: float, v_out=None) -> pg_run_stats:
    st = pg_run_stats()
    _check(lib().pg_step(h, float(step_h), _ptr(v_out), C.byref(st)), "pg_step")
    return st


def pg_solve(h, step_h: float, b, x, tol: float) -> pg_run_stats:
    st = pg_run_stats()
    _check(lib().pg_solve(h, float(step_h), _ptr(b), _ptr(x), float(tol), C.byref(st)), "pg_solve")
    return st


def pg_update_values(h, r_g=None, c_val=None, l_val=None):
    _check(lib().pg_update_values(h, _ptr(r_g), _ptr(c_val), _ptr(l_val), _on_host(r_g, c_val, l_val)),
           "pg_update_values")


def pg_adjoint(h, step_h: float, nsteps: int, vref: float = 1.0, margin: float = 0.05, ckpt_every: int = 50,
               dJ_dG=None, dJ_dC=None, dJ_dL=None):
    """Returns ``(J, stats)``; gradients land in ``dJ_dG`` / ``dJ_dC`` / ``dJ_dL`` (netlist order)."""
    obj = pg_objective(0, float(vref), float(margin))
    J = C.c_double()
    st = pg_run_stats()
    _check(lib().pg_adjoint(h, float(step_h), int(nsteps), C.byref(obj), int(ckpt_every), C.byref(J),
                            _ptr(dJ_dG), _ptr(dJ_dC), _ptr(dJ_dL), _on_host(dJ_dG, dJ_dC, dJ_dL), C.byref(st)),
           "pg_adjoint")
    return J.value, st


def pg_solve_noalloc(h, step_h: float, b, x, tol: float) -> pg_run_stats:
    """pg_solve without device allocations (fixed 32 MiB scratch inside the library)."""
    st = pg_run_stats()
    _check(lib().pg_solve_noalloc(h, float(step_h), _ptr(b), _ptr(x), float(tol), C.byref(st)),
           "pg_solve_noalloc")
    return st


def pg_autotune(net, step_h: float, trial_steps: int, stream=None, **base):
    """Fastest options for ``net`` by timed trials; returns ``(pg_options, trial_ms)``."""
    nl, keep = _netlist(net)
    b = pg_default_options(**base)
    best = pg_options()
    ms = C.c_double()
    _check(lib().pg_autotune(C.byref(nl), C.byref(b), float(step_h), int(trial_steps),
                             None if stream is None else C.c_void_p(stream), C.byref(best), C.byref(ms)),
           "pg_autotune")
    del keep
    return best, ms.value


def options_dict(o: pg_options) -> dict:
    """The fields of a ``pg_options`` as keyword arguments for :class:`Grid`."""
    return {name: getattr(o, name) for name, _ in o._fields_}


class Grid:
    """Owning wrapper around a ``pg_grid`` handle (still argument marshalling only)."""

    def __init__(self, net, **options):
        self.net = net
        self.handle = pg_create_grid(net, pg_default_options(**options))
        self.info = pg_grid_info(self.handle)

    def close(self):
        if self.handle is not None:
            pg_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def pg_block_half_sweep(nx: int, rows: int, nl: int, y0: int, w_e, w_n, w_u, inv_d, rhs, x, colour: int,
                        omega: float, max_update, stream: int = 0) -> None:
    """One colour half-sweep over a row block (device FP64 tensors, see ``pg_row_block``);
    ``max_update`` is a device float64 scalar the caller zeroes (max-merged)."""
    for name, t in (("w_e", w_e), ("w_n", w_n), ("w_u", w_u), ("inv_d", inv_d), ("rhs", rhs), ("x", x),
                    ("max_update", max_update)):
        if not (hasattr(t, "is_cuda") and t.is_cuda and t.is_contiguous()):
            raise TypeError(f"pg_block_half_sweep: {name} must be a contiguous CUDA tensor")
    blk = pg_row_block(int(nx), int(rows), int(nl), int(y0), _ptr(w_e), _ptr(w_n), _ptr(w_u), _ptr(inv_d),
                       _ptr(rhs), _ptr(x))
    _check(lib().pg_block_half_sweep(C.byref(blk), int(colour), float(omega), _ptr(max_update),
                                     C.c_void_p(stream)), "pg_block_half_sweep")


def pg_transient_scenarios(h, step_h: float, nsteps: int, i_v, v_all=None, vmin=None) -> pg_run_stats:
    """``i_v``: ``[n_scen, n_points]`` PWL breakpoint values of each scenario (host or
    device); outputs ``v_all`` ``[nsteps, n_scen, n_nodes]`` and ``vmin`` ``[nsteps, n_scen]``."""
    n_scen = int(i_v.shape[0])
    out = pg_scenario_output()
    out.on_host = _on_host(v_all, vmin)
    out.v_all = _ptr(v_all); out.vmin = _ptr(vmin)
    st = pg_run_stats()
    _check(lib().pg_transient_scenarios(h, float(step_h), int(nsteps), n_scen, _ptr(i_v), C.byref(out), C.byref(st)),
           "pg_transient_scenarios")
    return st
