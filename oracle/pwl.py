"""Piecewise-linear current sources (the I_s of Eq. 8, Section II-A).

The paper models gate currents as piecewise-linear ideal current sources.
Semantics used on both sides of the parity tests:

* ``t <= t_0``               -> ``v_0``
* ``t >  t_{K-1}``           -> ``v_{K-1}``
* otherwise, on the first segment with ``t_k < t <= t_{k+1}``:
  ``v_k + (v_{k+1} - v_k) * ((t - t_k) / (t_{k+1} - t_k))``

Breakpoint times must be non-decreasing.
"""
from __future__ import annotations

import numpy as np


def pwl_values(i_ptr: np.ndarray, i_t: np.ndarray, i_v: np.ndarray, t: float) -> np.ndarray:
    """Value of every current source at time ``t`` (vectorised over sources)."""
    i_ptr = np.asarray(i_ptr, dtype=np.int64)
    m = i_ptr.size - 1
    out = np.zeros(m)
    if m == 0:
        return out
    first = i_ptr[:-1]
    last = i_ptr[1:] - 1
    npts = last - first + 1
    out[:] = i_v[first]                      # t <= t_0 (and single-point sources)
    after = t > i_t[last]
    out[after] = i_v[last[after]]
    done = (t <= i_t[first]) | after
    for k in range(int(npts.max()) - 1):
        has = (npts > k + 1) & ~done
        if not has.any():
            break
        j = first[has] + k
        t0, t1 = i_t[j], i_t[j + 1]
        hit = (t0 < t) & (t <= t1)
        if hit.any():
            idx = np.nonzero(has)[0][hit]
            jj = j[hit]
            out[idx] = i_v[jj] + (i_v[jj + 1] - i_v[jj]) * ((t - i_t[jj]) / (i_t[jj + 1] - i_t[jj]))
            done[idx] = True
    return out


def pwl_scalar(ts, vs, t: float) -> float:
    """Single-source version written as a plain loop (used to pin the vectorised one)."""
    if t <= ts[0]:
        return float(vs[0])
    for k in range(len(ts) - 1):
        if ts[k] < t <= ts[k + 1]:
            return float(vs[k] + (vs[k + 1] - vs[k]) * ((t - ts[k]) / (ts[k + 1] - ts[k])))
    return float(vs[-1])
