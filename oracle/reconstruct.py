"""Batch reconstruction of (IJ|KL) with momentum-conservation bookkeeping (oracle).

Sec. II, Eq. 14 evaluated for a list of quadruples; Sec. I (abstract) and Sec. III: for
planewaves only quadruples with n_J - n_I + n_L - n_K = 0 are nonzero ("due to closure").
Bookkeeping order for each quadruple, with the three counters it feeds:
  1. any id outside [0, Nb) (id form) or any vector with |n|^2 > R^2 (vector form):
     value 0, counter[2] += 1;
  2. otherwise, not momentum conserving: value 0, counter[0] += 1;
  3. otherwise q = n_J - n_I; periodic kernel with q = 0 (the excluded G = 0 term):
     value 0, counter[1] += 1;
  4. otherwise the value V(q) (exact, node sum, or box node sum).
"""
import numpy as np

from .basis import basis
from .coulomb import V_exact, V_separable, V_box_separable


def decode(quads, R: int, fmt: str = "ids"):
    """Return (vectors int64[n, 4, 3], in_range bool[n]) for id or int8x4 quadruples."""
    B = basis(R)
    quads = np.asarray(quads)
    n = quads.shape[0]
    if fmt == "ids":
        ids = quads.astype(np.int64).reshape(n, 4)
        ok = np.all((ids >= 0) & (ids < len(B)), axis=1)
        v = np.zeros((n, 4, 3), dtype=np.int64)
        v[ok] = B[ids[ok]]
        return v, ok
    v = quads.astype(np.int64).reshape(n, 4, 4)[:, :, :3]
    ok = np.all((v * v).sum(axis=2) <= R * R, axis=1)
    return v, ok


def reconstruct(quads, R: int, L: float, value: str = "exact", fmt: str = "ids",
                a=None, w=None, box_table=None):
    """Values float64[n] and counters int64[3] for a batch of quadruples.

    value: 'exact'     -> 1/(pi L |q|^2);
           'separable' -> Eq. 14 node sum of the periodic kernel with nodes (a, w);
           'box'       -> Eq. 14 node sum of the box kernel with nodes (a, w) and the
                          per-axis table box_table[s, |D|].
    """
    v, ok = decode(quads, R, fmt)
    q = v[:, 1] - v[:, 0]
    cons = np.all(q + v[:, 3] - v[:, 2] == 0, axis=1)
    q0 = np.all(q == 0, axis=1)
    counters = np.zeros(3, dtype=np.int64)
    counters[2] = int((~ok).sum())
    counters[0] = int((ok & ~cons).sum())
    live = ok & cons
    if value != "box":
        counters[1] = int((live & q0).sum())
        live = live & ~q0
    out = np.zeros(len(q))
    if value == "exact":
        out[live] = V_exact(q[live], L)
    elif value == "separable":
        out[live] = V_separable(q[live], L, a, w)
    elif value == "box":
        out[live] = V_box_separable(q[live], a, w, L, box_table)
    else:
        raise ValueError(value)
    return out, counters


def pair_matrix(R: int, L: float, rows=None, value: str = "exact", a=None, w=None,
                box_table=None):
    """V(n_j - n_i) for rows i (default all) and every column j of basis(R)."""
    B = basis(R)
    ri = np.arange(len(B)) if rows is None else np.asarray(rows)
    d = B[None, :, :] - B[ri][:, None, :]
    if value == "exact":
        return V_exact(d, L)
    if value == "separable":
        return V_separable(d, L, a, w)
    return V_box_separable(d, a, w, L, box_table)
