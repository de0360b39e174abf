"""Laplace-variable quadrature meshes (oracle; test infrastructure only).

Sec. II, Eqs. 5-7: 1/p^2 = int_0^inf exp(-alpha p^2) d alpha, split at alpha_c.
Eqs. 11-13: on [alpha_c, inf) substitute t = alpha^{-1/2}; then d alpha = -2 t^{-3} dt and
    int_{alpha_c}^inf F(alpha) d alpha = int_0^{alpha_c^{-1/2}} F(1/t^2) (2 / t^3) dt,
so a Gauss-Legendre point (t_i, w_2i) on the t interval becomes the node alpha_i = 1/t_i^2
with weight Omega_i = 2 w_2i / t_i^3.  (The printed Eq. 13 weight, 1/2 w alpha^{3/2} t^{2n},
is garbled: the t^{2n} belongs to the asymptotic series and cancels, and the Jacobian of
t = alpha^{-1/2} is 2/t^3.)  Eq. 14 is the resulting single node sum over both intervals.
Table I discussion: "Mesh 1" is Q points on [0, alpha_c] plus Q tail points; "Mesh 2"
splits [0, alpha_c] at alpha_c 5^{-7}, ..., alpha_c 5^{-1} into eight sub-intervals.
Generalised here to n_sub geometric split points (n_sub + 1 sub-intervals).

Gauss-Legendre points come from numpy.polynomial.legendre.leggauss (a library routine
that serves as one step; the paper defers to standard references for them).
"""
from functools import lru_cache

import numpy as np
from numpy.polynomial.legendre import leggauss


@lru_cache(maxsize=64)
def _reference_rule(q: int):
    x, w = leggauss(q)
    x.setflags(write=False)
    w.setflags(write=False)
    return x, w


def gauss_legendre(q: int, a: float, b: float):
    """q-point Gauss-Legendre nodes and weights on [a, b], ascending."""
    x, w = _reference_rule(q)
    return 0.5 * (b - a) * x + 0.5 * (b + a), 0.5 * (b - a) * w


def interval1_edges(n_sub: int, alpha_c: float = 1.0, ratio: float = 5.0):
    """Edges of the sub-intervals of [0, alpha_c]: 0, alpha_c ratio^-n_sub, ...,
    alpha_c/ratio, alpha_c (the paper's Mesh 2: ratio 5)."""
    if n_sub == 0:
        return [0.0, alpha_c]
    return [0.0] + [alpha_c * ratio ** (-k) for k in range(n_sub, 0, -1)] + [alpha_c]


def interval1_counts(S: int, n_sub: int, q_tail: int):
    """Points per sub-interval: floor((S - q_tail)/(n_sub + 1)) each, one more for the
    first (S - q_tail) mod (n_sub + 1) sub-intervals (the paper uses equal counts)."""
    n = S - q_tail
    k = n_sub + 1
    return [n // k + (1 if i < n % k else 0) for i in range(k)]


def laplace_mesh(S: int, n_sub: int, q_tail: int, alpha_c: float = 1.0, ratio: float = 5.0):
    """Nodes and weights with int_0^inf F(alpha) d alpha ~= sum_s w_s F(alpha_s).

    Returns (alpha[S], w[S], part[S]); part is 0 on interval 1 ([0, alpha_c]) and 1 on the
    tail.  Order: sub-intervals ascending, nodes ascending inside each, then the tail
    in ascending t.
    """
    edges = interval1_edges(n_sub, alpha_c, ratio)
    counts = interval1_counts(S, n_sub, q_tail)
    al, wl, pl = [], [], []
    for i, q in enumerate(counts):
        if q <= 0:
            continue
        x, w = gauss_legendre(q, edges[i], edges[i + 1])
        al.append(x)
        wl.append(w)
        pl.append(np.zeros(q, dtype=np.int64))
    if q_tail > 0:
        t, wt = gauss_legendre(q_tail, 0.0, alpha_c ** -0.5)   # Eq. 11: t in (0, alpha_c^-1/2]
        al.append(1.0 / t ** 2)                                # Eq. 13: alpha_i = 1/t_i^2
        wl.append(2.0 * wt / t ** 3)                           # Jacobian of t = alpha^-1/2
        pl.append(np.ones(q_tail, dtype=np.int64))
    return np.concatenate(al), np.concatenate(wl), np.concatenate(pl)


def paper_mesh1(Q: int):
    """Table I "Mesh 1": Q points on [0, 1] and Q tail points (2Q nodes, Eq. 14)."""
    return laplace_mesh(2 * Q, 0, Q, 1.0)


def paper_mesh2(q: int, q_tail: int = 90):
    """Table I "Mesh 2": eight geometric sub-intervals of [0, 1] with q points each, plus
    the tail.  The paper does not state the tail order; any q_tail >= 5 gives the same
    six printed digits, 90 is used."""
    return laplace_mesh(8 * q + q_tail, 7, q_tail, 1.0)


def tune_points(R: int):
    """The |n|^2 values a mesh is judged on: m_k = 1 + floor((12 R^2 - 1) k^3 / 95^3),
    k = 0..95 (dense near m = 1, reaching the largest |n|^2 of the (2R+1)^3 grid)."""
    top = 12 * R * R - 1
    return np.unique(np.array([1 + (top * k ** 3) // 857375 for k in range(96)], dtype=np.int64))


def mesh_error(S: int, n_sub: int, q_tail: int, R: int, alpha_c: float = 1.0,
               ratio: float = 5.0) -> float:
    """max_m |sum_s w_s exp(-a_s m) - 1/m| * m over tune_points(R) (relative error of the
    node sum of 1/m; the Laplace form of the periodic kernel in index units)."""
    a, w, _ = laplace_mesh(S, n_sub, q_tail, alpha_c, ratio)
    m = tune_points(R).astype(np.float64)
    return float(np.max(np.abs(np.exp(-np.outer(m, a)) @ w - 1.0 / m) * m))


def default_periodic_mesh(S: int, R: int):
    """(n_sub, q_tail) of the periodic kernel for S nodes at cutoff R.

    Explicit choices for the four single-box workloads (S, R) = (32, 4), (64, 13),
    (96, 31), (128, 63).  Otherwise a small search (the paper's remark that the split
    of the Laplace integral decides how many points are needed, Sec. II): with
    r = max(1, floor(log5(12 R^2)) - 1), every n_sub in {r, r + 1} and q_tail in
    3 .. max(3, round(0.45 S)) with S - q_tail >= n_sub + 1, the pair with the smallest
    mesh_error (floored at 1e-10, where FP64 rounding noise starts to decide) wins; candidates are visited n_sub ascending, then q_tail ascending, and
    replace the best only when smaller by more than 0.1 % relative (errors on a plateau
    differ in their last digits between implementations; the margin keeps the choice
    reproducible).
    """
    table = {(32, 4): (2, 10), (64, 13): (3, 21), (96, 31): (4, 29), (128, 63): (5, 34)}
    if (S, R) in table:
        return table[(S, R)]
    r = max(1, int(np.floor(np.log(12.0 * R * R) / np.log(5.0))) - 1)
    # (fewer than 5 nodes leave no candidate: one interval plus a tail of S // 2)
    best, arg = None, None
    for n_sub in (r, r + 1):
        for q_tail in range(3, max(3, int(np.rint(0.45 * S))) + 1):
            if S - q_tail < n_sub + 1:
                continue
            e = max(mesh_error(S, n_sub, q_tail, R), 1e-10)   # below: rounding noise
            if best is None or e < best * (1.0 - 1e-3):
                best, arg = e, (n_sub, q_tail)
    if arg is None:  # fewer than 5 nodes: one interval and a tail of half the nodes
        return 0, max(1, S // 2)
    return arg


def mesh_for_error(R: int, target: float, S_max: int):
    """The fewest nodes S in 2 .. S_max whose default mesh reaches mesh_error <= target
    (the node count as a function of the accuracy wanted, Sec. II): (S, n_sub, q_tail,
    error), or None when no S up to S_max does."""
    for S in range(2, S_max + 1):
        n_sub, q_tail = default_periodic_mesh(S, R)
        e = mesh_error(S, n_sub, q_tail, R)
        if e <= target:
            return S, n_sub, q_tail, e
    return None


TUNE_RATIOS = (3.0, 4.0, 5.0, 6.0, 8.0)
TUNE_ALPHAS = (0.5, 1.0, 2.0)


def mesh_tune(R: int, target: float, S_max: int):
    """The fewest nodes over a wider mesh family that reach mesh_error <= target (Sec. II:
    the split point alpha_c and the sub-intervals decide how many nodes the accuracy needs;
    the paper fixes alpha_c = 1 and leaves a better choice open).  Candidates: sub-interval
    ratio in TUNE_RATIOS, alpha_c in TUNE_ALPHAS, n_sub in {r, r + 1} with
    r = max(1, floor(log_ratio(12 R^2)) - 1), q_tail in 3 .. max(3, round(0.45 S)) with
    S - q_tail >= n_sub + 1, for S from max(2, floor(0.8 S_d)) to S_d, S_d the count of
    mesh_for_error.  The first S whose best candidate (smallest error floored at 1e-10,
    replaced only when smaller by more than 0.1 %, visited ratio, alpha_c, n_sub, q_tail
    ascending) reaches the target wins.  Returns (S, n_sub, q_tail, alpha_c, ratio, error)
    or None."""
    d = mesh_for_error(R, target, S_max)
    if d is None:
        return None
    Sd = d[0]
    m = 12.0 * R * R
    for S in range(max(2, int(0.8 * Sd)), Sd + 1):
        best = None
        for ratio in TUNE_RATIOS:
            r = max(1, int(np.floor(np.log(m) / np.log(ratio))) - 1)
            for ac in TUNE_ALPHAS:
                for n_sub in (r, r + 1):
                    for q_tail in range(3, max(3, int(np.rint(0.45 * S))) + 1):
                        if S - q_tail < n_sub + 1:
                            continue
                        raw = mesh_error(S, n_sub, q_tail, R, ac, ratio)
                        e = max(raw, 1e-10)
                        if best is None or e < best[0] * (1.0 - 1e-3):
                            best = (e, raw, n_sub, q_tail, ac, ratio)
        if best is not None and best[1] <= target:
            return S, best[2], best[3], best[4], best[5], best[1]
    return d[0], d[1], d[2], 1.0, 5.0, d[3]


def prune_periodic(alpha_idx, w, R: int, tol: float):
    """Keep-mask of nodes for the periodic kernel in index units.

    Node s adds w_s exp(-a_s m) to 1/m for an integer m = |n|^2 >= 1; it is dropped when
    even its largest contribution (m = 1) is below tol times the smallest value in range,
    1/(12 R^2): w_s exp(-a_s) < tol / (12 R^2).  tol <= 0 keeps every node.
    """
    if tol <= 0:
        return np.ones(len(w), dtype=bool)
    return w * np.exp(-alpha_idx) >= tol / (12.0 * R * R)
