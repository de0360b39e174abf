"""Exact exchange of the uniform electron gas in a cubic box (oracle; test infrastructure).

Sec. III: M electrons of each spin occupy every planewave inside a Fermi sphere at a
shell closing; the exchange energy per spin channel is
    E_x^sigma = -1/2 sum_{i, j in F} (ij|ji),
and the Kohn-Sham (local density) value it approaches for large M is
    E_KS = -(3/4) (6/pi)^{1/3} M^{4/3} / L          (per spin channel, Sec. III).
With (ij|ji) = V(n_j - n_i) (Eq. 2 reading in coulomb.py) the exchange potential of a
basis function k is eps(k) = -sum_{j in F, n_j != k} V(k - n_j) for the periodic kernel
(the q = 0 term excluded) and -sum_{j in F} V_box(k - n_j) for the box kernel (j = k
included, V_box(0) is finite), and E_x^sigma = 1/2 sum_{i in F} eps(n_i).
Sec. III also states E_x = beta(M, {q_k}) / L: E_x L does not depend on L.
"""
import numpy as np

from .basis import basis, occupied
from .coulomb import (BOX_GL_POINTS, V_exact, V_separable, V_box_separable, box_table,
                      V_of_m_separable)


def E_KS(M: int, L: float) -> float:
    """Kohn-Sham exchange of M electrons per spin in a cube of side L (Sec. III)."""
    return -0.75 * (6.0 / np.pi) ** (1.0 / 3.0) * M ** (4.0 / 3.0) / L


def r_s(M: int, L: float) -> float:
    """Wigner-Seitz radius of 2M electrons in L^3: (4 pi / 3) r_s^3 = L^3 / (2 M)."""
    return (3.0 * L ** 3 / (8.0 * np.pi * M)) ** (1.0 / 3.0)


def _pairs(R, R_F, k_idx, chunk, value_of_diff):
    k = basis(R)
    if k_idx is not None:
        k = k[np.asarray(k_idx)]
    F = occupied(R_F)
    out = np.empty(len(k))
    for s in range(0, len(k), chunk):
        d = k[s:s + chunk, None, :] - F[None, :, :]
        out[s:s + chunk] = -value_of_diff(d).sum(axis=1)
    return out


def eps_exact(R: int, R_F: int, L: float, k_idx=None, chunk: int = 256):
    """eps(k) = -sum_{j in F, n_j != k} 1/(pi L |k - n_j|^2) for basis functions k
    (all of basis(R), or the rows k_idx of it)."""
    return _pairs(R, R_F, k_idx, chunk, lambda d: V_exact(d, L))


def eps_separable(R: int, R_F: int, L: float, a, w, k_idx=None, chunk: int = 256):
    """Same sum with V replaced by its Eq. 14 node sum (j = k still excluded).  The node
    sum is evaluated once for every integer m = |k - n_j|^2 that can occur and indexed."""
    m_all = np.arange((R + R_F) ** 2 * 3 + 1)
    Vm = V_of_m_separable(m_all, L, a, w)

    def val(d):
        return Vm[(d * d).sum(axis=-1)]
    return _pairs(R, R_F, k_idx, chunk, val)


def eps_box(R: int, R_F: int, L: float, alpha, omega, k_idx=None, chunk: int = 64,
            points: int = BOX_GL_POINTS):
    """eps(k) = -sum_{j in F} V_box(k - n_j), node-sum form of the box kernel (`points`
    Gauss-Legendre points per axis integral of the table)."""
    table = box_table(alpha, R + R_F, L, points)
    return _pairs(R, R_F, k_idx, chunk, lambda d: V_box_separable(d, alpha, omega, L, table))


def eps_separable_grid(R: int, R_F: int, L: float, a, w) -> np.ndarray:
    """eps_separable on the whole (2R+1)^3 grid, as a 3D linear convolution: eps = -(O * V)
    with O the 0/1 Fermi-sphere occupation on [-R_F, R_F]^3 and V(n) the node sum of
    V_of_m_separable at m = |n|^2 on [-(R + R_F), R + R_F]^3 (V(0) = 0, the excluded j = k
    term).  The convolution is taken with an FP64 FFT (a library routine serving as one step)
    and the cube [-R, R]^3 of the full result is returned, 0 outside the basis sphere.
    Same values as eps_separable up to the FFT's rounding (about 1e-14 relative: every term
    is positive)."""
    G = 2 * R_F + 1
    rv = np.arange(-(R + R_F), R + R_F + 1)
    m = rv[:, None, None] ** 2 + rv[None, :, None] ** 2 + rv[None, None, :] ** 2
    V = V_of_m_separable(np.arange(int(m.max()) + 1), L, a, w)[m]
    r = np.arange(-R_F, R_F + 1)
    occ = ((r[:, None, None] ** 2 + r[None, :, None] ** 2 + r[None, None, :] ** 2)
           <= R_F * R_F).astype(np.float64)
    n = V.shape[0] + G - 1
    ax = (0, 1, 2)
    full = np.fft.irfftn(np.fft.rfftn(V, s=(n, n, n), axes=ax) *
                         np.fft.rfftn(occ, s=(n, n, n), axes=ax), s=(n, n, n), axes=ax)
    # full[i] = sum_j occ[j] V[i - j]; output index i <-> k = i - (R + R_F) - R_F
    lo = R_F + R_F
    sub = -full[lo:lo + 2 * R + 1, lo:lo + 2 * R + 1, lo:lo + 2 * R + 1]
    k = np.arange(-R, R + 1)
    inside = (k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2) <= R * R
    return np.where(inside, sub, 0.0)


def eps_on_grid(R: int, values) -> np.ndarray:
    """Place per-basis values on the (2R+1)^3 cube grid (0 outside the basis sphere)."""
    G = 2 * R + 1
    grid = np.zeros((G, G, G))
    k = basis(R) + R
    grid[k[:, 0], k[:, 1], k[:, 2]] = values
    return grid


def difference_histogram(R_F: int, method: str = "direct") -> np.ndarray:
    """C(n) = #{(i, j) in F x F : n_i - n_j = n} on [-2 R_F, 2 R_F]^3 (int64).

    'direct' adds the shifted occupation cube once per occupied point (exact integers);
    'fft' takes the FFT autocorrelation of the occupation cube and rounds to the nearest
    integer, then checks sum C = M^2 and C(0) = M.
    """
    G = 2 * R_F + 1
    H = 2 * G - 1
    r = np.arange(-R_F, R_F + 1)
    occ = ((r[:, None, None] ** 2 + r[None, :, None] ** 2 + r[None, None, :] ** 2)
           <= R_F * R_F).astype(np.int64)
    M = int(occ.sum())
    if method == "direct":
        C = np.zeros((H, H, H), dtype=np.int64)
        for p in np.argwhere(occ):
            # n_i = a, n_j = p: difference index a - p + (G - 1)
            C[G - 1 - p[0]:2 * G - 1 - p[0], G - 1 - p[1]:2 * G - 1 - p[1],
              G - 1 - p[2]:2 * G - 1 - p[2]] += occ
    else:
        f = np.fft.rfftn(occ.astype(np.float64), s=(H, H, H), axes=(0, 1, 2))
        full = np.fft.irfftn(f * np.conj(f), s=(H, H, H), axes=(0, 1, 2))
        C = np.rint(np.fft.fftshift(full)).astype(np.int64)
        if int(C.sum()) != M * M or int(C[G - 1, G - 1, G - 1]) != M:
            raise ArithmeticError("FFT autocorrelation failed its integer checks")
    return C


def _hist_vectors(C):
    H = C.shape[0]
    c = (H - 1) // 2
    r = np.arange(-c, c + 1)
    return r, C


def Ex_exact_periodic(R_F: int, L: float, C=None) -> float:
    """E_x^sigma = -1/2 sum_{n != 0} C(n) / (pi L |n|^2) (periodic kernel, exact V)."""
    if C is None:
        C = difference_histogram(R_F)
    r, C = _hist_vectors(C)
    m = r[:, None, None] ** 2 + r[None, :, None] ** 2 + r[None, None, :] ** 2
    nz = m > 0
    return -0.5 * float((C[nz] / (np.pi * L * m[nz])).sum())


def Ex_separable_periodic(R_F: int, L: float, a, w, C=None) -> float:
    """E_x^sigma with V replaced by its node sum (n = 0 excluded)."""
    if C is None:
        C = difference_histogram(R_F)
    r, C = _hist_vectors(C)
    m = r[:, None, None] ** 2 + r[None, :, None] ** 2 + r[None, None, :] ** 2
    nz = m > 0
    Vm = V_of_m_separable(np.arange(int(m.max()) + 1), L, a, w)
    return -0.5 * float((C[nz] * Vm[m[nz]]).sum())


def Ex_box(R_F: int, L: float, alpha, omega, C=None, table=None) -> float:
    """E_x^sigma = -1/2 sum_n C(n) V_box(n) with the node sum of the box kernel
    (n = 0 included).  The node sum runs over every (n_x, n_y, n_z) of the histogram."""
    if C is None:
        C = difference_histogram(R_F)
    r, C = _hist_vectors(C)
    if table is None:
        table = box_table(alpha, 2 * R_F, L)
    ar = np.abs(r)
    Cf = C.astype(np.float64)
    total = 0.0
    for s in range(len(alpha)):
        Ax = table[s, ar]
        total += omega[s] * float(np.einsum("ijk,i,j,k->", Cf, Ax, Ax, Ax, optimize=True))
    return -0.5 * total / (2.0 * np.pi ** 2)


def Ex_from_eps(R: int, R_F: int, eps_basis) -> float:
    """E_x^sigma = 1/2 sum_{i in F} eps(n_i) from per-basis values of basis(R)."""
    k = basis(R)
    occ = (k * k).sum(axis=1) <= R_F * R_F
    return 0.5 * float(np.asarray(eps_basis)[occ].sum())
