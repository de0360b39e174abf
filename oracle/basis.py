"""Planewave basis and occupations (oracle; test infrastructure only).

Sec. II, Eq. 1: g_I(r) = prod_x f_{I_x}(x), here f_l(x) = L^{-1/2} exp(i 2 pi l x / L).
Sec. II (text after Eq. 1): all products with (2 pi / L)|I| below a cutoff.  The cutoff is
read as |n|^2 <= R^2 (inclusive), the only reading that gives the shell-closing counts
7, 33, ..., 9171 printed in Sec. III.
Canonical order (the paper is silent): lexicographic ascending (n_x, n_y, n_z); the id of
a function is its rank in that order.
"""
import numpy as np


def basis(R: int) -> np.ndarray:
    """int64[Nb, 3]: every integer vector with |n|^2 <= R^2, lexicographic order."""
    out = []
    for x in range(-R, R + 1):
        for y in range(-R, R + 1):
            for z in range(-R, R + 1):
                if x * x + y * y + z * z <= R * R:
                    out.append((x, y, z))
    return np.array(out, dtype=np.int64).reshape(-1, 3)


def count(R: int) -> int:
    """Number of planewaves with |n|^2 <= R^2 (Sec. III shell closings for R = 1..13)."""
    r = np.arange(-R, R + 1)
    return int(((r[:, None, None] ** 2 + r[None, :, None] ** 2 + r[None, None, :] ** 2)
                <= R * R).sum())


def occupied(R_F: int) -> np.ndarray:
    """Sec. III: occupation 1 for every planewave inside the Fermi sphere |n| <= R_F."""
    return basis(R_F)


def occupation_grid(R: int, R_F: int) -> np.ndarray:
    """0/1 float64 tensor on the (2R+1)^3 grid n in [-R, R]^3, index [n_x+R, n_y+R, n_z+R]."""
    r = np.arange(-R, R + 1)
    m = r[:, None, None] ** 2 + r[None, :, None] ** 2 + r[None, None, :] ** 2
    return (m <= R_F * R_F).astype(np.float64)
