"""Coulomb integrals over planewaves (oracle; test infrastructure only).

Definition (Sec. II, Eq. 2, read with complex conjugates on the first function of each
pair, chemists' notation; the printed Eq. 2 puts all four functions at r and has no
conjugates):
    (IJ|KL) = int int g_I*(r) g_J(r) |r - r'|^-1 g_K*(r') g_L(r') d^3r d^3r'.

PERIODIC kernel (planewaves g_n = Omega^{-1/2} exp(i 2 pi n.r / L), Omega = L^3, periodic
images, neutralising background so that the q = 0 term is removed):
    (IJ|KL) = delta(n_J - n_I + n_L - n_K) V(n_J - n_I),   V(n) = 4 pi / (Omega |q|^2)
with q = 2 pi n / L, i.e. V(n) = 1 / (pi L |n|^2); V(0) is excluded (returned as 0).
Laplace form (Eqs. 5-7 in index units a = alpha (2 pi / L)^2):
    V(n) = 1/(pi L) int_0^inf exp(-a |n|^2) da = 1/(pi L) int_0^inf prod_x exp(-a n_x^2) da,
whose node sum (Eq. 14) is V_s(n) = 1/(pi L) sum_s w_s prod_x T_s[n_x], T_s[D] = exp(-a_s D^2).

BOX kernel (the model behind the paper's printed numbers): the continuous Fourier
transform of 1/|r| (Eqs. 3-5), 1/|r| = 1/(2 pi^2) int_0^inf d alpha prod_x int dp
exp(-alpha p^2 + i p x), and the p integral done in closed form (Eq. 9 form),
int dp exp(-alpha p^2 + i p u) = sqrt(pi/alpha) exp(-u^2 / (4 alpha)).  With box-normalised
planewaves on [0, L] the per-axis integral of Eq. 8 for a momentum-conserving pair
difference Delta becomes, with u = x - x',
    A(alpha, Delta) = 2/L^2 int_0^L (L - u) cos(2 pi Delta u / L) sqrt(pi/alpha)
                      exp(-u^2 / (4 alpha)) du,
and V_box(n) = 1/(2 pi^2) int_0^inf prod_x A(alpha, n_x) d alpha, finite at n = 0.
"""
import numpy as np

from .quadrature import gauss_legendre


# ---------------------------------------------------------------- periodic kernel
def V_exact(n, L: float):
    """V(n) = 1/(pi L |n|^2) for n != 0, 0 for n = 0.  n: int[..., 3]."""
    n = np.asarray(n, dtype=np.int64)
    m = (n * n).sum(axis=-1).astype(np.float64)
    out = np.zeros(m.shape)
    nz = m > 0
    out[nz] = 1.0 / (np.pi * L * m[nz])
    return out


def integral_exact(nI, nJ, nK, nL, L: float):
    """(IJ|KL) of four planewave index vectors (arrays [..., 3]), periodic kernel."""
    nI, nJ, nK, nL = (np.asarray(v, dtype=np.int64) for v in (nI, nJ, nK, nL))
    q = nJ - nI
    conserving = np.all(q + nL - nK == 0, axis=-1)
    return np.where(conserving, V_exact(q, L), 0.0)


def periodic_table(a, Dmax: int):
    """T_s[D] = exp(-a_s D^2) for D = 0..Dmax: float64[S, Dmax + 1]."""
    D = np.arange(Dmax + 1, dtype=np.float64)
    return np.exp(-np.outer(a, D * D))


def V_separable(n, L: float, a, w):
    """Eq. 14 node sum of the periodic kernel: 1/(pi L) sum_s w_s prod_x exp(-a_s n_x^2);
    0 at n = 0 (the excluded term)."""
    n = np.asarray(n, dtype=np.int64)
    shape = n.shape[:-1]
    n2 = n.reshape(-1, 3).astype(np.float64) ** 2
    acc = np.zeros(n2.shape[0])
    for s in range(len(a)):
        acc += w[s] * np.exp(-a[s] * n2[:, 0]) * np.exp(-a[s] * n2[:, 1]) * np.exp(-a[s] * n2[:, 2])
    acc /= np.pi * L
    acc[(n2.sum(axis=1) == 0)] = 0.0
    return acc.reshape(shape)


def V_of_m_separable(m, L: float, a, w):
    """The node sum as a function of the integer m = |n|^2 only (the product of the three
    per-axis Gaussians of one node depends on n through |n|^2): 1/(pi L) sum_s w_s
    exp(-a_s m), 0 at m = 0."""
    m = np.asarray(m, dtype=np.float64)
    acc = np.zeros(m.shape)
    for s in range(len(a)):
        acc += w[s] * np.exp(-a[s] * m)
    acc /= np.pi * L
    return np.where(m == 0, 0.0, acc)


# ---------------------------------------------------------------- box kernel
BOX_GL_POINTS = 2000


def A_box(alpha, Delta, L: float, points: int = BOX_GL_POINTS):
    """A(alpha, Delta) of the finite box for every alpha in `alpha`, Delta in `Delta`.

    Gauss-Legendre on [0, min(L, 14 sqrt(alpha))]; beyond 14 sqrt(alpha) the Gaussian is
    below exp(-49).  Returns float64[len(alpha), len(Delta)].
    """
    alpha = np.atleast_1d(np.asarray(alpha, dtype=np.float64))
    Delta = np.atleast_1d(np.asarray(Delta, dtype=np.float64))
    out = np.empty((alpha.size, Delta.size))
    for s, al in enumerate(alpha):
        ub = min(L, 14.0 * np.sqrt(al))
        u, wu = gauss_legendre(points, 0.0, ub)
        g = np.sqrt(np.pi / al) * np.exp(-u * u / (4.0 * al))
        for d, D in enumerate(Delta):
            out[s, d] = 2.0 / L ** 2 * np.sum(wu * (L - u) * np.cos(2.0 * np.pi * D * u / L) * g)
    return out


def A_box_general(alpha, D1, D2, L: float, points: int = BOX_GL_POINTS):
    """Per-axis integral of the box kernel for a general (not necessarily momentum-
    conserving) quadruple (Sec. II Eq. 8 with box-normalised planewaves on [0, L]):
        A(alpha, D1, D2) = 1/L^2 int_0^L int_0^L g(x - x') exp(2 pi i (D1 x + D2 x') / L)
                           dx dx',   g(u) = sqrt(pi/alpha) exp(-u^2 / (4 alpha)),
    with D1 = J_x - I_x (the pair at r) and D2 = L_x - K_x (the pair at r').  With
    u = x - x' the x integral at fixed u is elementary because D1 + D2 is an integer:
        D1 + D2 = 0:  2/L^2 int_0^L (L - u) cos(2 pi D1 u / L) g(u) du   (= A_box),
        otherwise:    -1/(pi (D1 + D2) L) int_0^L g(u) (sin(2 pi D1 u / L)
                                                         + sin(2 pi D2 u / L)) du,
    real and symmetric in (D1, D2).  Gauss-Legendre on [0, min(L, 14 sqrt(alpha))] as in
    A_box.  D1, D2: int arrays of one shape; returns float64[len(alpha), *shape]."""
    alpha = np.atleast_1d(np.asarray(alpha, dtype=np.float64))
    D1 = np.asarray(D1, dtype=np.int64)
    D2 = np.asarray(D2, dtype=np.int64)
    shape = np.broadcast(D1, D2).shape
    d1 = np.broadcast_to(D1, shape).reshape(-1).astype(np.float64)
    d2 = np.broadcast_to(D2, shape).reshape(-1).astype(np.float64)
    sig = d1 + d2
    out = np.empty((alpha.size, d1.size))
    for s, al in enumerate(alpha):
        ub = min(L, 14.0 * np.sqrt(al))
        u, wu = gauss_legendre(points, 0.0, ub)
        g = np.sqrt(np.pi / al) * np.exp(-u * u / (4.0 * al))
        c = np.cos(2.0 * np.pi * np.outer(d1, u) / L)
        sn = np.sin(2.0 * np.pi * np.outer(d1, u) / L) + np.sin(2.0 * np.pi * np.outer(d2, u) / L)
        cons = 2.0 / L ** 2 * ((L - u) * g * wu) @ c.T
        with np.errstate(divide="ignore", invalid="ignore"):
            gen = -(sn @ (g * wu)) / (np.pi * sig * L)
        out[s] = np.where(sig == 0, cons, gen)
    return out.reshape((alpha.size,) + shape)


def V_box_general(nI, nJ, nK, nL, alpha, omega, L: float, points: int = BOX_GL_POINTS,
                  absolute: bool = False):
    """(IJ|KL) of the box kernel for any quadruple of planewave index vectors ([..., 3]),
    momentum-conserving or not: 1/(2 pi^2) sum_s omega_s prod_x A(alpha_s, D1_x, D2_x)
    with D1 = n_J - n_I, D2 = n_L - n_K (the Eq. 14 node sum of Eq. 8); `points`
    Gauss-Legendre points per axis integral.  A is evaluated once per distinct (D1, D2)
    pair of the batch.  absolute=True returns 1/(2 pi^2) sum_s |omega_s prod_x A| instead,
    the scale against which the rounding of the (sign-changing) node sum is measured."""
    D1 = np.asarray(nJ, dtype=np.int64) - np.asarray(nI, dtype=np.int64)
    D2 = np.asarray(nL, dtype=np.int64) - np.asarray(nK, dtype=np.int64)
    shape = D1.shape[:-1]
    D1 = D1.reshape(-1, 3)
    D2 = D2.reshape(-1, 3)
    pairs = np.stack([D1.reshape(-1), D2.reshape(-1)], axis=1)   # [n * 3, 2], axis fastest
    uniq, inv = np.unique(pairs, axis=0, return_inverse=True)
    inv = inv.reshape(-1, 3)
    A = A_box_general(alpha, uniq[:, 0], uniq[:, 1], L, points)  # [S, distinct pairs]
    acc = np.zeros(D1.shape[0])
    for s in range(len(alpha)):
        term = omega[s] * A[s, inv[:, 0]] * A[s, inv[:, 1]] * A[s, inv[:, 2]]
        acc += np.abs(term) if absolute else term
    return (acc / (2.0 * np.pi ** 2)).reshape(shape)


def box_table(alpha, Dmax: int, L: float, points: int = BOX_GL_POINTS):
    """A(alpha_s, D) for D = 0..Dmax: float64[S, Dmax + 1] (`points` Gauss-Legendre points
    per axis integral)."""
    return A_box(alpha, np.arange(Dmax + 1), L, points)


def V_box_separable(n, alpha, omega, L: float, table=None):
    """Eq. 14 node sum of the box kernel: 1/(2 pi^2) sum_s omega_s prod_x A(alpha_s, n_x);
    n = 0 included."""
    n = np.abs(np.asarray(n, dtype=np.int64))
    shape = n.shape[:-1]
    n = n.reshape(-1, 3)
    if table is None:
        table = box_table(alpha, int(n.max()) if n.size else 0, L)
    acc = np.zeros(n.shape[0])
    for s in range(len(alpha)):
        acc += omega[s] * table[s, n[:, 0]] * table[s, n[:, 1]] * table[s, n[:, 2]]
    return (acc / (2.0 * np.pi ** 2)).reshape(shape)
