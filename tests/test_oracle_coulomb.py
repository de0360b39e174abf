"""Oracle pins: planewave Coulomb integrals (Sec. II Eqs. 2-8, 14; Table I)."""
import os
import itertools

import numpy as np
import pytest

from oracle import basis as ob
from oracle import coulomb as oc
from oracle import exchange as ox
from oracle import quadrature as oq

GOLD = os.path.join(os.path.dirname(__file__), "golden", "table1.txt")


def _poisson_fft(nI, nJ, nK, nL, L, N=16):
    """(IJ|KL) from its definition on a real-space grid: pair densities
    conj(g_I) g_J and conj(g_K) g_L sampled, periodic Poisson equation solved by FFT
    with the G = 0 component removed, energy = int rho_IJ phi_KL."""
    j = np.arange(N) * (L / N)
    X, Y, Z = np.meshgrid(j, j, j, indexing="ij")
    r = np.stack([X, Y, Z], axis=-1)
    Om = L ** 3

    def g(n):
        return np.exp(1j * 2 * np.pi / L * (r @ np.asarray(n, float))) / np.sqrt(Om)

    rho_ij = np.conj(g(nI)) * g(nJ)
    rho_kl = np.conj(g(nK)) * g(nL)
    c = np.fft.fftn(rho_kl) / N ** 3
    k = np.fft.fftfreq(N, d=1.0 / N)
    KX, KY, KZ = np.meshgrid(k, k, k, indexing="ij")
    G2 = (2 * np.pi / L) ** 2 * (KX ** 2 + KY ** 2 + KZ ** 2)
    kern = np.zeros_like(G2)
    kern[G2 > 0] = 4 * np.pi / G2[G2 > 0]
    phi = np.fft.ifftn(c * kern) * N ** 3
    return Om * np.mean(rho_ij * phi)


def test_closed_form_matches_fft_poisson():
    rng = np.random.default_rng(7)
    B = ob.basis(2)
    L = 3.7
    for _ in range(40):
        I, J, K = rng.integers(0, len(B), 3)
        # half conserving, half random
        nL = B[I] + B[K] - B[J]
        if rng.random() < 0.5 or (nL * nL).sum() > 4:
            nL = B[rng.integers(0, len(B))]
        ref = _poisson_fft(B[I], B[J], B[K], nL, L)
        val = oc.integral_exact(B[I], B[J], B[K], nL, L)
        assert abs(ref.imag) < 1e-12
        assert abs(ref.real - val) < 1e-12 * max(1.0, abs(val))


def test_symmetries_and_conservation():
    rng = np.random.default_rng(11)
    B = ob.basis(3)
    L = 10.0
    ids = rng.integers(0, len(B), (3000, 4))
    v = B[ids]
    base = oc.integral_exact(v[:, 0], v[:, 1], v[:, 2], v[:, 3], L)
    # (IJ|KL) = (KL|IJ) = (JI|LK) = (LK|JI)
    for p in [(2, 3, 0, 1), (1, 0, 3, 2), (3, 2, 1, 0)]:
        assert np.array_equal(base, oc.integral_exact(*(v[:, i] for i in p), L))
    cons = np.all(v[:, 1] - v[:, 0] + v[:, 3] - v[:, 2] == 0, axis=1)
    assert np.all(base[~cons] == 0.0)
    # cubic group (axis permutations x sign flips) and pair translations
    for perm in itertools.permutations(range(3)):
        for sg in itertools.product((1, -1), repeat=3):
            w = v[:, :, list(perm)] * np.array(sg)
            assert np.array_equal(base, oc.integral_exact(w[:, 0], w[:, 1], w[:, 2], w[:, 3], L))
    t = np.array([2, -1, 5])
    assert np.array_equal(base, oc.integral_exact(v[:, 0] + t, v[:, 1] + t, v[:, 2], v[:, 3], L))


def test_separable_converges_to_exact():
    R = 4
    r = np.arange(-2 * R, 2 * R + 1)
    n = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3)
    n = n[(n * n).sum(1) > 0]
    L = 10.0
    ex = oc.V_exact(n, L)
    prev = np.inf
    for S in (32, 64, 96):
        n_sub, q_tail = oq.default_periodic_mesh(S, R)
        a, w, _ = oq.laplace_mesh(S, n_sub, q_tail)
        err = np.max(np.abs(oc.V_separable(n, L, a, w) - ex) / ex)
        assert err < prev / 10
        prev = err
    assert prev < 1e-9
    # the |n|^2 form of the node sum is the same sum
    a, w, _ = oq.laplace_mesh(32, 2, 10)
    m = (n * n).sum(1)
    assert np.allclose(oc.V_of_m_separable(m, L, a, w), oc.V_separable(n, L, a, w),
                       rtol=1e-14, atol=0)
    assert oc.V_separable(np.zeros(3, int), L, a, w) == 0.0


def test_box_self_term_is_mean_inverse_distance():
    """V_box(0) = (1/L^6) int int_{box} 1/|r - r'| = (1/L) E[1/|r - r'|] for uniform
    points of the unit cube, independent of the Laplace route:
    E[1/|d|] = int_{[0,1]^3} 8 (1-u)(1-v)(1-w) / |d| d^3d (difference density of two
    uniform points).  Split by the largest coordinate (3 equal parts), put v = u s,
    w = u t and integrate u in closed form:
    int_0^1 u (1-u)(1-su)(1-tu) du = 1/2 - (1+s+t)/3 + (s+t+st)/4 - st/5,
    leaving a smooth 2D integral over (s, t) in [0,1]^2 (adaptive cubature, scipy)."""
    from scipy import integrate
    f = lambda t, s: (0.5 - (1 + s + t) / 3 + (s + t + s * t) / 4 - s * t / 5) \
        / np.sqrt(1 + s * s + t * t)
    part, _ = integrate.dblquad(f, 0, 1, 0, 1, epsabs=1e-13, epsrel=1e-13)
    ref = 24.0 * part
    L = 2.0
    a, w, _ = oq.paper_mesh2(10)
    v0 = oc.V_box_separable(np.zeros(3, int), a, w, L)
    assert abs(v0 * L - ref) < 2e-7 * ref
    # and the kernel scales as 1/L at a fixed node set (scale alpha with L^2)
    L2 = 5.0
    v0b = oc.V_box_separable(np.zeros(3, int), a * (L2 / L) ** 2, w * (L2 / L) ** 2, L2)
    assert abs(v0b * L2 - v0 * L) < 1e-12


def test_box_axis_integral_properties():
    al = np.array([1e-5, 3e-3, 0.2, 1.0, 50.0, 1e4])
    A = oc.A_box(al, np.array([0, 1, 3, -3]), 2.0)
    assert np.allclose(A[:, 2], A[:, 3], rtol=0, atol=1e-15)   # even in Delta
    # small alpha: A -> (2/L^2) L sqrt(pi/alpha) * 2 sqrt(pi alpha) / 2 = 2 pi / L
    assert abs(A[0, 0] - np.pi) < 1e-2
    # large alpha: sqrt(alpha/pi) A(alpha, 0) -> (2/L^2) int_0^L (L - u) du = 1
    assert abs(A[-1, 0] * np.sqrt(al[-1] / np.pi) - 1.0) < 1e-4


def _table1():
    rows = [l.split() for l in open(GOLD) if l.strip() and not l.startswith("#")]
    return [(m, int(q), float(i1), float(t)) for m, q, i1, t in rows]


@pytest.fixture(scope="module")
def hist13():
    return ox.difference_histogram(13)


@pytest.mark.parametrize("mesh,q,int1,total", _table1())
def test_table1_reproduced(mesh, q, int1, total, hist13):
    """Table I: E_x/E_KS for M = 9171 under the paper's meshes, finite-box kernel, L = 2,
    alpha_c = 1, to 2e-6 (six printed digits)."""
    L = 2.0
    a, w, part = oq.paper_mesh1(q) if mesh == "mesh1" else oq.paper_mesh2(q)
    M = ob.count(13)
    tab = oc.box_table(a, 26, L)
    e1 = ox.Ex_box(13, L, a[part == 0], w[part == 0], hist13, tab[part == 0])
    e2 = ox.Ex_box(13, L, a[part == 1], w[part == 1], hist13, tab[part == 1])
    ks = ox.E_KS(M, L)
    assert abs(e1 / ks - int1) < 2e-6
    assert abs((e1 + e2) / ks - total) < 2e-6


def test_box_general_axis_integral_brute_force():
    """The per-axis integral of a general (non-conserving) box quadruple, Eq. 8 with
    box-normalised planewaves, against a brute-force 2D Gauss-Legendre quadrature of its
    defining double integral (complex exponentials over the square, no substitution):
    the closed-form inner integral of A_box_general, its signs and factors."""
    from oracle.quadrature import gauss_legendre
    L = 2.0
    # composite rule on [0, L]: 40 panels of 8 points
    edges = np.linspace(0.0, L, 41)
    xs, ws = [], []
    for lo, hi in zip(edges[:-1], edges[1:]):
        x, w = gauss_legendre(8, lo, hi)
        xs.append(x)
        ws.append(w)
    x = np.concatenate(xs)
    w = np.concatenate(ws)
    X, XP = np.meshgrid(x, x, indexing="ij")
    W = np.outer(w, w)
    pairs = [(0, 0), (1, -1), (2, 1), (-1, 2), (3, 0), (1, 1), (-2, -3), (4, -1)]
    for al in (0.05, 0.4, 2.5):
        g = np.sqrt(np.pi / al) * np.exp(-(X - XP) ** 2 / (4.0 * al))
        got = oc.A_box_general(al, [p[0] for p in pairs], [p[1] for p in pairs], L)[0]
        for (d1, d2), v in zip(pairs, got):
            ph = np.exp(2j * np.pi * (d1 * X + d2 * XP) / L)
            ref = np.sum(W * g * ph) / L ** 2
            assert abs(ref.imag) < 1e-10
            assert abs(v - ref.real) < 1e-9 * max(1.0, abs(ref.real)), (al, d1, d2, v, ref)


def test_box_general_integrals_symmetries_and_conserving_case():
    """(IJ|KL) = (KL|IJ) = (JI|LK) for the real box-kernel integrals of arbitrary quadruples,
    and on momentum-conserving ones the general form equals the conserving node sum."""
    a, w, _ = oq.paper_mesh2(6, 24)
    L = 3.0
    rng = np.random.default_rng(5)
    n = rng.integers(-3, 4, size=(40, 4, 3))
    I, J, K, Lq = n[:, 0], n[:, 1], n[:, 2], n[:, 3]
    v = oc.V_box_general(I, J, K, Lq, a, w, L)
    assert np.allclose(v, oc.V_box_general(K, Lq, I, J, a, w, L), rtol=1e-13, atol=0)
    assert np.allclose(v, oc.V_box_general(J, I, Lq, K, a, w, L), rtol=1e-13, atol=0)
    # conserving quadruples: L = K + I - J
    Lc = K + I - J
    vc = oc.V_box_general(I, J, K, Lc, a, w, L)
    assert np.allclose(vc, oc.V_box_separable(J - I, a, w, L), rtol=1e-12, atol=0)
    # non-conserving ones are not zero in a finite box
    assert np.all(np.abs(v[np.any(J - I + Lq - K != 0, axis=1)]) > 0)
