"""Oracle pins: exchange sums of the uniform electron gas (Sec. III, Fig. 1)."""
import numpy as np
import pytest

from oracle import basis as ob
from oracle import coulomb as oc
from oracle import exchange as ox
from oracle import quadrature as oq


def test_histogram_direct_equals_fft_and_invariants():
    for R_F in (1, 2, 3, 4):
        Cd = ox.difference_histogram(R_F, "direct")
        Cf = ox.difference_histogram(R_F, "fft")
        M = ob.count(R_F)
        assert np.array_equal(Cd, Cf)
        assert Cd.sum() == M * M
        c = 2 * R_F
        assert Cd[c, c, c] == M
        assert np.array_equal(Cd, Cd[::-1, ::-1, ::-1])   # C(n) = C(-n)


def test_brute_force_pair_sum_tiny_box():
    R, R_F, L = 2, 1, 7.5
    B = ob.basis(R)
    F = ob.occupied(R_F)
    eps = ox.eps_exact(R, R_F, L)
    for k in range(len(B)):
        s = 0.0
        for j in range(len(F)):
            d = B[k] - F[j]
            m = int(d @ d)
            if m:
                s += 1.0 / (np.pi * L * m)
        assert abs(eps[k] + s) < 1e-14
    # E_x^sigma two ways: from eps on the occupied set and from the histogram
    assert abs(ox.Ex_from_eps(R, R_F, eps) - ox.Ex_exact_periodic(R_F, L)) < 1e-13


def test_exchange_scales_as_one_over_L():
    """Sec. III: E_x = beta(M, {q_k}) / L."""
    for R_F in (1, 3):
        e1 = ox.Ex_exact_periodic(R_F, 4.0) * 4.0
        e2 = ox.Ex_exact_periodic(R_F, 23.0) * 23.0
        assert abs(e1 - e2) < 1e-12 * abs(e1)


def test_continuum_limit_minus_0_4582_over_rs():
    """Fig. 1: E_x / E_KS converges linearly in M^{-1/3} to 1 (periodic kernel, exact V).
    E_KS / M = -0.4582 / r_s, so the same extrapolation checks E_x per electron against
    the continuum value at fixed r_s."""
    ratios, xs = [], []
    for R_F in range(1, 14):
        M = ob.count(R_F)
        L = 10.0
        r = ox.Ex_exact_periodic(R_F, L) / ox.E_KS(M, L)
        ratios.append(r)
        xs.append(M ** (-1.0 / 3.0))
        assert abs(ox.E_KS(M, L) / M * ox.r_s(M, L) + 0.4582) < 5e-5
    assert all(np.diff(ratios) > 0)
    slope = (ratios[-1] - ratios[-2]) / (xs[-1] - xs[-2])
    r_inf = ratios[-1] - slope * xs[-1]
    assert abs(r_inf - 1.0) < 0.01


def test_separable_exchange_matches_exact_within_method_error():
    R, R_F, L = 4, 2, 10.0
    a, w, _ = oq.laplace_mesh(32, 2, 10)
    ex = ox.eps_exact(R, R_F, L)
    sp = ox.eps_separable(R, R_F, L, a, w)
    assert np.max(np.abs(sp - ex) / np.abs(ex)) < 2e-5
    assert abs(ox.Ex_separable_periodic(R_F, L, a, w) - ox.Ex_from_eps(R, R_F, sp)) < 1e-12
    # pruning (drops the huge-weight tail nodes) changes the values by < 1e-9 relative
    keep = oq.prune_periodic(a, w, R, 1e-9)
    sp2 = ox.eps_separable(R, R_F, L, a[keep], w[keep])
    assert np.max(np.abs(sp2 - sp) / np.abs(sp)) < 1e-9


def test_box_exchange_two_ways():
    R, R_F, L = 3, 2, 2.0
    a, w, _ = oq.paper_mesh2(5, 20)
    eps = ox.eps_box(R, R_F, L, a, w)
    assert abs(ox.Ex_from_eps(R, R_F, eps) - ox.Ex_box(R_F, L, a, w)) < 1e-12 * abs(eps).max() * 100
    assert np.all(eps < 0)


def test_whole_grid_convolution_equals_pair_sums():
    """eps on the whole grid as a 3D convolution of the occupation with the node sum (FFT)
    equals the direct pair sum of eps_separable at every basis function, and is 0 outside
    the basis sphere; a brute-force loop pins one point independently of both."""
    for R, R_F, L, S in ((4, 2, 10.0, 32), (6, 6, 7.0, 40), (9, 3, 12.0, 48), (12, 9, 20.0, 64)):
        n_sub, q_tail = oq.default_periodic_mesh(S, R)
        a, w, _ = oq.laplace_mesh(S, n_sub, q_tail)
        grid = ox.eps_separable_grid(R, R_F, L, a, w)
        ref = ox.eps_on_grid(R, ox.eps_separable(R, R_F, L, a, w))
        inside = ref != 0
        assert np.array_equal(grid == 0, ~inside)
        assert np.max(np.abs(grid[inside] - ref[inside]) / np.abs(ref[inside])) < 1e-13
    R, R_F, L, S = 3, 2, 5.0, 24
    a, w, _ = oq.laplace_mesh(S, *oq.default_periodic_mesh(S, R))
    grid = ox.eps_separable_grid(R, R_F, L, a, w)
    k = np.array([1, -2, 2])
    s = 0.0
    for j in ob.occupied(R_F):
        d = k - j
        if np.any(d != 0):
            s += np.sum(w * np.exp(-a * float(d @ d))) / (np.pi * L)
    assert abs(grid[k[0] + R, k[1] + R, k[2] + R] + s) < 1e-14 * s
