"""Oracle pins: Laplace-variable meshes (Sec. II Eqs. 5-14, Table I meshes)."""
import numpy as np
import pytest

from oracle import quadrature as oq


@pytest.mark.parametrize("q", [1, 2, 5, 16, 60])
def test_gauss_legendre_exact_for_polynomials(q):
    a, b = 0.3, 1.7
    x, w = oq.gauss_legendre(q, a, b)
    assert abs(w.sum() - (b - a)) < 1e-13
    for k in range(2 * q):  # exact up to degree 2q - 1
        exact = (b ** (k + 1) - a ** (k + 1)) / (k + 1)
        assert abs((w * x ** k).sum() - exact) <= 1e-12 * max(1.0, abs(exact))


def test_mesh_structure():
    a, w, part = oq.laplace_mesh(64, 3, 21)
    assert len(a) == 64 and (part == 0).sum() == 43 and (part == 1).sum() == 21
    assert oq.interval1_counts(64, 3, 21) == [11, 11, 11, 10]
    assert np.all(a[part == 0] > 0) and np.all(a[part == 0] < 1)
    assert np.all(a[part == 1] > 1)
    assert np.all(w > 0)
    # paper meshes: 2Q nodes for Mesh 1, 8q + q_tail for Mesh 2
    assert len(oq.paper_mesh1(90)[0]) == 180
    assert len(oq.paper_mesh2(10)[0]) == 170
    assert oq.interval1_edges(7)[1] == pytest.approx(5.0 ** -7)


@pytest.mark.parametrize("S,R", [(32, 4), (64, 13), (96, 31), (128, 63)])
def test_closed_forms_per_interval(S, R):
    """int_0^1 e^{-am} da = (1 - e^{-m})/m and int_1^inf e^{-am} da = e^{-m}/m, m = |n|^2.
    A wrong tail Jacobian (w/t^3, 2w/t^2, ...) or a wrong sub-interval map fails here."""
    n_sub, q_tail = oq.default_periodic_mesh(S, R)
    a, w, part = oq.laplace_mesh(S, n_sub, q_tail)
    m = np.arange(1, 12 * R * R + 1, dtype=np.float64)
    E = np.exp(-np.outer(m, a))
    i1 = E[:, part == 0] @ w[part == 0]
    i2 = E[:, part == 1] @ w[part == 1]
    ex1 = -np.expm1(-m) / m
    ex2 = np.exp(-m) / m
    tot_err = np.max(np.abs(i1 + i2 - 1.0 / m) * m)
    bound = {32: 2e-5, 64: 3e-8, 96: 1e-10, 128: 5e-12}[S]
    assert tot_err < bound
    # each interval on its own meets the same bound (in units of the exact 1/m)
    assert np.max(np.abs(i2 - ex2) * m) < bound
    assert np.max(np.abs(i1 - ex1) * m) < bound


def test_error_shrinks_with_nodes():
    R = 13
    m = np.arange(1, 12 * R * R + 1, dtype=np.float64)
    errs = []
    for S in (24, 48, 72, 96):  # fixed structure: 4 sub-intervals, a third in the tail
        a, w, _ = oq.laplace_mesh(S, 3, S // 3)
        errs.append(np.max(np.abs(np.exp(-np.outer(m, a)) @ w - 1.0 / m) * m))
    assert all(errs[i + 1] < errs[i] / 10 for i in range(len(errs) - 1))


@pytest.mark.parametrize("S,R", [(32, 4), (64, 13), (96, 31), (128, 63)])
def test_pruning_keeps_accuracy(S, R):
    n_sub, q_tail = oq.default_periodic_mesh(S, R)
    a, w, _ = oq.laplace_mesh(S, n_sub, q_tail)
    keep = oq.prune_periodic(a, w, R, 1e-9)
    assert 0 < keep.sum() < S
    m = np.arange(1, 12 * R * R + 1, dtype=np.float64)
    full = np.exp(-np.outer(m, a)) @ w
    kept = np.exp(-np.outer(m, a[keep])) @ w[keep]
    assert np.max(np.abs(full - kept) * m) < 1e-9
    # the dropped nodes carry almost all of the (divergent) m = 0 weight
    assert w[keep].sum() < 100 and w.sum() > 1e3


def test_plain_two_interval_mesh_is_poor_at_large_m():
    """Sec. III remark on sharp structure near alpha = 0: one interval on [0, 1] with Q
    points converges slowly for large |q|, the geometric split does not."""
    m = np.arange(1, 12 * 13 * 13 + 1, dtype=np.float64)
    a1, w1, _ = oq.laplace_mesh(64, 0, 32)
    a2, w2, _ = oq.laplace_mesh(64, 3, 21)
    e1 = np.max(np.abs(np.exp(-np.outer(m, a1)) @ w1 - 1 / m) * m)
    e2 = np.max(np.abs(np.exp(-np.outer(m, a2)) @ w2 - 1 / m) * m)
    assert e1 > 1e-2 and e2 < 1e-7
