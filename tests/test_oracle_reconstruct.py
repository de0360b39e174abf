"""Oracle pins: quadruple bookkeeping and batch reconstruction (Sec. II Eq. 14)."""
import numpy as np

import coulomb_inputs as ci
from oracle import basis as ob
from oracle import coulomb as oc
from oracle import quadrature as oq
from oracle import reconstruct as orc


def test_bookkeeping_counters_and_values():
    R, L = 4, 10.0
    B = ob.basis(R)
    q = ci.quads(R, 0, 4000, stream=ci.STREAM_PLANTED)
    q[:7, 2] = len(B) + 3     # out of range ids
    q[7:9, 0] = -1
    vals, cnt = orc.reconstruct(q, R, L, "exact")
    v = B[np.clip(q, 0, len(B) - 1)]
    bad = np.any((q < 0) | (q >= len(B)), axis=1)
    cons = np.all(v[:, 1] - v[:, 0] + v[:, 3] - v[:, 2] == 0, axis=1)
    q0 = np.all(v[:, 1] == v[:, 0], axis=1)
    assert cnt[2] == bad.sum() == 9
    assert cnt[0] == (~bad & ~cons).sum() > 100
    assert cnt[1] == (~bad & cons & q0).sum() > 10
    live = ~bad & cons & ~q0
    direct = np.array([oc.integral_exact(*B[row], L) for row in q[live]])
    assert np.array_equal(vals[live], direct)
    assert np.all(vals[~live] == 0.0)


def test_vector_form_equals_id_form():
    R, L = 4, 10.0
    B = ob.basis(R)
    q = ci.quads(R, 0, 2000, stream=ci.STREAM_PLANTED)
    vq = ci.quads_as_vectors(q, B)
    a, w, _ = oq.laplace_mesh(32, 2, 10)
    v1, c1 = orc.reconstruct(q, R, L, "separable", a=a, w=w)
    v2, c2 = orc.reconstruct(vq, R, L, "separable", fmt="vec", a=a, w=w)
    assert np.array_equal(v1, v2) and np.array_equal(c1, c2)
    vq[0, 1, 0] = 5  # |n|^2 > R^2
    _, c3 = orc.reconstruct(vq, R, L, "separable", fmt="vec", a=a, w=w)
    assert c3[2] == 1


def test_pair_matrix_is_exchange_integrals():
    R, L = 2, 5.0
    B = ob.basis(R)
    P = orc.pair_matrix(R, L)
    for i in range(0, len(B), 5):
        for j in range(0, len(B), 3):
            # (ij|ji) with conjugates on i and j: q = n_j - n_i
            assert P[i, j] == oc.integral_exact(B[i], B[j], B[j], B[i], L)
    assert np.all(np.diag(P) == 0)
    assert np.array_equal(P, P.T)
