"""GPU parity: general (not necessarily momentum-conserving) integrals of the box kernel,
(IJ|KL) = 1/(2 pi^2) sum_s w_s prod_x A(alpha_s, D1_x, D2_x) (Sec. II Eqs. 8 and 14), from
the library's two-index per-axis tables, against the FP64 oracle at the library's point
count per axis integral.

The box integrand changes sign, so a node sum can cancel: results are compared against
the sum of the absolute node terms (the sum's condition scale), and the plain relative
error is checked where the sum does not cancel."""
import numpy as np
import pytest

import coulomb_inputs as ci
from gpu_common import BOX_POINTS, TOL_FP32, TOL_FP64_BOX, need_gpu
from oracle import basis as ob
from oracle import coulomb as oc
from oracle import quadrature as oq

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    return need_gpu()


def _box_tables(R, L, mesh):
    import paper_1502_08043_gb300 as cc
    if mesh[0] == "mesh2":
        a, w, _ = oq.paper_mesh2(mesh[1], mesh[2])
        t = cc.build_tables("box", R=R, L=L, S=len(a), n_sub=7, q_tail=mesh[2])
    else:
        a, w, _ = oq.paper_mesh1(mesh[1])
        t = cc.build_tables("box", R=R, L=L, S=2 * mesh[1], n_sub=0, q_tail=mesh[1])
    return t, a, w


def _codes(R):
    """(d1, d2) of every canonical code d1^2 + d1 + d2, d1 >= |d2|, in code order."""
    out = []
    for d1 in range(2 * R + 1):
        for d2 in range(-d1, d1 + 1):
            out.append((d1, d2))
    return np.array(out)


def _run(t, q_np, dtype, dev, fmt="ids", lookup="general"):
    import torch
    import paper_1502_08043_gb300 as cc
    qd = torch.from_numpy(q_np).to(dev)
    out = torch.full((len(q_np),), float("nan"), dtype=dtype, device=dev)
    cnt = torch.zeros(3, dtype=torch.int64, device=dev)
    cc.reconstruct_integrals(t, qd, out, lookup=lookup, counters=cnt)
    return out.cpu().numpy().astype(np.float64), cnt.cpu().numpy()


def _oracle(q, R, L, a, w):
    """Values, absolute-term sums and counters of id quadruples (ids outside the basis: 0)."""
    B = ob.basis(R)
    ok = np.all((q >= 0) & (q < len(B)), axis=1)
    v = B[np.where(ok[:, None], q, 0)]
    ref = oc.V_box_general(v[:, 0], v[:, 1], v[:, 2], v[:, 3], a, w, L, BOX_POINTS)
    ab = oc.V_box_general(v[:, 0], v[:, 1], v[:, 2], v[:, 3], a, w, L, BOX_POINTS,
                          absolute=True)
    nonc = np.any(v[:, 1] - v[:, 0] + v[:, 3] - v[:, 2] != 0, axis=1)
    cnt = np.array([int((ok & nonc).sum()), 0, int((~ok).sum())])
    return np.where(ok, ref, 0.0), np.where(ok, ab, 1.0), cnt, ok, nonc


def test_general_tables_vs_oracle(dev):
    R, L = 6, 2.0
    t, a, w = _box_tables(R, L, ("mesh2", 5, 20))
    assert t.info["general_codes"] == (2 * R + 1) ** 2
    G = t.general_values()
    d = _codes(R)
    Go = oc.A_box_general(a, d[:, 0], d[:, 1], L, BOX_POINTS)
    scale = np.max(np.abs(Go), axis=1, keepdims=True)
    assert np.max(np.abs(G - Go) / scale) < 1e-12
    # D1 + D2 = 0 entries are the conserving table, bit for bit
    T = t.values()
    for d1 in range(2 * R + 1):
        assert np.array_equal(G[:, d1 * d1], T[:, d1])
    t.free()


@pytest.mark.parametrize("fmt", ["ids", "ids16", "vec"])
def test_general_lookup_planted_and_uniform(dev, fmt):
    import torch
    R, L = 6, 2.0
    t, a, w = _box_tables(R, L, ("mesh2", 5, 20))
    B = ob.basis(R)
    q = np.concatenate([ci.quads(R, 0, 6000, stream=ci.STREAM_PLANTED),
                        ci.quads_uniform(R, 0, 6000)])
    if fmt != "vec":
        q[5::997, 3] = len(B) + 2
        q[7::1201, 0] = -4 if fmt == "ids" else len(B)
    ref, ab, cnt_ref, ok, nonc = _oracle(q, R, L, a, w)
    assert cnt_ref[0] > 5000 and (fmt == "vec" or cnt_ref[2] > 10)
    if fmt == "ids":
        qin = q
    elif fmt == "ids16":
        qin = (q.astype(np.int64) & 0xFFFF).astype(np.uint16).view(np.int16)
    else:
        qin = ci.quads_as_vectors(q, B)
    cancel = ab > 1.000001 * np.abs(ref)
    for dtype, tol in ((torch.float64, TOL_FP64_BOX), (torch.float32, TOL_FP32)):
        got, cnt = _run(t, qin, dtype, dev, fmt)
        assert np.array_equal(cnt, cnt_ref)
        assert np.all(got[~ok] == 0) and not np.isnan(got).any()
        assert np.max(np.abs(got - ref) / ab) < tol
        plain = ok & ~cancel & (ref != 0)
        assert np.max(np.abs(got[plain] - ref[plain]) / np.abs(ref[plain])) < tol
        # conserving quadruples: the same bits as the one-index (separable) lookup
        sep, _ = _run(t, qin, dtype, dev, fmt, lookup="separable")
        cons = ok & ~nonc
        assert np.array_equal(got[cons], sep[cons])
    t.free()


@pytest.mark.parametrize("n", [0, 1, 31, 33, 257, 100003])
def test_general_lookup_ragged(dev, n):
    import torch
    R, L = 4, 2.0
    t, a, w = _box_tables(R, L, ("mesh1", 12))
    q = ci.quads_uniform(R, 11, n)
    got, cnt = _run(t, q, torch.float32, dev)
    if n:
        ref, ab, cnt_ref, _, _ = _oracle(q, R, L, a, w)
        assert np.array_equal(cnt, cnt_ref)
        assert np.max(np.abs(got - ref) / ab) < TOL_FP32
    else:
        assert np.array_equal(cnt, [0, 0, 0])
    t.free()


def test_general_lookup_paper_table(dev):
    """The paper's stored-table case: 9171 planewaves (|n| <= 13), box side 2, Mesh 1 with
    Q = 90 (180 nodes): the FP32 two-index table (729 codes x 192 padded nodes, 560 KB)
    exceeds shared memory and is read through L1 from global memory.  1e6 uniform
    quadruples generated on the device, 3000 sampled against the oracle."""
    import torch
    import paper_1502_08043_gb300 as cc
    R, L, n = 13, 2.0, 1_000_000
    t, a, w = _box_tables(R, L, ("mesh1", 90))
    assert t.info["general_codes"] == 729 and t.info["S_eff"] == 180
    assert t.info["general_table_bytes"] == 729 * 192 * 4
    qd = torch.empty((n, 4), dtype=torch.int32, device=dev)
    ci.quads_device(R, 0, n, qd, stream=ci.STREAM_UNIFORM)
    idx = np.unique(np.random.default_rng(3).integers(0, n, 3000))
    q = ci.quads_uniform(R, 0, n)[idx]
    assert np.array_equal(qd.cpu().numpy()[idx], q)
    ref, ab, _, _, _ = _oracle(q, R, L, a, w)
    for dtype, tol in ((torch.float64, TOL_FP64_BOX), (torch.float32, TOL_FP32)):
        out = torch.full((n,), float("nan"), dtype=dtype, device=dev)
        cnt = torch.zeros(3, dtype=torch.int64, device=dev)
        cc.reconstruct_integrals(t, qd, out, lookup="general", counters=cnt)
        got = out.cpu().numpy().astype(np.float64)
        assert not np.isnan(got).any()
        assert int(cnt[2]) == 0 and int(cnt[1]) == 0 and int(cnt[0]) > 0.99 * n
        assert np.max(np.abs(got[idx] - ref) / ab) < tol
    t.free()


def test_general_lookup_rejected_for_periodic(dev):
    import torch
    import paper_1502_08043_gb300 as cc
    t = cc.build_tables("periodic", R=4, L=10.0, S=32)
    assert t.info["general_codes"] == 0 and t.info["general_table_bytes"] == 0
    q = torch.zeros((4, 4), dtype=torch.int32, device=dev)
    out = torch.empty(4, dtype=torch.float32, device=dev)
    with pytest.raises(cc.CoulombError) as e:
        cc.reconstruct_integrals(t, q, out, lookup="general")
    assert e.value.status == 6
    with pytest.raises(cc.CoulombError) as e:
        t.general_values()
    assert e.value.status == 6
    t.free()
