"""GPU parity: integral reconstruction and pair matrices vs the FP64 oracle."""
import numpy as np
import pytest

import coulomb_inputs as ci
from gpu_common import (BOX_POINTS, CFG1, CFG2, CFG3, CFG5, TOL_FP32, TOL_FP64, TOL_FP64_BOX,
                        need_gpu, oracle_nodes, rel_err)
from oracle import basis as ob
from oracle import coulomb as oc
from oracle import quadrature as oq
from oracle import reconstruct as orc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    return need_gpu()


def _tables(cfg):
    import paper_1502_08043_gb300 as cc
    return cc.build_tables("periodic", R=cfg["R"], L=cfg["L"], S=cfg["S"])


def _run(t, q_np, lookup, dtype, dev, fmt="ids"):
    import torch
    import paper_1502_08043_gb300 as cc
    qd = torch.from_numpy(q_np).to(dev)
    out = torch.full((len(q_np),), float("nan"), dtype=dtype, device=dev)
    cnt = torch.zeros(3, dtype=torch.int64, device=dev)
    cc.reconstruct_integrals(t, qd, out, lookup=lookup, counters=cnt)
    return out.cpu().numpy(), cnt.cpu().numpy()


def as_ids16(q):
    """uint16 bit patterns of int32 ids (negative ids wrap to large, out-of-range ones)."""
    return (np.asarray(q, dtype=np.int64) & 0xFFFF).astype(np.uint16).view(np.int16)


@pytest.mark.parametrize("fmt", ["ids", "vec", "ids16"])
@pytest.mark.parametrize("lookup", ["separable", "collapsed"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_small_box_all_paths(dev, fmt, lookup, prec):
    """1e5 planted quadruples (5 % non-conserving, 1 % q = 0) plus out-of-range ones."""
    import torch
    R, L = CFG1["R"], CFG1["L"]
    t = _tables(CFG1)
    a, w = oracle_nodes(R, CFG1["S"])
    B = ob.basis(R)
    q = ci.quads(R, 0, 100000, stream=ci.STREAM_PLANTED)
    q[5::9973, 3] = len(B) + 1
    q[7::12011, 0] = -3
    ref, cnt_ref = orc.reconstruct(q, R, L, "separable", a=a, w=w)
    exact, _ = orc.reconstruct(q, R, L, "exact")
    qin = {"ids": q, "ids16": as_ids16(q)}.get(fmt)
    if qin is None:
        qin = ci.quads_as_vectors(np.clip(q, 0, len(B) - 1), B)
    if fmt == "vec":   # out-of-range vectors instead of out-of-range ids
        bad = np.any((q < 0) | (q >= len(B)), axis=1)
        qin[bad, 1, 0] = R + 1
        ref, cnt_ref = orc.reconstruct(qin, R, L, "separable", fmt="vec", a=a, w=w)
    dtype = torch.float64 if prec == "fp64" else torch.float32
    got, cnt = _run(t, qin, lookup, dtype, dev, fmt)
    assert np.array_equal(cnt, cnt_ref)
    assert np.array_equal(got == 0, ref == 0)          # bookkeeping is bit exact
    assert np.all(np.signbit(got[ref == 0]) == False)   # +0.0
    tol = TOL_FP64 if prec == "fp64" else TOL_FP32
    assert rel_err(got, ref) < tol
    # stated method error of the S = 32 mesh against the exact 1/(pi L |q|^2)
    assert rel_err(got, ref if fmt == "vec" else exact) < 2e-5
    t.free()


@pytest.mark.parametrize("n", [0, 1, 31, 33, 1000, 4097, 200003])
def test_ragged_sizes_paper_scale(dev, n):
    R, L = CFG2["R"], CFG2["L"]
    t = _tables(CFG2)
    a, w = oracle_nodes(R, CFG2["S"])
    q = ci.quads(R, 12345, n, stream=ci.STREAM_PLANTED)
    import torch
    ref, cnt_ref = orc.reconstruct(q, R, L, "separable", a=a, w=w)
    for lookup in ("separable", "collapsed"):
        for qin in (q, as_ids16(q)):
            got, cnt = _run(t, qin, lookup, torch.float32, dev)
            assert np.array_equal(cnt, cnt_ref)
            assert np.array_equal(got == 0, ref == 0)
            assert rel_err(got, ref) < TOL_FP32
    t.free()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_ids16_alignment_forms(dev, prec):
    """uint16-id quadruples on a 16-byte aligned buffer, on a buffer that is only 8-byte
    aligned (the stated minimum) and with the output one value off its allocation: the
    same values and counters bit for bit, and the oracle's."""
    import torch
    import paper_1502_08043_gb300 as cc
    R, L = CFG2["R"], CFG2["L"]
    t = _tables(CFG2)
    a, w = oracle_nodes(R, CFG2["S"])
    n = 4099
    q = ci.quads(R, 777, n, stream=ci.STREAM_PLANTED)
    q[3::1021, 2] = 65000  # out of range (also as a uint16 id)
    ref, cnt_ref = orc.reconstruct(q, R, L, "separable", a=a, w=w)
    dtype = torch.float64 if prec == "fp64" else torch.float32
    q16 = torch.from_numpy(as_ids16(q)).to(dev)
    big = torch.zeros((n + 1, 4), dtype=torch.int16, device=dev)
    big[1:] = q16
    outs = []
    for qin, shift in ((q16, 0), (big[1:], 0), (q16, 1)):
        assert qin.is_contiguous()
        ob_ = torch.full((n + 1,), float("nan"), dtype=dtype, device=dev)
        out = ob_[shift:shift + n]
        cnt = torch.zeros(3, dtype=torch.int64, device=dev)
        cc.reconstruct_integrals(t, qin, out, lookup="collapsed", counters=cnt)
        outs.append((out.cpu().numpy(), cnt.cpu().numpy()))
    assert (big[1:].data_ptr() % 16) == 8
    for got, cnt in outs:
        assert np.array_equal(cnt, cnt_ref)
        assert np.array_equal(got == 0, ref == 0)
        assert np.array_equal(got, outs[0][0])
    assert rel_err(outs[0][0], ref) < (TOL_FP64 if prec == "fp64" else TOL_FP32)
    t.free()


def _full_size(dev, cfg, n, sample):
    """Full-size batch generated on the GPU, both lookups as the bench launches them;
    sampled outputs recomputed by the oracle from its own copy of the inputs."""
    import torch
    import paper_1502_08043_gb300 as cc
    R, L = cfg["R"], cfg["L"]
    t = _tables(cfg)
    a, w = oracle_nodes(R, cfg["S"])
    q = torch.empty((n, 4), dtype=torch.int32, device=dev)
    ci.quads_device(R, 0, n, q)
    n_q0 = int((q[:, 0] == q[:, 1]).sum().item())
    rng = np.random.default_rng(5)
    idx = np.unique(np.concatenate([rng.integers(0, n, sample), [0, n - 1]]))
    q_np = ci.quads(R, 0, 0, indices=idx)
    assert np.array_equal(q[torch.from_numpy(idx).to(dev)].cpu().numpy(), q_np)
    ref, _ = orc.reconstruct(q_np, R, L, "separable", a=a, w=w)
    out = torch.empty(n, dtype=torch.float32, device=dev)
    forms = [q]
    if t.info["Nb"] <= 65536:   # the 8-byte uint16 form, as the bench step reads it
        forms.append(torch.where(q >= 32768, q - 65536, q).to(torch.int16))
    for qf in forms:
        for lookup in ("separable", "collapsed"):
            cnt = torch.zeros(3, dtype=torch.int64, device=dev)
            out.fill_(float("nan"))
            cc.reconstruct_integrals(t, qf, out, lookup=lookup, counters=cnt)
            assert cnt.cpu().tolist() == [0, n_q0, 0]
            got = out[torch.from_numpy(idx).to(dev)].cpu().numpy()
            assert np.array_equal(got == 0, ref == 0)
            assert rel_err(got, ref) < TOL_FP32
            assert not torch.isnan(out).any().item()
    del q, forms, out
    t.free()


def test_full_size_paper_scale(dev):
    _full_size(dev, CFG2, 100_000_000, 20000)


def test_full_size_large(dev):
    _full_size(dev, CFG5, 1_000_000_000, 4000)


@pytest.mark.parametrize("R", [15, 24, 63])
def test_id_decode_every_id(dev, R):
    """Lookups of bases too large to stage decode ids on chip from line hints (collapsed and
    separable).
    Every id of the basis is looked up against four anchors (0,0,0), (1,0,0), (0,1,0),
    (0,0,1) as (a, id, id, a), whose values V(|n_id - n_a|^2) (V strictly decreasing in m)
    fix n_id; the decoded and the gathered forms agree bit for bit in values and counters,
    in every id format and precision, and a sample agrees with the oracle."""
    import torch
    import paper_1502_08043_gb300 as cc
    L, S = 10.0, 48
    B = ob.basis(R)
    Nb = len(B)
    t = cc.build_tables("periodic", R=R, L=L, S=S)
    a, w = oracle_nodes(R, S)
    anchors = [int(np.flatnonzero((B == v).all(axis=1))[0])
               for v in ((0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1))]
    ids = np.arange(Nb, dtype=np.int32)
    q = np.concatenate([np.stack([np.full(Nb, an, np.int32), ids, ids,
                                  np.full(Nb, an, np.int32)], axis=1) for an in anchors])
    planted = ci.quads(R, 4242, 50000, stream=ci.STREAM_PLANTED)
    planted[11::4999, 1] = Nb      # out of range
    q = np.concatenate([q, planted])
    forms = [q] + ([as_ids16(q)] if Nb <= 65536 else [])
    rng = np.random.default_rng(7)
    idx = rng.integers(0, len(q), 20000)
    ref, _ = orc.reconstruct(q[idx], R, L, "separable", a=a, w=w)
    try:
        cases = [(p_, f_, l_) for p_ in (torch.float32, torch.float64) for f_ in forms
                 for l_ in ("collapsed", "separable")]
        for prec, qin, lookup in cases:
            res = []
            for on in (1, 0):
                assert cc.lib().cc_set_id_decode(on) == 0
                res.append(_run(t, qin, lookup, prec, dev))
            (got, cnt), (gat, cnt_g) = res
            assert np.array_equal(cnt, cnt_g)
            assert np.array_equal(got, gat)
            assert cnt[2] == len(range(11, 50000, 4999))
            tol = TOL_FP64 if prec == torch.float64 else TOL_FP32
            assert np.array_equal(got[idx] == 0, ref == 0)
            assert rel_err(got[idx], ref) < tol
        assert cc.lib().cc_set_id_decode(2) != 0
    finally:
        cc.lib().cc_set_id_decode(1)
        t.free()


def test_box_kernel_separable(dev):
    import torch
    import paper_1502_08043_gb300 as cc
    R, L = 6, 2.0
    ao, wo, _ = oq.paper_mesh2(5, 20)
    t = cc.build_tables("box", R=R, L=L, S=len(ao), n_sub=7, q_tail=20)
    q = ci.quads(R, 0, 20000, stream=ci.STREAM_PLANTED)
    tab = oc.box_table(ao, 2 * R, L, BOX_POINTS)
    ref, cnt_ref = orc.reconstruct(q, R, L, "box", a=ao, w=wo, box_table=tab)
    assert cnt_ref[1] == 0 and cnt_ref[0] > 0
    for dtype, tol in ((torch.float64, TOL_FP64_BOX), (torch.float32, TOL_FP32)):
        got, cnt = _run(t, q, "separable", dtype, dev)
        assert np.array_equal(cnt, cnt_ref)
        assert rel_err(got, ref) < tol
    with pytest.raises(cc.CoulombError) as e:
        _run(t, q, "collapsed", torch.float32, dev)
    assert e.value.status == 6
    t.free()


@pytest.mark.parametrize("lookup", ["separable", "collapsed"])
def test_pair_matrix(dev, lookup):
    import torch
    import paper_1502_08043_gb300 as cc
    # plain FP64 and FP32, every pair of the small basis
    R, L = CFG1["R"], CFG1["L"]
    t = _tables(CFG1)
    a, w = oracle_nodes(R, CFG1["S"])
    ref = orc.pair_matrix(R, L, value="separable", a=a, w=w)
    for dtype, tol in ((torch.float64, TOL_FP64), (torch.float32, TOL_FP32)):
        out = torch.empty(ref.shape, dtype=dtype, device=dev)
        cc.pair_matrix(t, 0, ref.shape[0], out, lookup=lookup)
        got = out.cpu().numpy()
        assert np.array_equal(got == 0, ref == 0)
        assert rel_err(got, ref) < tol
    t.free()
    # paper scale: all 9171^2 pairs as the bench launches them, sampled rows checked
    R, L = CFG2["R"], CFG2["L"]
    t = _tables(CFG2)
    a, w = oracle_nodes(R, CFG2["S"])
    Nb = t.info["Nb"]
    out = torch.empty((Nb, Nb), dtype=torch.float32, device=dev)
    cc.pair_matrix(t, 0, Nb, out, lookup=lookup)
    rows = [0, 1, 4585, 9000, Nb - 1]
    ref = orc.pair_matrix(R, L, rows=rows, value="separable", a=a, w=w)
    got = out[rows].cpu().numpy()
    assert np.array_equal(got == 0, ref == 0)
    assert rel_err(got, ref) < TOL_FP32
    # a row block in the middle
    part = torch.empty((7, Nb), dtype=torch.float32, device=dev)
    cc.pair_matrix(t, 4000, 7, part, lookup=lookup)
    assert torch.equal(part, out[4000:4007])
    t.free()


def test_unsupported_and_bad_args(dev):
    import torch
    import paper_1502_08043_gb300 as cc
    t = _tables(CFG1)
    L = cc.lib()
    q = torch.zeros((4, 4), dtype=torch.int32, device=dev)
    out = torch.empty(4, dtype=torch.float32, device=dev)
    # mixed precision is an exchange-only mode
    assert L.cc_reconstruct_integrals(t.handle, q.data_ptr(), 4, 0, 0, 2, out.data_ptr(),
                                      None, None) == 6
    # misaligned quadruple buffer
    assert L.cc_reconstruct_integrals(t.handle, q.data_ptr() + 4, 3, 0, 0, 1, out.data_ptr(),
                                      None, None) == 1
    # uint16 ids: 8-byte alignment; a basis above 65536 functions is out of range
    q16 = torch.zeros((4, 4), dtype=torch.int16, device=dev)
    assert L.cc_reconstruct_integrals(t.handle, q16.data_ptr() + 2, 3, 2, 0, 1, out.data_ptr(),
                                      None, None) == 1
    assert L.cc_reconstruct_integrals(t.handle, q16.data_ptr() + 8, 3, 2, 0, 1, out.data_ptr(),
                                      None, None) == 0
    t3 = _tables(CFG3)
    assert t3.info["Nb"] > 65536
    assert L.cc_reconstruct_integrals(t3.handle, q16.data_ptr(), 4, 2, 0, 1, out.data_ptr(),
                                      None, None) == 2
    t3.free()
    # unknown format
    assert L.cc_reconstruct_integrals(t.handle, q.data_ptr(), 4, 3, 0, 1, out.data_ptr(),
                                      None, None) == 1
    # rows beyond the basis
    assert L.cc_pair_matrix(t.handle, 250, 10, 0, 1, out.data_ptr(), None) == 1
    # empty batch is fine and touches nothing
    assert L.cc_reconstruct_integrals(t.handle, None, 0, 0, 0, 1, None, None, None) == 0
    t.free()
