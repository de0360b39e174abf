"""GPU parity: the batched engine (256 uneven boxes, one persistent graph-captured
launch) against the FP64 oracle, box by box."""
import numpy as np
import pytest

import coulomb_inputs as ci
from gpu_common import TOL_FP32, TOL_FP64, need_gpu, rel_err
from oracle import basis as ob
from oracle import exchange as ox
from oracle import quadrature as oq

pytestmark = pytest.mark.gpu


def _nodes(b):
    n_sub, q_tail = oq.default_periodic_mesh(b["S"], b["R"])
    a, w, _ = oq.laplace_mesh(b["S"], n_sub, q_tail)
    keep = oq.prune_periodic(a, w, b["R"], 1e-9)
    return a[keep], w[keep]


@pytest.fixture(scope="module")
def batch():
    import paper_1502_08043_gb300 as cc
    dev = need_gpu()
    boxes = ci.box_params(256)
    B = cc.Batch(boxes)
    yield dev, boxes, B
    B.free()


def _run(B, dev, dtype):
    import torch
    eps = torch.full((int(B.offsets[-1]),), float("nan"), dtype=dtype, device=dev)
    Ex = torch.zeros((B.nbox, 2), dtype=torch.float64, device=dev)
    B.exchange(eps, Ex)
    torch.cuda.synchronize()
    return eps.cpu().numpy().astype(np.float64), Ex.cpu().numpy()


def _box_eps(B, eps, i, R):
    Mg = 2 * R + 1
    g = eps[B.offsets[i]:B.offsets[i + 1]].reshape(Mg, Mg, Mg)
    k = ob.basis(R) + R
    return g, g[k[:, 0], k[:, 1], k[:, 2]]


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_all_boxes_exchange_energy(batch, prec):
    import torch
    dev, boxes, B = batch
    eps, Ex = _run(B, dev, torch.float32 if prec == "fp32" else torch.float64)
    tol = TOL_FP32 if prec == "fp32" else TOL_FP64
    assert not np.isnan(eps).any()
    for i, b in enumerate(boxes):
        a, w = _nodes(b)
        C = ox.difference_histogram(b["R_F"], "fft")
        ref = ox.Ex_separable_periodic(b["R_F"], b["L"], a, w, C)
        assert abs(Ex[i, 0] - ref) < tol * abs(ref), (i, b)
        assert Ex[i, 1] == 2 * Ex[i, 0]


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_all_boxes_full_grids(batch, prec):
    """Every grid point of all 256 boxes, element by element, against the oracle's eps on
    the whole grid (its FFT-convolution form, pinned to the direct pair sum on CPU)."""
    import torch
    dev, boxes, B = batch
    eps, _ = _run(B, dev, torch.float32 if prec == "fp32" else torch.float64)
    tol = TOL_FP32 if prec == "fp32" else TOL_FP64
    for i, b in enumerate(boxes):
        a, w = _nodes(b)
        grid, _ = _box_eps(B, eps, i, b["R"])
        ref = ox.eps_separable_grid(b["R"], b["R_F"], b["L"], a, w)
        assert np.array_equal(grid == 0, ref == 0), (i, b)
        assert rel_err(grid, ref) < tol, (i, b)


def test_replay_is_deterministic_and_tuner_keeps_results(batch):
    import torch
    dev, boxes, B = batch
    e1, x1 = _run(B, dev, torch.float32)
    e2, x2 = _run(B, dev, torch.float32)
    assert np.array_equal(e1, e2) and np.array_equal(x1, x2)
    eps = torch.empty((int(B.offsets[-1]),), dtype=torch.float32, device=dev)
    Ex = torch.zeros((B.nbox, 2), dtype=torch.float64, device=dev)
    choice = B.tune(eps, Ex, reps=3)
    assert choice["ctas_per_sm"] in (2, 4, 8) and choice["oversub"] in (1, 2, 4)
    assert choice["ms"] > 0
    e3, x3 = _run(B, dev, torch.float32)
    assert rel_err(e3, e1) < TOL_FP32 and np.max(np.abs(x3 - x1) / np.abs(x1)) < TOL_FP32


def test_batch_argument_errors():
    import paper_1502_08043_gb300 as cc
    need_gpu()
    with pytest.raises(cc.CoulombError) as e:
        cc.Batch([{"R": 25, "L": 10.0, "R_F": 5, "S": 32}])    # grid side 51 > 49
    assert e.value.status == 2
    with pytest.raises(cc.CoulombError) as e:
        cc.Batch([{"R": 6, "L": 10.0, "R_F": 7, "S": 32}])     # R_F > R
    assert e.value.status == 2


def test_mixed_batch_all_boxes(batch):
    """The tensor-core (bf16x3) form of the batched engine: every box within 1e-4."""
    import torch
    dev, boxes, B = batch
    eps = torch.full((int(B.offsets[-1]),), float("nan"), dtype=torch.float32, device=dev)
    Ex = torch.zeros((B.nbox, 2), dtype=torch.float64, device=dev)
    B.exchange(eps, Ex, precision="bf16x3")
    torch.cuda.synchronize()
    e = eps.cpu().numpy().astype(np.float64)
    x = Ex.cpu().numpy()
    assert not np.isnan(e).any()
    for i, b in enumerate(boxes):
        a, w = _nodes(b)
        C = ox.difference_histogram(b["R_F"], "fft")
        ref = ox.Ex_separable_periodic(b["R_F"], b["L"], a, w, C)
        assert abs(x[i, 0] - ref) < 1e-4 * abs(ref), (i, b)
    for i, b in enumerate(boxes):   # every grid point of every box
        a, w = _nodes(b)
        grid, _ = _box_eps(B, e, i, b["R"])
        ref = ox.eps_separable_grid(b["R"], b["R_F"], b["L"], a, w)
        assert np.array_equal(grid == 0, ref == 0), (i, b)
        assert rel_err(grid, ref) < 1e-4, (i, b)
    # replay through the captured graph gives the same bits
    eps2 = torch.empty_like(eps)
    Ex2 = torch.zeros_like(Ex)
    B.exchange(eps2, Ex2, precision="bf16x3")
    B.exchange(eps2, Ex2, precision="bf16x3")
    torch.cuda.synchronize()
    assert torch.equal(eps2, eps) and torch.equal(Ex2, Ex)


def test_mixed_batch_slab_kernel_vs_chain(batch):
    """The bf16x3 batch through the fused slab kernel (the automatic choice) against the same
    batch through the five-launch step chain, element by element, and E_x of every box."""
    import torch
    import paper_1502_08043_gb300 as cc
    dev, boxes, B = batch
    n = int(B.offsets[-1])
    eps_s = torch.full((n,), float("nan"), dtype=torch.float32, device=dev)
    Ex_s = torch.zeros((B.nbox, 2), dtype=torch.float64, device=dev)
    B.exchange(eps_s, Ex_s, precision="bf16x3")
    assert cc.lib().cc_set_mixed_variant(1) == 0
    try:  # fresh buffers: a graph of its own, captured with the chain
        eps_c = torch.full((n,), float("nan"), dtype=torch.float32, device=dev)
        Ex_c = torch.zeros((B.nbox, 2), dtype=torch.float64, device=dev)
        B.exchange(eps_c, Ex_c, precision="bf16x3")
        torch.cuda.synchronize()
    finally:
        assert cc.lib().cc_set_mixed_variant(0) == 0
    s = eps_s.cpu().numpy().astype(np.float64)
    c = eps_c.cpu().numpy().astype(np.float64)
    assert not np.isnan(s).any() and np.array_equal(s == 0, c == 0)
    nz = c != 0
    assert np.max(np.abs(s[nz] - c[nz]) / np.abs(c[nz])) < 1e-4
    xs, xc = Ex_s.cpu().numpy(), Ex_c.cpu().numpy()
    assert np.max(np.abs(xs[:, 0] - xc[:, 0]) / np.abs(xc[:, 0])) < 1e-4


def test_mixed_batch_tuner_keeps_results(batch):
    """The tensor-core engine's autotuner times every work decomposition (box order x cut of
    the unit sequence among the CTAs) and keeps the fastest.  Every decomposition sums the
    same products; only the grouping of the FP32 accumulation in tensor memory changes (the
    two runs differ by ~1e-5, the same level as their error against the FP64 oracle), so the
    tuned batch is checked against the oracle on every grid point of every box."""
    import torch
    dev, boxes, B = batch
    n = int(B.offsets[-1])
    e0 = torch.empty((n,), dtype=torch.float32, device=dev)
    x0 = torch.zeros((B.nbox, 2), dtype=torch.float64, device=dev)
    B.exchange(e0, x0, precision="bf16x3")
    torch.cuda.synchronize()
    e1 = torch.empty_like(e0)
    x1 = torch.zeros_like(x0)
    choice = B.tune(e1, x1, reps=2, precision="bf16x3")
    assert choice["order"] in ("as given", "by decreasing cost")
    assert choice["cut"] in ("equal units", "equal estimated cost") and choice["ms"] > 0
    e2 = torch.full_like(e0, float("nan"))
    x2 = torch.zeros_like(x0)
    B.exchange(e2, x2, precision="bf16x3")
    torch.cuda.synchronize()
    a = e0.cpu().numpy().astype(np.float64)
    b = e2.cpu().numpy().astype(np.float64)
    assert not np.isnan(b).any() and np.array_equal(a == 0, b == 0)
    nz = a != 0
    assert np.max(np.abs(a[nz] - b[nz]) / np.abs(a[nz])) < 1e-4
    xb = x2.cpu().numpy()
    for i, bx in enumerate(boxes):
        aa, ww = _nodes(bx)
        grid, _ = _box_eps(B, b, i, bx["R"])
        ref = ox.eps_separable_grid(bx["R"], bx["R_F"], bx["L"], aa, ww)
        assert np.array_equal(grid == 0, ref == 0), (i, bx)
        assert rel_err(grid, ref) < 1e-4, (i, bx)
        ex_ref = ox.Ex_separable_periodic(bx["R_F"], bx["L"], aa, ww,
                                          ox.difference_histogram(bx["R_F"], "fft"))
        assert abs(xb[i, 0] - ex_ref) < 1e-4 * abs(ex_ref), (i, bx)
