"""GPU parity: the small-grid tensor-core exchange (bf16x3, grid sides up to 64: two slabs
share every 128-row MMA, R^T x T then U x T with U as an MN-major operand), against the
FP64 oracle on every grid point and E_x, and element by element against the five-launch
step chain and the 128-row slab kernel on the same handle."""
import numpy as np
import pytest

from gpu_common import BOX_POINTS, need_gpu, oracle_nodes, rel_err
from oracle import basis as ob
from oracle import exchange as ox
from oracle import quadrature as oq

pytestmark = pytest.mark.gpu
TOL_MIXED = 1e-4


@pytest.fixture(scope="module")
def dev():
    return need_gpu()


def _run(t, R_F, dev, variant):
    import torch
    import paper_1502_08043_gb300 as cc
    Mg = t.info["Mg"]
    eps = torch.full((Mg ** 3,), float("nan"), dtype=torch.float32, device=dev)
    Ex = torch.zeros(2, dtype=torch.float64, device=dev)
    assert cc.lib().cc_set_mixed_variant(variant) == 0
    try:
        cc.exchange_sums(t, R_F, eps, Ex, precision="bf16x3")
        torch.cuda.synchronize()
        assert cc.mixed_status(t) == 0
    finally:
        assert cc.lib().cc_set_mixed_variant(0) == 0
    return eps.cpu().numpy().astype(np.float64).reshape(Mg, Mg, Mg), Ex.cpu().numpy()


# (R, R_F, L, S): grid sides 3 .. 63; bands of 3 .. 63 rows; the |n| <= 31 workload
PERIODIC = [(1, 1, 5.0, 8), (4, 2, 10.0, 32), (13, 8, 20.0, 64), (25, 5, 30.0, 48),
            (31, 20, 40.0, 96), (31, 31, 40.0, 64), (22, 17, 25.0, 40)]


@pytest.mark.parametrize("R,R_F,L,S", PERIODIC)
def test_small_kernel_periodic_full_grid(dev, R, R_F, L, S):
    import paper_1502_08043_gb300 as cc
    t = cc.build_tables("periodic", R=R, L=L, S=S)
    a, w = oracle_nodes(R, S)
    g, e = _run(t, R_F, dev, 3)
    ref = ox.eps_separable_grid(R, R_F, L, a, w)
    assert not np.isnan(g).any()
    assert np.array_equal(g == 0, ref == 0)
    assert rel_err(g, ref) < TOL_MIXED
    C = ox.difference_histogram(R_F, "fft")
    ex_ref = ox.Ex_separable_periodic(R_F, L, a, w, C)
    assert abs(e[0] - ex_ref) < TOL_MIXED * abs(ex_ref) and e[1] == 2 * e[0]
    # the automatic choice is this kernel; the step chain agrees element by element
    g0, e0 = _run(t, R_F, dev, 0)
    assert np.array_equal(g0, g) and np.array_equal(e0, e)
    gc, _ = _run(t, R_F, dev, 1)
    assert rel_err(g, gc) < TOL_MIXED
    if R >= 13:   # the 128-row slab kernel (grid sides >= 27 in its tests)
        gs, _ = _run(t, R_F, dev, 2)
        assert rel_err(g, gs) < TOL_MIXED
    t.free()


def test_small_kernel_box(dev):
    import paper_1502_08043_gb300 as cc
    R, R_F, L = 20, 12, 2.0
    a, w, _ = oq.paper_mesh2(5, 20)
    t = cc.build_tables("box", R=R, L=L, S=len(a), n_sub=7, q_tail=20)
    g, e = _run(t, R_F, dev, 3)
    Nb = ob.count(R)
    idx = np.unique(np.concatenate([np.random.default_rng(9).integers(0, Nb, 300), [0, Nb - 1]]))
    ref = ox.eps_box(R, R_F, L, a, w, k_idx=idx, points=BOX_POINTS)
    k = ob.basis(R)[idx] + R
    assert rel_err(g[k[:, 0], k[:, 1], k[:, 2]], ref) < TOL_MIXED
    C = ox.difference_histogram(R_F, "fft")
    ex_ref = ox.Ex_box(R_F, L, a, w, C, table=None)
    assert abs(e[0] - ex_ref) < TOL_MIXED * abs(ex_ref)
    gc, _ = _run(t, R_F, dev, 1)
    assert np.array_equal(g == 0, gc == 0) and rel_err(g, gc) < TOL_MIXED
    t.free()


def test_small_kernel_bounded_wait(dev):
    """The stall hook on the small-grid kernel: error word 5, context usable afterwards."""
    import torch
    import paper_1502_08043_gb300 as cc
    R, L, R_F = 13, 20.0, 8
    t = cc.build_tables("periodic", R=R, L=L, S=64)
    Mg = t.info["Mg"]
    g0, e0 = _run(t, R_F, dev, 0)
    eps = torch.empty(Mg ** 3, dtype=torch.float32, device=dev)
    Ex = torch.zeros(2, dtype=torch.float64, device=dev)
    assert cc.lib().cc_test_stall_next_mixed() == 0
    cc.exchange_sums(t, R_F, eps, Ex, precision="bf16x3")
    torch.cuda.synchronize()
    assert cc.mixed_status(t) == 5
    assert cc.mixed_status(t) == 0
    g1, e1 = _run(t, R_F, dev, 0)
    assert np.array_equal(g0, g1) and np.array_equal(e0, e1)
    t.free()


def test_small_kernel_rejects_large_grids(dev):
    import torch
    import paper_1502_08043_gb300 as cc
    t = cc.build_tables("periodic", R=33, L=30.0, S=32)
    Mg = t.info["Mg"]
    eps = torch.empty(Mg ** 3, dtype=torch.float32, device=dev)
    Ex = torch.zeros(2, dtype=torch.float64, device=dev)
    assert cc.lib().cc_set_mixed_variant(3) == 0
    try:
        with pytest.raises(cc.CoulombError) as e:
            cc.exchange_sums(t, 20, eps, Ex, precision="bf16x3")
        assert e.value.status == 6
    finally:
        assert cc.lib().cc_set_mixed_variant(0) == 0
    t.free()


@pytest.mark.parametrize("R,R_F,S", [(13, 8, 64), (33, 21, 64)])
def test_lo_plane_correction(dev, R, R_F, S):
    """What the split precision buys: with the lo planes (hi*hi + hi*lo + lo*hi) the
    tensor-core exchange is within 1e-4 of the FP64 node sum; with hi*hi only (the plain
    bf16 product) it is off by about the bf16 rounding, 2^-9 .. 2^-8 relative, and at least
    ten times worse.  Grid side 27 runs the small-grid kernel, 67 the 128-row kernel."""
    import paper_1502_08043_gb300 as cc
    L = 30.0
    t = cc.build_tables("periodic", R=R, L=L, S=S)
    a, w = oracle_nodes(R, S)
    ref = ox.eps_separable_grid(R, R_F, L, a, w)
    g3, _ = _run(t, R_F, dev, 0)
    assert cc.lib().cc_set_mixed_terms(1) == 0
    try:
        g1, _ = _run(t, R_F, dev, 0)
    finally:
        assert cc.lib().cc_set_mixed_terms(3) == 0
    e3, e1 = rel_err(g3, ref), rel_err(g1, ref)
    assert e3 < TOL_MIXED and e1 > 10 * e3 and 1e-4 < e1 < 1e-2, (e3, e1)
    assert cc.lib().cc_set_mixed_terms(2) == 1
    t.free()
