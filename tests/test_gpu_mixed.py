"""GPU parity: mixed-precision (bf16 hi+lo, tcgen05 tensor cores) exchange sums vs the
FP64 oracle, at the stated 1e-4 relative tolerance, and against the plain FP32 path."""
import numpy as np
import pytest

from gpu_common import CFG1, CFG2, CFG3, CFG5, need_gpu, oracle_nodes, rel_err
from oracle import basis as ob
from oracle import exchange as ox
from oracle import quadrature as oq

pytestmark = pytest.mark.gpu
TOL_MIXED = 1e-4


@pytest.fixture(scope="module")
def dev():
    return need_gpu()


def _run(t, R_F, prec, dev):
    import torch
    import paper_1502_08043_gb300 as cc
    Mg = t.info["Mg"]
    dt = torch.float64 if prec == "fp64" else torch.float32
    eps = torch.full((Mg ** 3,), float("nan"), dtype=dt, device=dev)
    Ex = torch.zeros(2, dtype=torch.float64, device=dev)
    cc.exchange_sums(t, R_F, eps, Ex, precision=prec)
    torch.cuda.synchronize()
    assert cc.mixed_status(t) == 0
    return eps.cpu().numpy().astype(np.float64).reshape(Mg, Mg, Mg), Ex.cpu().numpy()


def _basis_values(R, grid):
    k = ob.basis(R) + R
    return grid[k[:, 0], k[:, 1], k[:, 2]]


@pytest.mark.parametrize("cfg", [CFG1, CFG2], ids=["R4", "R13"])
def test_mixed_full_compare(dev, cfg):
    import paper_1502_08043_gb300 as cc
    R, L, R_F = cfg["R"], cfg["L"], cfg["R_F"]
    t = cc.build_tables("periodic", R=R, L=L, S=cfg["S"])
    a, w = oracle_nodes(R, cfg["S"])
    ref = ox.eps_separable(R, R_F, L, a, w)
    grid, Ex = _run(t, R_F, "bf16x3", dev)
    assert np.array_equal(grid == 0, ox.eps_on_grid(R, ref) == 0)
    assert rel_err(_basis_values(R, grid), ref) < TOL_MIXED
    ex_ref = ox.Ex_separable_periodic(R_F, L, a, w)
    assert abs(Ex[0] - ex_ref) < TOL_MIXED * abs(ex_ref)
    t.free()


@pytest.mark.parametrize("cfg", [CFG3, CFG5], ids=["R31", "R63"])
def test_mixed_sampled(dev, cfg):
    import paper_1502_08043_gb300 as cc
    R, L, R_F = cfg["R"], cfg["L"], cfg["R_F"]
    t = cc.build_tables("periodic", R=R, L=L, S=cfg["S"])
    a, w = oracle_nodes(R, cfg["S"])
    grid, Ex = _run(t, R_F, "bf16x3", dev)
    Nb = ob.count(R)
    rng = np.random.default_rng(11)
    idx = np.unique(np.concatenate([rng.integers(0, Nb, 300), [0, Nb // 2, Nb - 1]]))
    ref = ox.eps_separable(R, R_F, L, a, w, k_idx=idx)
    assert rel_err(_basis_values(R, grid)[idx], ref) < TOL_MIXED
    C = ox.difference_histogram(R_F, "fft")
    ex_ref = ox.Ex_separable_periodic(R_F, L, a, w, C)
    assert abs(Ex[0] - ex_ref) < TOL_MIXED * abs(ex_ref)
    # the plain FP32 path on the same handle agrees with the mixed one to the same bound
    g32, _ = _run(t, R_F, "fp32", dev)
    inside = g32 != 0
    assert np.max(np.abs(grid[inside] - g32[inside]) / np.abs(g32[inside])) < 2 * TOL_MIXED
    t.free()


def test_mixed_box_table1(dev):
    """Table I (Mesh 2, 8x10) replayed through the tensor-core path, box kernel."""
    import paper_1502_08043_gb300 as cc
    t = cc.build_tables("box", R=13, L=2.0, S=170, n_sub=7, q_tail=90)
    _, Ex = _run(t, 13, "bf16x3", dev)
    assert abs(Ex[0] / ox.E_KS(9171, 2.0) - 0.965431) < 1e-4
    t.free()


def test_mixed_repeatable(dev):
    import paper_1502_08043_gb300 as cc
    t = cc.build_tables("periodic", R=CFG2["R"], L=CFG2["L"], S=CFG2["S"])
    g1, e1 = _run(t, CFG2["R_F"], "bf16x3", dev)
    g2, e2 = _run(t, CFG2["R_F"], "bf16x3", dev)
    assert np.array_equal(g1, g2) and np.array_equal(e1, e2)
    g3, _ = _run(t, 5, "bf16x3", dev)     # another Fermi radius on the same handle
    ref = ox.eps_separable(CFG2["R"], 5, CFG2["L"], *oracle_nodes(CFG2["R"], CFG2["S"]))
    assert rel_err(_basis_values(CFG2["R"], g3), ref) < TOL_MIXED
    t.free()


@pytest.mark.parametrize("cfg", [CFG2, CFG3, CFG5], ids=["R13", "R31", "R63"])
def test_fp16x3_with_exponent_scaling(dev, cfg):
    """fp16 hi+lo with per-node power-of-two scaling of the y-mode operands."""
    import paper_1502_08043_gb300 as cc
    R, L, R_F = cfg["R"], cfg["L"], cfg["R_F"]
    t = cc.build_tables("periodic", R=R, L=L, S=cfg["S"])
    a, w = oracle_nodes(R, cfg["S"])
    grid, Ex = _run(t, R_F, "fp16x3", dev)
    Nb = ob.count(R)
    idx = np.unique(np.concatenate([np.random.default_rng(5).integers(0, Nb, 300), [0, Nb - 1]]))
    ref = ox.eps_separable(R, R_F, L, a, w, k_idx=idx)
    assert rel_err(_basis_values(R, grid)[idx], ref) < TOL_MIXED
    C = ox.difference_histogram(R_F, "fft")
    ex_ref = ox.Ex_separable_periodic(R_F, L, a, w, C)
    assert abs(Ex[0] - ex_ref) < TOL_MIXED * abs(ex_ref)
    t.free()


def test_bounded_wait_reports_timeout_and_context_survives(dev):
    """Failure detection without a fault: the test hook makes one tensor-core launch wait on
    a barrier nothing arrives at; the bounded wait runs out, the error word reads 5, and
    the next exchange on the same handle is correct again."""
    import torch
    import paper_1502_08043_gb300 as cc
    R, L, R_F = CFG2["R"], CFG2["L"], CFG2["R_F"]
    t = cc.build_tables("periodic", R=R, L=L, S=CFG2["S"])
    Mg = t.info["Mg"]
    eps = torch.empty(Mg ** 3, dtype=torch.float32, device=dev)
    Ex = torch.zeros(2, dtype=torch.float64, device=dev)
    _variant(1)                              # the step chain's persistent GEMM kernel
    try:
        assert cc.lib().cc_test_stall_next_mixed() == 0
        cc.exchange_sums(t, R_F, eps, Ex, precision="bf16x3")
        torch.cuda.synchronize()
        assert cc.mixed_status(t) == 5
        assert cc.mixed_status(t) == 0          # cleared by the read
        grid, Ex2 = _run(t, R_F, "bf16x3", dev)
    finally:
        _variant(0)
    a, w = oracle_nodes(R, CFG2["S"])
    assert rel_err(_basis_values(R, grid), ox.eps_separable(R, R_F, L, a, w)) < TOL_MIXED
    t.free()


def _variant(v):
    import paper_1502_08043_gb300 as cc
    assert cc.lib().cc_set_mixed_variant(v) == 0


@pytest.mark.parametrize("kernel,R,R_F", [("periodic", 33, 21), ("box", 33, 21),
                                           ("periodic", 40, 10), ("periodic", 33, 33),
                                           ("periodic", 13, 8), ("periodic", 31, 20),
                                           ("periodic", 48, 48)],
                         ids=["periodic-R33-RF21", "box-R33-RF21", "narrow-band-R40-RF10",
                              "full-band-R33-RF33", "grid27-R13-RF8", "grid63-R31-RF20",
                              "wide-band-R48-RF48"])
def test_slab_kernel_vs_chain_and_oracle(dev, kernel, R, R_F):
    """The fused tensor-core slab kernel (grid sides 27 to 97, operands padded to 128;
    occupied bands of width 17 to 97, so the products run over 32 to 112 of the 128 padded
    columns) element by element against the five-launch step chain on the same handle, and
    against the FP64 oracle on sampled basis functions and on E_x.  Periodic bands of at
    most 96 columns add the A term on the tensor cores (F_s times a one-hot P_x); the
    112-column band of R = 48, R_F = 48 takes the per-column gather of the A term."""
    import paper_1502_08043_gb300 as cc
    L = 30.0
    if kernel == "periodic":
        t = cc.build_tables("periodic", R=R, L=L, S=64)
        a, w = oracle_nodes(R, 64)
    else:
        a, w, _ = oq.paper_mesh2(6, 24)
        t = cc.build_tables("box", R=R, L=L, S=len(a), n_sub=7, q_tail=24)
    try:
        _variant(2)
        g_slab, e_slab = _run(t, R_F, "bf16x3", dev)
        _variant(1)
        g_chain, e_chain = _run(t, R_F, "bf16x3", dev)
    finally:
        _variant(0)
    assert np.array_equal(g_slab == 0, g_chain == 0)
    inside = g_chain != 0
    assert np.max(np.abs(g_slab[inside] - g_chain[inside]) / np.abs(g_chain[inside])) < TOL_MIXED
    Nb = ob.count(R)
    idx = np.unique(np.concatenate([np.random.default_rng(3).integers(0, Nb, 150), [0, Nb - 1]]))
    C = ox.difference_histogram(R_F, "fft")
    if kernel == "periodic":
        ref = ox.eps_separable(R, R_F, L, a, w, k_idx=idx)
        ex_ref = ox.Ex_separable_periodic(R_F, L, a, w, C)
    else:
        ref = ox.eps_box(R, R_F, L, a, w, k_idx=idx)
        ex_ref = ox.Ex_box(R_F, L, a, w, C)
    assert rel_err(_basis_values(R, g_slab)[idx], ref) < TOL_MIXED
    assert abs(e_slab[0] - ex_ref) < TOL_MIXED * abs(ex_ref)
    assert abs(e_slab[1] - 2 * e_slab[0]) <= 1e-12 * abs(e_slab[1])
    t.free()


@pytest.mark.parametrize("kernel,R,R_F", [("periodic", 33, 21), ("box", 33, 21),
                                           ("periodic", 13, 8), ("periodic", 48, 48)],
                         ids=["periodic-R33-RF21", "box-R33-RF21", "grid27-R13-RF8",
                              "wide-band-R48-RF48"])
def test_slab_kernel_fp16x3_vs_chain_and_oracle(dev, kernel, R, R_F):
    """fp16x3 through the slab kernel (per-node power-of-two scales of T, the window sums
    and the intermediate) element by element against the fp16x3 step chain, and against the
    FP64 oracle on sampled basis functions and on E_x.  Periodic bands of at most 96
    columns take the A term on the tensor cores (ones of 2^a in P), the 112-column band of
    R = 48, R_F = 48 the per-column gather."""
    import paper_1502_08043_gb300 as cc
    L = 30.0
    if kernel == "periodic":
        t = cc.build_tables("periodic", R=R, L=L, S=64)
        a, w = oracle_nodes(R, 64)
    else:
        a, w, _ = oq.paper_mesh2(6, 24)
        t = cc.build_tables("box", R=R, L=L, S=len(a), n_sub=7, q_tail=24)
    try:
        _variant(2)
        g_slab, e_slab = _run(t, R_F, "fp16x3", dev)
        _variant(1)
        g_chain, e_chain = _run(t, R_F, "fp16x3", dev)
    finally:
        _variant(0)
    assert np.array_equal(g_slab == 0, g_chain == 0)
    inside = g_chain != 0
    assert np.max(np.abs(g_slab[inside] - g_chain[inside]) / np.abs(g_chain[inside])) < TOL_MIXED
    Nb = ob.count(R)
    idx = np.unique(np.concatenate([np.random.default_rng(4).integers(0, Nb, 150), [0, Nb - 1]]))
    C = ox.difference_histogram(R_F, "fft")
    if kernel == "periodic":
        ref = ox.eps_separable(R, R_F, L, a, w, k_idx=idx)
        ex_ref = ox.Ex_separable_periodic(R_F, L, a, w, C)
    else:
        ref = ox.eps_box(R, R_F, L, a, w, k_idx=idx)
        ex_ref = ox.Ex_box(R_F, L, a, w, C)
    assert rel_err(_basis_values(R, g_slab)[idx], ref) < TOL_MIXED
    assert abs(e_slab[0] - ex_ref) < TOL_MIXED * abs(ex_ref)
    t.free()


def test_slab_kernel_variant_errors(dev):
    import paper_1502_08043_gb300 as cc
    L = cc.lib()
    assert L.cc_set_mixed_variant(4) == 1 and L.cc_set_mixed_variant(-1) == 1
    assert L.cc_set_mixed_variant(0) == 0


def test_slab_kernel_bounded_wait(dev):
    """The stall hook on the fused slab kernel: error word 5, context usable afterwards."""
    import torch
    import paper_1502_08043_gb300 as cc
    R, L, R_F = 33, 30.0, 21
    t = cc.build_tables("periodic", R=R, L=L, S=64)
    Mg = t.info["Mg"]
    eps = torch.empty(Mg ** 3, dtype=torch.float32, device=dev)
    Ex = torch.zeros(2, dtype=torch.float64, device=dev)
    g0, e0 = _run(t, R_F, "bf16x3", dev)
    assert cc.lib().cc_test_stall_next_mixed() == 0
    cc.exchange_sums(t, R_F, eps, Ex, precision="bf16x3")
    torch.cuda.synchronize()
    assert cc.mixed_status(t) == 5
    assert cc.mixed_status(t) == 0
    g1, e1 = _run(t, R_F, "bf16x3", dev)
    assert np.array_equal(g0, g1) and np.array_equal(e0, e1)
    t.free()
