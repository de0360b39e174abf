"""GPU parity: exchange sums by Toeplitz mode products vs the FP64 oracle."""
import os

import numpy as np
import pytest

from gpu_common import (BOX_POINTS, CFG1, CFG2, CFG3, TOL_FP32, TOL_FP64, need_gpu, oracle_nodes,
                        rel_err)
from oracle import basis as ob
from oracle import exchange as ox
from oracle import quadrature as oq

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden", "table1.txt")


@pytest.fixture(scope="module")
def dev():
    return need_gpu()


def _exchange(t, R_F, prec, dev):
    import torch
    import paper_1502_08043_gb300 as cc
    Mg = t.info["Mg"]
    dt = torch.float64 if prec == "fp64" else torch.float32
    eps = torch.full((Mg ** 3,), float("nan"), dtype=dt, device=dev)
    Ex = torch.zeros(2, dtype=torch.float64, device=dev)
    cc.exchange_sums(t, R_F, eps, Ex, precision=prec)
    return eps.cpu().numpy().astype(np.float64).reshape(Mg, Mg, Mg), Ex.cpu().numpy()


def _basis_values(R, grid):
    k = ob.basis(R) + R
    return grid[k[:, 0], k[:, 1], k[:, 2]]


@pytest.mark.parametrize("prec,tol", [("fp64", TOL_FP64), ("fp32", TOL_FP32)])
def test_small_box(dev, prec, tol):
    import paper_1502_08043_gb300 as cc
    R, L, R_F = CFG1["R"], CFG1["L"], CFG1["R_F"]
    t = cc.build_tables("periodic", R=R, L=L, S=CFG1["S"])
    a, w = oracle_nodes(R, CFG1["S"])
    grid, Ex = _exchange(t, R_F, prec, dev)
    ref = ox.eps_separable(R, R_F, L, a, w)
    refg = ox.eps_on_grid(R, ref)
    assert np.array_equal(grid == 0, refg == 0)        # zero outside the basis sphere
    assert rel_err(_basis_values(R, grid), ref) < tol
    ex_ref = ox.Ex_separable_periodic(R_F, L, a, w)
    assert abs(Ex[0] - ex_ref) < tol * abs(ex_ref) and Ex[1] == 2 * Ex[0]
    # stated method error against the exact pair sums (S = 32 mesh)
    assert rel_err(_basis_values(R, grid), ox.eps_exact(R, R_F, L)) < 2e-5
    t.free()


def test_paper_scale(dev):
    import paper_1502_08043_gb300 as cc
    R, L, R_F = CFG2["R"], CFG2["L"], CFG2["R_F"]
    t = cc.build_tables("periodic", R=R, L=L, S=CFG2["S"])
    a, w = oracle_nodes(R, CFG2["S"])
    grid, Ex = _exchange(t, R_F, "fp32", dev)
    ref = ox.eps_separable(R, R_F, L, a, w)
    assert rel_err(_basis_values(R, grid), ref) < TOL_FP32
    ex_ref = ox.Ex_separable_periodic(R_F, L, a, w)
    assert abs(Ex[0] - ex_ref) < TOL_FP32 * abs(ex_ref)
    # stated method error of the 64-node mesh (oracle node sum vs exact pair sum), and the
    # FP32 result against the exact sum within method error + FP32 bound
    exact = ox.eps_exact(R, R_F, L)
    assert rel_err(ref, exact) < 3e-8
    assert rel_err(_basis_values(R, grid), exact) < TOL_FP32 + 3e-8
    t.free()


def test_precision_form_sampled(dev):
    import paper_1502_08043_gb300 as cc
    R, L, R_F = CFG3["R"], CFG3["L"], CFG3["R_F"]
    t = cc.build_tables("periodic", R=R, L=L, S=CFG3["S"])
    a, w = oracle_nodes(R, CFG3["S"])
    grid, Ex = _exchange(t, R_F, "fp32", dev)
    Nb = ob.count(R)
    rng = np.random.default_rng(3)
    idx = np.unique(np.concatenate([rng.integers(0, Nb, 1500), [0, Nb // 2, Nb - 1]]))
    ref = ox.eps_separable(R, R_F, L, a, w, k_idx=idx)
    assert rel_err(_basis_values(R, grid)[idx], ref) < TOL_FP32
    C = ox.difference_histogram(R_F, "fft")
    ex_ref = ox.Ex_separable_periodic(R_F, L, a, w, C)
    assert abs(Ex[0] - ex_ref) < TOL_FP32 * abs(ex_ref)
    t.free()


def _table1():
    rows = [l.split() for l in open(GOLD) if l.strip() and not l.startswith("#")]
    return [(m, int(q), float(i1), float(tt)) for m, q, i1, tt in rows]


@pytest.mark.parametrize("mesh,q,int1,total", _table1())
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_table1_on_gpu(dev, mesh, q, int1, total, prec):
    """Table I replayed by the GPU box-kernel mode products (M = 9171, L = 2)."""
    import paper_1502_08043_gb300 as cc
    R = 13
    if mesh == "mesh1":
        t = cc.build_tables("box", R=R, L=2.0, S=2 * q, n_sub=0, q_tail=q)
    else:
        t = cc.build_tables("box", R=R, L=2.0, S=8 * q + 90, n_sub=7, q_tail=90)
    grid, Ex = _exchange(t, 13, prec, dev)
    ratio = Ex[0] / ox.E_KS(9171, 2.0)
    assert abs(ratio - total) < (2e-6 if prec == "fp64" else 5e-6)
    t.free()


def test_fig1_on_gpu(dev):
    """Fig. 1 replayed on the GPU: E_x / E_KS for R_F = 1 .. 13 (periodic kernel, |n| <= 13)
    equals the oracle's node sum on the same nodes, rises with R_F, and extrapolates
    linearly in M^(-1/3) to 1."""
    import paper_1502_08043_gb300 as cc
    R, L = 13, 10.0
    t = cc.build_tables("periodic", R=R, L=L, S=64)
    a, w = oracle_nodes(R, 64)
    ratios, xs = [], []
    for R_F in range(1, 14):
        _, Ex = _exchange(t, R_F, "fp64", dev)
        C = ox.difference_histogram(R_F, "fft")
        ref = ox.Ex_separable_periodic(R_F, L, a, w, C)
        assert abs(Ex[0] - ref) < 1e-11 * abs(ref)
        M = ob.count(R_F)
        ratios.append(Ex[0] / ox.E_KS(M, L))
        xs.append(M ** (-1.0 / 3.0))
    assert all(np.diff(ratios) > 0)
    slope = (ratios[-1] - ratios[-2]) / (xs[-1] - xs[-2])
    assert abs(ratios[-1] - slope * xs[-1] - 1.0) < 0.01
    t.free()


def test_box_exchange_vs_oracle(dev):
    import paper_1502_08043_gb300 as cc
    R, R_F, L = 5, 3, 3.0
    ao, wo, _ = oq.paper_mesh2(6, 24)
    t = cc.build_tables("box", R=R, L=L, S=len(ao), n_sub=7, q_tail=24)
    ref = ox.eps_box(R, R_F, L, ao, wo, points=BOX_POINTS)
    for prec, tol in (("fp64", 1e-11), ("fp32", TOL_FP32)):
        grid, Ex = _exchange(t, R_F, prec, dev)
        assert rel_err(_basis_values(R, grid), ref) < tol
    t.free()


def test_exchange_errors(dev):
    import torch
    import paper_1502_08043_gb300 as cc
    t = cc.build_tables("periodic", R=4, L=10.0, S=32)
    eps = torch.empty(729, dtype=torch.float32, device=dev)
    Ex = torch.empty(2, dtype=torch.float64, device=dev)
    for R_F in (0, 5):
        with pytest.raises(cc.CoulombError) as e:
            cc.exchange_sums(t, R_F, eps, Ex)
        assert e.value.status == 2
    t.free()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_gemm_tile_autotuner(dev, prec):
    """The SIMT GEMM tile autotuner: times the dense chain with every tile pair and keeps the
    fastest for the grid side; every tile pair sums each output in the same order (16-wide K
    tiles, Kahan across them), so the results are bit-identical before and after tuning."""
    import torch
    import paper_1502_08043_gb300 as cc
    R, R_F, L, S = 27, 12, 25.0, 40
    t = cc.build_tables("periodic", R=R, L=L, S=S)
    Mg = t.info["Mg"]
    dt = torch.float64 if prec == "fp64" else torch.float32
    assert cc.lib().cc_set_simt_variant(1) == 0   # the dense chain (grid side 55 > 49)
    try:
        e0 = torch.empty(Mg ** 3, dtype=dt, device=dev)
        x0 = torch.zeros(2, dtype=torch.float64, device=dev)
        cc.exchange_sums(t, R_F, e0, x0, precision=prec)
        choice = cc.autotune_gemm(t, R_F, precision=prec, reps=2)
        assert choice["small"] in cc.TILES.values() and choice["large"] in cc.TILES.values()
        assert cc.gemm_tiles_tuned(prec, Mg) == {"small": choice["small"], "large": choice["large"]}
        e1 = torch.empty_like(e0)
        x1 = torch.zeros_like(x0)
        cc.exchange_sums(t, R_F, e1, x1, precision=prec)
        torch.cuda.synchronize()
        assert torch.equal(e0, e1) and torch.equal(x0, x1)
    finally:
        assert cc.lib().cc_set_simt_variant(0) == 0
    t.free()
