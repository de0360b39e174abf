"""GPU parity: the plain FP32 exchange at grid sides 50..127 by the slab algorithm on the
SIMT cores (window sums for the first mode product, the other two restricted to the band
where they do not vanish), against the FP64 oracle on every grid point, and against the
dense chain of SIMT GEMMs (the other FP32 form) element by element."""
import numpy as np
import pytest

from gpu_common import BOX_POINTS, TOL_FP32, need_gpu, oracle_nodes, rel_err
from oracle import basis as ob
from oracle import exchange as ox
from oracle import quadrature as oq

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    return need_gpu()


def _exchange(t, R_F, dev, variant=0):
    import torch
    import paper_1502_08043_gb300 as cc
    Mg = t.info["Mg"]
    eps = torch.full((Mg ** 3,), float("nan"), dtype=torch.float32, device=dev)
    Ex = torch.zeros(2, dtype=torch.float64, device=dev)
    assert cc.lib().cc_set_simt_variant(variant) == 0
    try:
        cc.exchange_sums(t, R_F, eps, Ex, precision="fp32")
        torch.cuda.synchronize()
    finally:
        assert cc.lib().cc_set_simt_variant(0) == 0
    return eps.cpu().numpy().astype(np.float64).reshape(Mg, Mg, Mg), Ex.cpu().numpy()


# (R, R_F, L, S): grid sides 51 .. 127; bands narrow (2 R_F + 1 = 21) to full (127)
CASES = [(25, 25, 15.0, 48), (31, 20, 40.0, 96), (40, 10, 30.0, 64), (48, 33, 35.0, 80),
         (63, 40, 60.0, 128), (63, 63, 60.0, 64)]


@pytest.mark.parametrize("R,R_F,L,S", CASES)
def test_simt_slab_full_grid_vs_oracle(dev, R, R_F, L, S):
    import paper_1502_08043_gb300 as cc
    t = cc.build_tables("periodic", R=R, L=L, S=S)
    a, w = oracle_nodes(R, S)
    grid, Ex = _exchange(t, R_F, dev)
    ref = ox.eps_separable_grid(R, R_F, L, a, w)
    assert not np.isnan(grid).any()
    assert np.array_equal(grid == 0, ref == 0)
    assert rel_err(grid, ref) < TOL_FP32
    C = ox.difference_histogram(R_F, "fft")
    ex_ref = ox.Ex_separable_periodic(R_F, L, a, w, C)
    assert abs(Ex[0] - ex_ref) < TOL_FP32 * abs(ex_ref) and Ex[1] == 2 * Ex[0]
    # the dense GEMM chain computes the same sums in another order
    dense, Ex_d = _exchange(t, R_F, dev, variant=1)
    assert rel_err(grid, dense) < 2 * TOL_FP32
    t.free()


def test_simt_slab_box_kernel(dev):
    import paper_1502_08043_gb300 as cc
    R, R_F, L = 33, 21, 2.0
    ao, wo, _ = oq.paper_mesh2(3, 12)
    t = cc.build_tables("box", R=R, L=L, S=len(ao), n_sub=7, q_tail=12)
    grid, Ex = _exchange(t, R_F, dev)
    Nb = ob.count(R)
    idx = np.unique(np.random.default_rng(5).integers(0, Nb, 300))
    ref = ox.eps_box(R, R_F, L, ao, wo, k_idx=idx, points=BOX_POINTS)
    k = ob.basis(R)[idx] + R
    assert rel_err(grid[k[:, 0], k[:, 1], k[:, 2]], ref) < TOL_FP32
    dense, _ = _exchange(t, R_F, dev, variant=1)
    assert rel_err(grid, dense) < 2 * TOL_FP32
    t.free()


def test_simt_variant_argument():
    import paper_1502_08043_gb300 as cc
    need_gpu()
    assert cc.lib().cc_set_simt_variant(2) == 1 and cc.lib().cc_set_simt_variant(-1) == 1
