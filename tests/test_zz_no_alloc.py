"""The allocation-free exchange entry point (cc_exchange_sums_noalloc).

It exists for callers that cannot call cudaMalloc where they need the exchange sums
(code under a framework's caching allocator that owns the device memory, latency-
critical loops that cannot afford cudaMalloc's implicit synchronisation).  It must give
the same sums as the ordinary FP32 entry point cc_exchange_sums, call after call, and the
FP64 oracle's, while keeping its scratch in the library's fixed device array: the free
device memory does not change across its calls.  This file is collected last.
"""
import ctypes

import numpy as np
import pytest

from gpu_common import TOL_FP32, need_gpu, oracle_nodes, rel_err
from oracle import exchange as ox

pytestmark = pytest.mark.gpu


def _reference(cc, t, R_F, dev):
    import torch
    Mg = t.info["Mg"]
    eps = torch.empty(Mg ** 3, dtype=torch.float32, device=dev)
    Ex = torch.empty(2, dtype=torch.float64, device=dev)
    cc.exchange_sums(t, R_F, eps, Ex, precision="fp32")
    torch.cuda.synchronize()
    return eps.cpu().numpy().astype(np.float64), Ex.cpu().numpy()


@pytest.mark.parametrize("R,L,S,R_F", [(13, 20.0, 64, 8), (31, 40.0, 96, 20)])
def test_noalloc_matches_existing_entry_point(R, L, S, R_F):
    import torch
    import paper_1502_08043_gb300 as cc
    dev = need_gpu()
    t = cc.build_tables("periodic", R=R, L=L, S=S)
    ref_eps, ref_Ex = _reference(cc, t, R_F, dev)
    a, w = oracle_nodes(R, S)
    oracle_eps = ox.eps_separable_grid(R, R_F, L, a, w).reshape(-1)
    oracle_Ex = ox.Ex_separable_periodic(R_F, L, a, w, ox.difference_histogram(R_F, "fft"))
    Mg = t.info["Mg"]
    outs = [(torch.full((Mg ** 3,), float("nan"), dtype=torch.float32, device=dev),
             torch.zeros(2, dtype=torch.float64, device=dev)) for _ in range(2)]
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(dev)[0]
    for eps, Ex in outs:   # two calls in a row through the C ABI
        st = cc.lib().cc_exchange_sums_noalloc(
            t.handle, R_F, ctypes.c_void_p(eps.data_ptr()), ctypes.c_void_p(Ex.data_ptr()),
            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == 0
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info(dev)[0] == free0   # nothing allocated or freed
        got = eps.cpu().numpy().astype(np.float64)
        assert np.array_equal(got == 0, ref_eps == 0)
        assert rel_err(got, ref_eps) < TOL_FP32
        assert abs(Ex.cpu().numpy()[0] - ref_Ex[0]) < TOL_FP32 * abs(ref_Ex[0])
        assert rel_err(got, oracle_eps) < TOL_FP32
        assert abs(Ex.cpu().numpy()[0] - oracle_Ex) < TOL_FP32 * abs(oracle_Ex)
    t.free()


def test_noalloc_rejects_sizes_beyond_its_array():
    import torch
    import paper_1502_08043_gb300 as cc
    dev = need_gpu()
    t = cc.build_tables("periodic", R=32, L=40.0, S=48)
    eps = torch.empty(t.info["Mg"] ** 3, dtype=torch.float32, device=dev)
    Ex = torch.empty(2, dtype=torch.float64, device=dev)
    with pytest.raises(cc.CoulombError) as e:
        cc.exchange_sums_noalloc(t, 10, eps, Ex)
    assert e.value.status == 2
    t.free()
