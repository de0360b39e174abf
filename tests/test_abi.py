"""The C-ABI library loads and exports every symbol declared in include/*.h (CPU only:
no call here touches a GPU)."""
import glob
import os
import re
import ctypes

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names |= set(re.findall(r"^\s*(?:cc_status|const char\*)\s+(cc_\w+)\s*\(", txt, re.M))
    return names


@pytest.fixture(scope="module")
def lib():
    import paper_1502_08043_gb300 as cc
    from paper_1502_08043_gb300 import build as b
    b.build()
    return cc


def test_every_declared_symbol_is_exported(lib):
    declared = _declared()
    assert len(declared) >= 14
    L = ctypes.CDLL(lib.LIB_PATH)
    for name in declared:
        assert hasattr(L, name), name
    # the binding declares exactly the header's entry points
    assert declared == set(lib.SIGNATURES)


def test_status_strings_and_host_basis(lib):
    L = lib.lib()
    assert L.cc_status_string(0) == b"ok"
    assert L.cc_status_string(6) == b"not supported"
    from oracle import basis as ob
    for R in (1, 4, 13):
        v = lib.basis(R)
        assert np.array_equal(v[:, :3].astype(np.int64), ob.basis(R))
        assert np.all(v[:, 3] == 0)
    with pytest.raises(lib.CoulombError):
        lib.basis(0)
    with pytest.raises(lib.CoulombError):
        lib.basis(128)


def test_product_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1502_08043_gb300")
    for f in glob.glob(os.path.join(pkg, "**", "*.*"), recursive=True):
        if f.endswith((".py", ".cu", ".cuh", ".h")):
            txt = open(f).read()
            assert "import oracle" not in txt and "from oracle" not in txt, f


def test_library_mesh_rule_equals_oracle_rule(lib):
    """The default mesh search of the library (host code) and of the oracle pick the same
    (n_sub, q_tail) for every box of the batched workload and for assorted cases."""
    import coulomb_inputs as ci
    from oracle import quadrature as oq
    cases = {(b["S"], b["R"]) for b in ci.box_params(256)}
    cases |= {(32, 4), (64, 13), (96, 31), (128, 63), (40, 9), (17, 2), (36, 5), (4, 3), (2, 1)}
    for S, R in sorted(cases):
        assert lib.default_mesh(S, R) == oq.default_periodic_mesh(S, R), (S, R)


def test_library_mesh_for_error_equals_oracle(lib):
    """Fewest nodes for a stated method error (the inverse of the default rule): library
    and oracle give the same (S, n_sub, q_tail); that mesh reaches the target and the
    default mesh of S - 1 nodes does not."""
    from oracle import quadrature as oq
    for R in (4, 13, 31):
        for target in (1e-4, 1e-7):
            got = lib.mesh_for_error(R, target, 200)
            ref = oq.mesh_for_error(R, target, 200)
            assert ref is not None, (R, target)
            assert got[:3] == ref[:3], (R, target, got, ref)
            assert got[3] <= target and abs(got[3] - ref[3]) <= 1e-9 * target + 1e-15
            S = got[0]
            if S > 2:
                n, q = oq.default_periodic_mesh(S - 1, R)
                assert oq.mesh_error(S - 1, n, q, R) > target
    with pytest.raises(lib.CoulombError):
        lib.mesh_for_error(4, 1e-30, 8)   # not reachable with 8 nodes
    with pytest.raises(lib.CoulombError):
        lib.mesh_for_error(4, -1.0, 8)


def test_library_mesh_tune_equals_oracle(lib):
    """Mesh tuning over the wider family (sub-interval ratio, alpha_c): library and oracle
    pick the same mesh; it reaches the target with at most the default rule's node count,
    and no candidate of the family with one node fewer in the searched range does."""
    from oracle import quadrature as oq
    for R, target in ((4, 1e-5), (13, 1e-7), (13, 1e-8)):
        got = lib.mesh_tune(R, target, 200)
        ref = oq.mesh_tune(R, target, 200)
        assert ref is not None
        assert got[:3] == ref[:3] and got[3:5] == ref[3:5], (R, target, got, ref)
        # the two errors are the same quantity from two Gauss-Legendre constructions summed
        # in different orders: they agree to FP64 rounding of sums of order 1
        assert got[5] <= target and abs(got[5] - ref[5]) <= 1e-13
        S_d = oq.mesh_for_error(R, target, 200)[0]
        assert got[0] <= S_d
        # the mesh itself: its error recomputed from the oracle's nodes
        assert oq.mesh_error(got[0], got[1], got[2], R, got[3], got[4]) <= target
    # ratio 5 and alpha_c 1 give the nodes of the paper's geometric split (Mesh 2 edges)
    a1, w1, _ = oq.laplace_mesh(48, 7, 8)
    a2, w2, _ = oq.laplace_mesh(48, 7, 8, 1.0, 5.0)
    assert np.array_equal(a1, a2) and np.array_equal(w1, w2)
    edges = oq.interval1_edges(3, 2.0, 4.0)
    assert np.allclose(edges, [0.0, 2.0 / 64, 2.0 / 16, 2.0 / 4, 2.0], rtol=0, atol=0)
    with pytest.raises(lib.CoulombError):
        lib.mesh_tune(4, 1e-30, 8)
