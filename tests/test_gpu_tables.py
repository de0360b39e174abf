"""GPU parity: node sets, weights and tables built on the device vs the oracle."""
import numpy as np
import pytest

from gpu_common import need_gpu
from oracle import coulomb as oc
from oracle import quadrature as oq

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    return need_gpu()


@pytest.mark.parametrize("S,R,L", [(32, 4, 10.0), (64, 13, 20.0), (96, 31, 40.0),
                                   (128, 63, 60.0), (40, 9, 12.0), (17, 2, 3.0)])
def test_periodic_nodes_and_tables(dev, S, R, L):
    import paper_1502_08043_gb300 as cc
    t = cc.build_tables("periodic", R=R, L=L, S=S)
    n_sub, q_tail = oq.default_periodic_mesh(S, R)
    assert (t.info["n_sub"], t.info["q_tail"]) == (n_sub, q_tail)
    a, w, part, kept = t.nodes()
    ao, wo, po = oq.laplace_mesh(S, n_sub, q_tail)
    assert np.array_equal(part, po)
    assert np.max(np.abs(a - ao) / ao) < 1e-13
    assert np.max(np.abs(w - wo) / wo) < 1e-12
    ko = oq.prune_periodic(ao, wo, R, 1e-9)
    assert np.array_equal(kept, ko)
    assert t.info["S_eff"] == ko.sum()
    assert np.max(np.abs(t.values() - oc.periodic_table(ao[ko], 2 * R))) < 1e-14
    t.free()


@pytest.mark.parametrize("mesh,q", [("mesh1", 90), ("mesh2", 10), ("mesh2", 5)])
def test_box_tables(dev, mesh, q):
    import paper_1502_08043_gb300 as cc
    R, L = 13, 2.0
    ao, wo, po = oq.paper_mesh1(q) if mesh == "mesh1" else oq.paper_mesh2(q)
    S = len(ao)
    n_sub = 0 if mesh == "mesh1" else 7
    q_tail = q if mesh == "mesh1" else 90
    t = cc.build_tables("box", R=R, L=L, S=S, n_sub=n_sub, q_tail=q_tail)
    a, w, part, kept = t.nodes()
    assert kept.all() and np.array_equal(part, po)
    assert np.max(np.abs(a - ao) / ao) < 1e-13 and np.max(np.abs(w - wo) / wo) < 1e-12
    T = t.values()
    To = oc.box_table(ao, 2 * R, L)
    assert np.max(np.abs(T - To)) < 1e-12 * np.abs(To).max()
    t.free()


def test_save_load_roundtrip(dev, tmp_path):
    import torch
    import paper_1502_08043_gb300 as cc
    t = cc.build_tables("periodic", R=5, L=9.0, S=36)
    p = tmp_path / "tab.cctb"
    t.save(p)
    u = cc.load_tables(p)
    assert u.info == t.info
    for x, y in zip(t.nodes(), u.nodes()):
        assert np.array_equal(x, y)
    assert np.array_equal(t.values(), u.values())
    q = torch.randint(0, t.info["Nb"], (999, 4), dtype=torch.int32, device=dev)
    o1 = torch.empty(999, dtype=torch.float32, device=dev)
    o2 = torch.empty_like(o1)
    cc.reconstruct_integrals(t, q, o1)
    cc.reconstruct_integrals(u, q, o2)
    assert torch.equal(o1, o2)
    raw = bytearray(p.read_bytes())
    raw[40] ^= 1
    bad = tmp_path / "bad.cctb"
    bad.write_bytes(bytes(raw))
    with pytest.raises(cc.CoulombError) as e:
        cc.load_tables(bad)
    assert e.value.status == 7


def test_parameter_errors(dev):
    import paper_1502_08043_gb300 as cc
    for kw, st in [(dict(R=0), 2), (dict(R=128), 2), (dict(S=1), 2), (dict(kernel=5), 1),
                   (dict(q_tail=32), 1), (dict(L=-1.0), 1), (dict(S=8, n_sub=7, q_tail=4), 1)]:
        args = dict(kernel="periodic", R=4, L=10.0, S=32)
        args.update(kw)
        with pytest.raises(cc.CoulombError) as e:
            cc.build_tables(**args)
        assert e.value.status == st, kw


def test_build_tables_for_error():
    """Tables built for a stated method error: the library's nodes are the oracle's tuned
    mesh (mesh_tune), pruned as usual; separable lookups on them reproduce the exact kernel
    1/(pi L |q|^2) to the stated error (plus FP32 rounding) on seeded conserving quadruples."""
    import torch
    import coulomb_inputs as ci
    import paper_1502_08043_gb300 as cc
    from gpu_common import need_gpu
    from oracle import reconstruct as orc
    dev = need_gpu()
    R, L, target = 13, 20.0, 1e-8
    t = cc.build_tables_for_error("periodic", R=R, L=L, target=target)
    S, n_sub, q_tail, ac, ratio, err = oq.mesh_tune(R, target, 1024)
    info = t.info
    assert (info["S"], info["n_sub"], info["q_tail"]) == (S, n_sub, q_tail)
    assert info["alpha_c"] == ac and info["ratio"] == ratio
    a, w, part, kept = t.nodes()
    ao, wo, _ = oq.laplace_mesh(S, n_sub, q_tail, ac, ratio)
    assert np.allclose(a, ao, rtol=1e-13) and np.allclose(w, wo, rtol=1e-12)
    assert np.array_equal(kept, oq.prune_periodic(ao, wo, R, 1e-9))
    q = ci.quads(R, 0, 200000)
    exact, _ = orc.reconstruct(q, R, L, "exact")
    out = torch.empty(len(q), dtype=torch.float64, device=dev)
    cc.reconstruct_integrals(t, torch.from_numpy(q).to(dev), out, lookup="separable")
    got = out.cpu().numpy()
    nz = exact != 0
    assert np.max(np.abs(got[nz] - exact[nz]) / exact[nz]) < target + 1e-12
    out32 = torch.empty(len(q), dtype=torch.float32, device=dev)
    cc.reconstruct_integrals(t, torch.from_numpy(q).to(dev), out32, lookup="separable")
    g32 = out32.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(g32[nz] - exact[nz]) / exact[nz]) < target + 1e-6
    t.free()
