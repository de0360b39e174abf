"""Helpers shared by the GPU parity tests (inputs and oracle references, no CUDA path)."""
import numpy as np
import pytest

from oracle import quadrature as oq

# single-box workloads: (R, L, S, R_F)
CFG1 = dict(R=4, L=10.0, S=32, R_F=2)
CFG2 = dict(R=13, L=20.0, S=64, R_F=8)
CFG3 = dict(R=31, L=40.0, S=96, R_F=20)
CFG5 = dict(R=63, L=60.0, S=128, R_F=40)

# FP32 parity bound against the FP64 node sum of the same nodes, and FP64 bound
TOL_FP32 = 1e-6
TOL_FP64 = 1e-12
# Gauss-Legendre points of one box-kernel axis integral in the library (its header states
# the 1200-point rule); box-kernel references are computed at the same point count so that
# the quadrature difference drops out of the comparison
BOX_POINTS = 1200
# FP64 bound of box-kernel results: a box axis integral A(alpha, D) is a quadrature sum of an
# oscillating integrand whose terms cancel, so its FP64 value carries ~1e-16 of the sum of
# the absolute terms; the library (tree reduction) and the oracle (numpy) sum in different
# orders, and at the entries that cancel most the two differ by up to ~3e-11 relative
TOL_FP64_BOX = 1e-10


def oracle_nodes(R, S, prune=1e-9):
    n_sub, q_tail = oq.default_periodic_mesh(S, R)
    a, w, part = oq.laplace_mesh(S, n_sub, q_tail)
    keep = oq.prune_periodic(a, w, R, prune)
    return a[keep], w[keep]


def need_gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1502_08043_gb300 import build
    build.build()
    return torch.device("cuda:0")


def rel_err(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    nz = ref != 0
    return float(np.max(np.abs(got[nz] - ref[nz]) / np.abs(ref[nz]))) if nz.any() else 0.0
