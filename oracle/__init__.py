"""Plain FP64 CPU oracle of the compressed Coulomb-integral engine.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline and reference legs may import anything from this package; the product
path (the CUDA library and its binding) never does, and this package never imports the
product.  Everything is numpy float64 written straight from the paper:

* basis.py       Sec. II (Eq. 1) and Sec. III: separable planewave basis, shell counts,
                 Fermi-sphere occupations.
* quadrature.py  Sec. II, Eqs. 5-14 and the Table I discussion: Laplace-variable meshes
                 (interval 1 on [0, alpha_c], geometric sub-intervals, the t = alpha^-1/2
                 tail) and the node pruning rule.
* coulomb.py     Sec. II, Eqs. 2-8 and 14: exact periodic planewave integrals, their
                 separable node-sum form, and the finite-box (free-space kernel) per-axis
                 integrals A(alpha, Delta).
* exchange.py    Sec. III: exchange sums eps(k), E_x, the Kohn-Sham reference E_KS and
                 the pair-difference histogram.
* reconstruct.py Sec. II, Eq. 14 applied to batches of quadruples with the
                 momentum-conservation bookkeeping.

Readings of silent or garbled passages (all stated in the functions that take them):
the tail weight of Eq. 13 is 2 w / t^3 (the printed 1/2 w alpha^{3/2} t^{2n} is garbled);
the 1/|r| transform carries 1/(2 pi^2); integrals are chemists' (IJ|KL) with complex
conjugates on I and K; the planewave cutoff is |n|^2 <= R^2; the periodic q = 0 term is
excluded; Table I is the finite-box model at side L = 2 with alpha_c = 1.

Parity pins live in tests/test_oracle_*.py.  The bf16/fp16 split-precision path has no
oracle of its own: it is compared with the FP64 separable values here, and its error
model (not a value) is the only extra statement ("parity unpinned" beyond that).
"""
from . import basis, quadrature, coulomb, exchange, reconstruct  # noqa: F401
