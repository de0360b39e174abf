"""Oracle pins: planewave basis and shell closings (Sec. II Eq. 1, Sec. III)."""
import os

import numpy as np

import coulomb_inputs as ci
from oracle import basis as ob

GOLD = os.path.join(os.path.dirname(__file__), "golden", "shell_counts.txt")


def _golden():
    rows = [l.split() for l in open(GOLD) if l.strip() and not l.startswith("#")]
    return [(int(a), int(b)) for a, b in rows]


def test_shell_counts_match_paper():
    for R_F, M in _golden():
        assert ob.count(R_F) == M
        assert len(ob.occupied(R_F)) == M
        assert int(ob.occupation_grid(R_F, R_F).sum()) == M


def test_basis_order_and_membership():
    for R in (0, 1, 2, 4, 7):
        B = ob.basis(R)
        assert len(B) == ob.count(R)
        assert np.all((B * B).sum(axis=1) <= R * R)
        # strictly increasing lexicographic order, hence unique
        key = ((B[:, 0] + R) * (2 * R + 1) + (B[:, 1] + R)) * (2 * R + 1) + (B[:, 2] + R)
        assert np.all(np.diff(key) > 0)
        # the input generator's own enumeration lists the same vectors in the same order
        assert np.array_equal(B, ci.sphere_vectors(R))


def test_counts_of_configured_cutoffs():
    # cutoffs of the workloads: R = 4, 13, 31 (63 is checked on the generator side)
    assert ob.count(4) == 257
    assert ob.count(13) == 9171
    assert ob.count(31) == 124487
