"""Host-side helpers of bench.py's paper replay (Table I, Fig. 1) against the oracle's own
definitions: the Kohn-Sham exchange E_KS of Sec. III and the occupied-state count."""
import bench
from oracle import basis as ob
from oracle import exchange as ox


def test_e_ks_matches_oracle():
    for M in (7, 33, 257, 9171, 267761):
        for L in (2.0, 10.0, 60.0):
            assert abs(bench._e_ks(M, L) - ox.E_KS(M, L)) <= 1e-14 * abs(ox.E_KS(M, L))


def test_occupied_count_matches_oracle():
    for R_F in range(0, 14):
        assert bench._n_occupied(R_F) == ob.count(R_F)
    # the shell count of the paper's Table I box
    assert bench._n_occupied(13) == 9171
