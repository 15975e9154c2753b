"""Host-side pieces of the joint block MPS path (no GPU): the choice of the
starting determinants against the oracle's, and the size query of a joint
iterate against the oracle's block dimensions."""
import numpy as np
import pytest

from oracle import bsmps as OB
from oracle import fermion as OF
from oracle import joint as OJ
from paper_2604_16118_gb300 import problem


@pytest.mark.parametrize("K,N,spin,D,seed", [(8, 3, 0, 5, 0), (6, 2, 1, 7, 1), (10, 5, 0, 1, 2), (4, 1, 1, 4, 3)])
def test_lowest_determinants_match_oracle(K, N, spin, D, seed):
    rng = np.random.default_rng(seed)
    n_orb = K // 2 if spin else K
    h = rng.standard_normal(n_orb)
    t_diag = np.repeat(h, 2) if spin else h
    n_up, n_dn = (N, N) if spin else (N, 0)
    occ = problem.lowest_determinants(t_diag, spin, n_up, n_dn, D)
    species = OF.site_species(n_orb, spin)
    ref = OJ.lowest_determinants(species, (n_up, n_dn), t_diag, D)
    assert [tuple(int(v) for v in row) for row in occ] == [tuple(o) for o in ref]
    # every string is in the particle sector
    for row in occ:
        assert sum(int(row[t]) for t in range(len(row)) if species[t] == 0) == n_up
        assert sum(int(row[t]) for t in range(len(row)) if species[t] == 1) == n_dn


def test_lowest_determinants_ties_follow_site_order():
    # all energies equal: occupied-first comparison from site 0
    occ = problem.lowest_determinants(np.zeros(5), 0, 2, 0, 4)
    assert [tuple(r) for r in occ] == [(1, 1, 0, 0, 0), (1, 0, 1, 0, 0), (1, 0, 0, 1, 0), (1, 0, 0, 0, 1)]


def test_lowest_determinants_rejects_bad_requests():
    from paper_2604_16118_gb300.native import BsmpsError
    with pytest.raises(BsmpsError):
        problem.lowest_determinants(np.zeros(4), 0, 2, 0, 7)       # C(4,2) = 6 < 7
    with pytest.raises(BsmpsError):
        problem.lowest_determinants(np.zeros(40), 0, 20, 0, 2, max_configs=1000)


@pytest.mark.parametrize("n_orb,spin,n_up,n_dn,r,D", [(6, 0, 3, 0, 6, 3), (3, 1, 2, 1, 6, 2), (12, 0, 6, 0, 32, 4)])
def test_joint_random_size_matches_oracle_dims(n_orb, spin, n_up, n_dn, r, D):
    from paper_2604_16118_gb300 import build, native
    build.build()
    n = native.mps_joint_random_size(n_orb, spin, n_up, n_dn, r, D)
    species = OF.site_species(n_orb, spin)
    dims = OB.default_dims(species, (n_up, n_dn), r, D)
    tot = OB.BSMPS(species, (n_up, n_dn), dims, [dict() for _ in species]).layout()[1]
    assert n == tot
    assert dims[len(species)] == {(n_up, n_dn): D}
    with pytest.raises(native.BsmpsError):
        native.mps_joint_random_size(n_orb, spin, n_up, n_dn, r, 0)
