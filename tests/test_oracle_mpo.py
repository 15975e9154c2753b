"""Pins of the oracle's MPO (Sec. 2.4, Thm. opranks) against dense Jordan--Wigner."""
import numpy as np
import pytest

from oracle import fermion as F
from oracle import mpo as M
from synth import hubbard_chain, molecule_like, spinless_random_chain


@pytest.mark.parametrize("wl,gamma", [
    (spinless_random_chain(K=5, N=2, seed=11), 0.0),
    (spinless_random_chain(K=7, N=3, seed=12), 1.3),
    (hubbard_chain(L=3, n_up=1, n_dn=2, U=3.0), 0.4),
    (molecule_like(L=3, n_up=2, n_dn=1, seed=13), 2.0),
])
def test_mpo_contracts_to_dense_hamiltonian(wl, gamma):
    Hf = F.full_hamiltonian(wl.h, wl.eri, wl.spin, wl.n_particles, gamma)
    mpo = M.build_mpo(wl.h, wl.eri, wl.spin, wl.n_particles, gamma)
    Hm = M.mpo_to_dense(mpo)
    assert np.abs(Hf - Hm).max() <= 1e-13 * max(1.0, np.abs(Hf).max())
    # the shift slot adds s * Id
    Hs = M.mpo_to_dense(mpo, shift=-0.77)
    assert np.abs(Hs - (Hf - 0.77 * np.eye(len(Hf)))).max() < 1e-12


def test_rank_bounds_dense_and_banded():
    # Thm. opranks (i): T <= K+2, V <= K^2/2 + 3K/2 + 2, so H = T + V below their sum
    K = 8
    wl = spinless_random_chain(K=K, N=4, seed=2)
    mpo = M.build_mpo(wl.h, wl.eri, 0, 4, 0.5)
    bound = (K + 2) + (K * K / 2 + 1.5 * K + 2)
    assert max(mpo.bond_dims) <= bound
    # Thm. opranks (ii): one-body operator of bandwidth d has MPO ranks <= 2d + 2
    for d in (1, 2, 3):
        h = np.zeros((K, K))
        rng = np.random.default_rng(d)
        for p in range(K):
            for q in range(K):
                if abs(p - q) <= d:
                    h[p, q] = rng.standard_normal()
        h = h + h.T
        mpo = M.build_mpo(h, np.zeros((K,) * 4), 0, 4, 0.0)
        assert max(mpo.bond_dims) <= 2 * d + 2, (d, mpo.bond_dims)


def test_hubbard_channel_counts():
    wl = hubbard_chain(L=6, U=4.0)
    mpo = M.build_mpo(wl.h, wl.eri, 1, 6, 0.0)
    dims = mpo.bond_dims
    assert dims[0] == dims[-1] == 1
    assert max(dims) <= 7


def test_entries_conserve_charge():
    wl = molecule_like(L=4, n_up=2, n_dn=2, seed=3)
    mpo = M.build_mpo(wl.h, wl.eri, 1, 4, 0.0)
    for t in range(mpo.K):
        sp = mpo.species[t]
        for (a, b, so, si, w) in mpo.entries(t):
            da, db = mpo.charges[t][a], mpo.charges[t + 1][b]
            d = [0, 0]
            d[sp] = so - si
            assert (db[0] - da[0], db[1] - da[1]) == tuple(d)
