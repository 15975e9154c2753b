"""Pins of the oracle's zip-up application (Sec. 2.4 with the QR sweep of Sec. 2.3)."""
import numpy as np
import pytest

from oracle import bsmps as B
from oracle import fermion as F
from oracle import mpo as M
from synth import hubbard_chain, molecule_like, spinless_random_chain

CASES = [
    ("spinless_K7", spinless_random_chain(K=7, N=3, seed=1), 6, 0.4),
    ("hubbard_L4", hubbard_chain(L=4, n_up=2, n_dn=2, U=4.0), 8, 1.0),
    ("molecule_L4", molecule_like(L=4, n_up=2, n_dn=1, seed=2), 10, 2.0),
]


def setup(wl, r, gamma, seed=3):
    species = F.site_species(wl.n_orb, wl.spin)
    target = (wl.n_up, wl.n_dn)
    dims = B.default_dims(species, target, r)
    n = B.BSMPS(species, target, dims, [dict() for _ in species]).layout()[1]
    x = B.BSMPS.from_flat(species, target, dims, np.random.default_rng(seed).standard_normal(n))
    return x, M.build_mpo(wl.h, wl.eri, wl.spin, wl.n_particles, gamma)


@pytest.mark.parametrize("name,wl,r,gamma", CASES)
def test_zipup_equals_dense_operator(name, wl, r, gamma):
    # the represented vector is (H_gamma + s) x computed with the dense Jordan-Wigner H
    x, W = setup(wl, r, gamma)
    y = B.apply_zipup(W, x, shift=-0.7)
    Hf = F.full_hamiltonian(wl.h, wl.eri, wl.spin, wl.n_particles, gamma)
    ref = Hf @ B.to_dense(x) - 0.7 * B.to_dense(x)
    assert np.linalg.norm(B.to_dense(y) - ref) <= 1e-13 * np.linalg.norm(ref)


@pytest.mark.parametrize("name,wl,r,gamma", CASES)
def test_zipup_is_left_orthogonal_with_exact_ranks(name, wl, r, gamma):
    # every core but the last is left-orthonormal per sector; each bond dim is the
    # rank rule min(stacked rows, exact columns) of the QR sweep
    x, W = setup(wl, r, gamma)
    y = B.apply_zipup(W, x, shift=0.3)
    ex = B.apply_exact(W, x, shift=0.3)
    for t in range(y.K - 1):
        sp = y.species[t]
        for m2, k in y.bonds[t + 1].items():
            S = np.vstack([y.cores[t][(m, s)] for (m, s) in y.block_keys(t)
                           if B.add_charge(m, B.delta(sp, s)) == m2])
            assert np.abs(S.T @ S - np.eye(k)).max() <= 1e-14 * max(1, S.shape[0])
            rows = sum(y.bonds[t][m] for (m, s) in y.block_keys(t) if B.add_charge(m, B.delta(sp, s)) == m2)
            assert k == min(rows, ex.bonds[t + 1][m2])
    # the last core carries the norm
    nrm = np.sqrt(sum(np.sum(Bk * Bk) for Bk in y.cores[-1].values()))
    assert abs(nrm - np.linalg.norm(B.to_dense(ex))) <= 1e-13 * nrm


@pytest.mark.parametrize("name,wl,r,gamma", CASES)
def test_zipup_then_truncation_equals_exact_then_truncation(name, wl, r, gamma):
    # the gauge of the zip-up bonds disappears in trunc_eps (left QR, right SVD with the
    # sign rule): same kept dims and the same cores as truncating the exact application
    x, W = setup(wl, r, gamma, seed=5)
    y = B.apply_zipup(W, x, shift=-1.1)
    ex = B.apply_exact(W, x, shift=-1.1)
    nrm = np.linalg.norm(B.to_dense(ex))
    for rel in (1e-13, 1e-6, 1e-2):
        a, da, _ = B.truncate(y, rel * nrm)
        b, db, _ = B.truncate(ex, rel * nrm)
        assert a.bonds == b.bonds
        assert abs(da - db) <= 1e-12 * nrm
        for t in range(a.K):
            for k in b.cores[t]:
                scale = max(1.0, nrm) if t == 0 else 1.0
                assert np.abs(a.cores[t][k] - b.cores[t][k]).max() <= 1e-11 * scale, (rel, t, k)
