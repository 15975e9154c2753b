"""Pins of the dense Jordan--Wigner reference (Sec. 1.1) against the mathematics."""
import math

import numpy as np
import pytest

from oracle import fermion as F
from synth import hubbard_chain, molecule_like, spinless_random_chain


def test_anticommutation_relations():
    # Eq. (anticomm)
    K = 4
    a = [F.annihilator_full(K, i) for i in range(K)]
    I = np.eye(1 << K)
    for i in range(K):
        for j in range(K):
            assert np.allclose(a[i] @ a[j].T + a[j].T @ a[i], I * (i == j))
            assert np.allclose(a[i] @ a[j] + a[j] @ a[i], 0)


def test_hamiltonian_hermitian_and_number_conserving():
    wl = spinless_random_chain(K=6, N=3, seed=3)
    H = F.full_hamiltonian(wl.h, wl.eri, 0, 3, gamma=0.5)
    P = F.number_operator_full(6)
    assert np.abs(H - H.T).max() < 1e-12
    assert np.abs(H @ P - P @ H).max() < 1e-12


@pytest.mark.parametrize("wl", [spinless_random_chain(K=6, N=3, seed=1),
                                hubbard_chain(L=3, n_up=2, n_dn=1),
                                molecule_like(L=3, n_up=1, n_dn=2, seed=4)])
def test_sector_matrix_is_restriction_of_full(wl):
    # two independent constructions: bitstring action vs Kronecker products
    Hf = F.full_hamiltonian(wl.h, wl.eri, wl.spin, wl.n_particles, gamma=0.3)
    Hs, states = F.sector_hamiltonian(wl.h, wl.eri, wl.spin, wl.n_up, wl.n_dn, gamma=0.3)
    K = wl.n_sites
    idx = [sum(((int(m) >> s) & 1) << (K - 1 - s) for s in range(K)) for m in states]
    assert np.abs(Hf[np.ix_(idx, idx)] - Hs).max() < 1e-13
    # the sector is an invariant subspace: no coupling out of it
    rest = np.setdiff1d(np.arange(1 << K), idx)
    assert np.abs(Hf[np.ix_(rest, idx)]).max() < 1e-13


def test_shift_adds_gamma_on_sector():
    # t_ii + gamma/N adds gamma * I on F_N (Sec. 7.1.1)
    wl = spinless_random_chain(K=6, N=2, seed=5)
    H0, _ = F.sector_hamiltonian(wl.h, wl.eri, 0, 2, 0)
    H1, _ = F.sector_hamiltonian(wl.h, wl.eri, 0, 2, 0, gamma=1.7)
    assert np.abs(H1 - H0 - 1.7 * np.eye(len(H0))).max() < 1e-13


def test_two_site_hubbard_closed_form():
    for t, U in [(1.0, 4.0), (0.7, 2.5)]:
        wl = hubbard_chain(L=2, n_up=1, n_dn=1, t=t, U=U)
        H, _ = F.sector_hamiltonian(wl.h, wl.eri, 1, 1, 1)
        e0 = np.linalg.eigvalsh(H)[0]
        assert abs(e0 - (U - math.sqrt(U * U + 16 * t * t)) / 2) < 1e-12


def test_free_fermion_limits():
    # U = 0 open chain: sum of the lowest single-particle levels -2t cos(pi j/(L+1)) per spin
    L, nu, nd = 5, 3, 2
    wl = hubbard_chain(L=L, n_up=nu, n_dn=nd, U=0.0)
    H, _ = F.sector_hamiltonian(wl.h, wl.eri, 1, nu, nd)
    eps = sorted(-2.0 * math.cos(math.pi * j / (L + 1)) for j in range(1, L + 1))
    assert abs(np.linalg.eigvalsh(H)[0] - (sum(eps[:nu]) + sum(eps[:nd]))) < 1e-12
    # molecule-like generator with the two-body part removed
    wl = molecule_like(L=4, n_up=2, n_dn=1, seed=7)
    H, _ = F.sector_hamiltonian(wl.h, 0 * wl.eri, 1, 2, 1)
    ev = np.linalg.eigvalsh(wl.h)
    assert abs(np.linalg.eigvalsh(H)[0] - (ev[:2].sum() + ev[:1].sum())) < 1e-12


def test_one_body_diagonal_e1_is_eigenvector():
    # Sec. 7.1.4: with diagonal t, e_1 (first N orbitals occupied) has energy sum_{i<=N} t_ii
    K, N = 6, 3
    h = np.diag(np.arange(K, dtype=float) * 0.3 - 0.5)
    H, states = F.sector_hamiltonian(h, np.zeros((K,) * 4), 0, N, 0)
    e1 = int(sum(1 << s for s in range(N)))
    i = list(states).index(e1)
    v = np.zeros(len(states)); v[i] = 1.0
    assert np.allclose(H @ v, h.diagonal()[:N].sum() * v)
    assert abs(np.linalg.eigvalsh(H)[0] - h.diagonal()[:N].sum()) < 1e-13
