"""The paper's own workload (Sec. 7.2): the one-dimensional Coulomb-like model.

Orbitals from a finite-difference grid stand in for the paper's multiwavelet
orbitals (`synth.coulomb_1d`).  Pins, against the printed numbers
(tests/golden/paper_coulomb1d.json): the one-body energies t_ii, the
preconditioner interval t_min, t_max, T = t_max / t_min and the number of
exponential-sum terms #S, the gap constant delta and the lowest eigenvalues of
the K = 14 problem by exact diagonalisation (within the paper's stated
discretisation error)."""
import json
import os

import numpy as np
import pytest

from oracle import fermion as F
from oracle import precond as P
from synth import coulomb_1d

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_coulomb1d.json")))


def half_unit(x):
    s = repr(x)
    d = len(s.split(".")[1]) if "." in s else 0
    return 0.5 * 10.0 ** (-d)


def interval(wl, gamma):
    t_so, v_so = P.spin_orbital_accessors(wl.h, wl.eri, 0)
    th = P.theta_diag(t_so, v_so, wl.n_up, gamma, wl.n_orb)
    species = F.site_species(wl.n_orb, 0)
    return th, P.spectrum_bounds(th, species, (wl.n_up, 0), t_diag=np.diag(wl.h))


@pytest.fixture(scope="module")
def k14():
    return coulomb_1d(K=14, n_grid=8192)


@pytest.mark.parametrize("K", [14, 30])
def test_one_body_energies_and_interval(K):
    g = GOLD[f"K{K}"]
    gamma = GOLD["model"]["gamma"]
    wl = coulomb_1d(K=K, n_grid=8192)
    t = np.diag(wl.h)
    for key, val in (("t_1", t[0]), ("t_2", t[1]), ("t_Km1", t[-2]), ("t_K", t[-1])):
        assert abs(val - g[key]) <= half_unit(g[key]) + 1e-3, key
    th, (tmin, tmax) = interval(wl, gamma)
    assert abs(tmin - g["t_min"]) <= half_unit(g["t_min"])
    assert abs(tmax - g["t_max"]) <= half_unit(g["t_max"]) + 2e-2
    assert abs(tmax / tmin - g["T"]) <= half_unit(g["T"]) + 2e-2
    h, m_minus, m_plus = P.expsum_params(0.1, tmax / tmin)
    assert m_plus - m_minus + 1 == g["lengthS"]
    # the N smallest theta would give a different, smaller t_min on this model
    assert np.sort(th)[:4].sum() < tmin - 0.1


def test_exact_eigenvalues_k14(k14):
    g = GOLD["K14"]
    gamma = GOLD["model"]["gamma"]
    H0, _ = F.sector_hamiltonian(k14.h, k14.eri, 0, 4, 0)
    lam = np.linalg.eigvalsh(H0)[:2] + gamma
    tol = GOLD["tolerances"]["discretisation"]
    assert abs(lam[0] - g["lambda1"]) <= tol
    assert abs(lam[1] - g["lambda2"]) <= tol
    delta = lam[1] / (lam[1] - lam[0])
    assert abs(delta - g["delta"]) <= 2e-3


def test_preconditioned_spectrum_and_higher_eigenvalues_k14(k14):
    # c is the spectral equivalence constant of A = S H_gamma S (eps_iter = c for omega = 1):
    # its exact value by diagonalisation gives the printed 1 - c, 1 + c, eps_iter and eps_num
    g = GOLD["K14"]
    gamma = GOLD["model"]["gamma"]
    H, states = F.sector_hamiltonian(k14.h, k14.eri, 0, 4, 0, gamma=gamma)
    th, (tmin, tmax) = interval(k14, gamma)
    prec = P.Preconditioner(th, tmin, tmax, 0.1, 1.0)
    occ = np.array([[(int(m) >> s) & 1 for s in range(k14.n_orb)] for m in states])
    S = prec.dense_diag(occ)
    mu = np.linalg.eigvalsh(S[:, None] * H * S[None, :])
    c = (mu[-1] - mu[0]) / (mu[-1] + mu[0])
    assert abs((1 - c) - g["one_minus_c"]) <= half_unit(g["one_minus_c"])
    assert abs((1 + c) - g["one_plus_c"]) <= half_unit(g["one_plus_c"])
    assert abs(c - g["eps_iter"]) <= half_unit(g["eps_iter"])
    assert abs(0.5 * (1 - c) - g["eps_num"]) <= half_unit(g["eps_num"])
    lam = np.linalg.eigvalsh(H)[:4]
    assert np.all(np.abs(lam - np.array(g["lambda_1to4"])) <= GOLD["tolerances"]["discretisation"])
