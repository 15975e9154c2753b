"""Pins of the exponential-sum preconditioner (Sec. 4) against printed values and theorems."""
import json
import math
import os

import numpy as np
import pytest

from oracle import bsmps as B
from oracle import fermion as F
from oracle import precond as P
from synth import spinless_random_chain

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
PARAMS = json.load(open(os.path.join(GOLDEN, "paper_parameters.json")))


@pytest.mark.parametrize("row", PARAMS["T_lengthS"])
def test_number_of_summands_matches_paper(row):
    h, mm, mp = P.expsum_params(PARAMS["c0"], row["T"])
    assert mp - mm + 1 == row["lengthS"]


@pytest.mark.parametrize("T", [9.53, 39.61, 186.52, 1000.0])
def test_expsum_relative_error_bound(T):
    # Eq. (Srelerror): |t^{-1/2} - S(t)| <= c0 t^{-1/2} on [1, T]
    c0 = 0.1
    h, mm, mp = P.expsum_params(c0, T)
    t = np.geomspace(1.0, T, 20001)
    rel = np.abs(1.0 / np.sqrt(t) - P.expsum(t, h, mm, mp)) * np.sqrt(t)
    assert rel.max() <= c0


@pytest.mark.parametrize("row", PARAMS["delta"])
def test_gap_constant_matches_paper(row):
    d = row["lambda2"] / (row["lambda2"] - row["lambda1"])
    assert abs(d - row["delta"]) < 5e-5


@pytest.mark.parametrize("row", PARAMS["eps"])
def test_eps_num_rule_matches_paper(row):
    # the oracle's default eps_num for c = eps_iter (Sec. 7.1.3) against the printed pair
    from oracle import pinvit as PI
    assert abs(PI.SolverParams(row["eps_iter"], 10.0).eps_num - row["eps_num"]) <= 0.005 + 1e-12


def _extremes(M, k=1):
    """Lowest k and highest eigenvalue of a symmetric matrix by Lanczos (library routine)."""
    from scipy.sparse.linalg import eigsh
    lo = np.sort(eigsh(M, k=k, which="SA", tol=0, return_eigenvectors=False))
    hi = eigsh(M, k=1, which="LA", tol=0, return_eigenvectors=False)[0]
    return lo, hi


@pytest.fixture(scope="module")
def exp14():
    """The appendix run exp14: the Coulomb-like model of Sec. 7.2 with the K = 14
    orbitals of the N = 4 runs (printed t_1 = -8.0, t_2 = 0.31 as there), N = 6
    particles, gamma = 0; finite-difference orbitals (synth.coulomb_1d)."""
    from synth import coulomb_1d
    wl = coulomb_1d(K=14, N=4, n_grid=8192)
    K, N, gamma = 14, 6, 0.0
    t_so, v_so = P.spin_orbital_accessors(wl.h, wl.eri, 0)
    th = P.theta_diag(t_so, v_so, N, gamma, K)
    tmin, tmax = P.spectrum_bounds(th, F.site_species(K, 0), (N, 0), t_diag=np.diag(wl.h))
    H, states = F.sector_hamiltonian(wl.h, wl.eri, 0, N, 0, gamma=gamma)
    occ = np.array([[(int(m) >> s) & 1 for s in range(K)] for m in states])
    return dict(wl=wl, th=th, tmin=tmin, tmax=tmax, H=H, occ=occ, N=N)


def half_unit(x):
    s = repr(x)
    d = len(s.split(".")[1]) if "." in s else 0
    return 0.5 * 10.0 ** (-d)


def test_exp14_interval_matches_printed(exp14):
    # printed t_min = 7.35, t_max = 70.01, T = 9.53, #S = 7 of run exp14
    assert abs(exp14["tmin"] - 7.35) <= half_unit(7.35)
    assert abs(exp14["tmax"] - 70.01) <= half_unit(70.01)
    assert abs(exp14["tmax"] / exp14["tmin"] - 9.53) <= half_unit(9.53)
    h, mm, mp = P.expsum_params(0.1, exp14["tmax"] / exp14["tmin"])
    assert mp - mm + 1 == 7


def test_alpha0_and_c_tight_bounds_and_exp14_printed_c(exp14):
    # Cor. lrprecond: with C_lower (1 - c0)^2 and C_upper (1 + c0)^2 the exact extremes
    # of sigma(S_0 H_gamma S_0), S_0 = t_min^{-1/2} S(D / t_min), the scaling alpha_0 of
    # Eq. (Sdef) makes the spectrum of A = S H_gamma S exactly [1 - c, 1 + c] with c of
    # Eq. (precondcdef); on exp14 that c is the printed 0.29 (lower/upper 0.71 / 1.29,
    # eps_iter 0.29, eps_num 0.36)
    from oracle import pinvit as PI
    c0, tmin = 0.1, exp14["tmin"]
    unit = P.Preconditioner(exp14["th"], tmin, exp14["tmax"], c0, 1.0)
    S0 = unit.dense_diag(exp14["occ"]) / np.sqrt(tmin)
    (nu_lo,), nu_hi = _extremes(S0[:, None] * exp14["H"] * S0[None, :])
    alpha0, c = P.alpha0_and_c(c0, tmin, nu_lo / (1 - c0) ** 2, nu_hi / (1 + c0) ** 2)
    S = P.Preconditioner(exp14["th"], tmin, exp14["tmax"], c0, alpha0).dense_diag(exp14["occ"])
    (a_lo,), a_hi = _extremes(S[:, None] * exp14["H"] * S[None, :])
    assert abs(a_lo - (1 - c)) <= 1e-12 and abs(a_hi - (1 + c)) <= 1e-12
    assert abs((1 - c) - 0.71) <= half_unit(0.71) and abs((1 + c) - 1.29) <= half_unit(1.29)
    assert abs(c - 0.29) <= half_unit(0.29)
    assert abs(PI.SolverParams(c, 10.0).eps_num - 0.36) <= half_unit(0.36)


def test_exp14_exact_eigenvalues_and_gap(exp14):
    # printed exact lambda_1 = 6.77932848602532, lambda_2 = 7.07168841064 and
    # delta = 24.1883 of exp14 / exp64, within the discretisation error 1e-4
    lam, _ = _extremes(exp14["H"], k=2)
    assert abs(lam[0] - 6.77932848602532) <= 1e-4
    assert abs(lam[1] - 7.07168841064) <= 1e-4
    assert abs(lam[1] / (lam[1] - lam[0]) - 24.1883) <= 2e-3


def test_product_form_equals_scaled_expsum():
    # Sec. 4.3: sum_m (x)_i diag(alpha_m^{1/K}, alpha_m^{1/K} e^{-beta_m d_i}) = alpha_0 S(D/t_min)
    # on every occupation vector -- pins beta_m = e^{mh}/t_min and alpha_m^{1/K}
    rng = np.random.default_rng(0)
    K = 7
    d = rng.uniform(0.5, 4.0, K)
    prec = P.Preconditioner(d, t_min=1.1, t_max=20.0, c0=0.1, alpha0=0.8)
    occ = np.array([[(i >> s) & 1 for s in range(K)] for i in range(1 << K)])
    prod = np.zeros(len(occ))
    for j in range(prec.n_terms):
        f0, f1 = prec.factors(j)
        prod += np.prod(np.where(occ == 1, f1[None, :], f0[None, :]), axis=1)
    ref = prec.dense_diag(occ)
    assert np.abs(prod - ref).max() <= 1e-14 * np.abs(ref).max()


def test_spectral_equivalence_by_exact_diagonalisation():
    # Cor. lrprecond: (1-c) <= spec(S H_gamma S) <= (1+c) with C_lower/C_upper from ED
    K, N = 8, 4
    wl = spinless_random_chain(K=K, N=N, seed=3)
    species = F.site_species(K, 0)
    H0, states = F.sector_hamiltonian(wl.h, wl.eri, 0, N, 0)
    gamma = 1.0 - np.linalg.eigvalsh(H0)[0]
    t_so, v_so = P.spin_orbital_accessors(wl.h, wl.eri, 0)
    th = P.theta_diag(t_so, v_so, N, gamma, K)
    tmin, tmax = P.spectrum_bounds(th, species, (N, 0))
    assert tmin > 0
    occ = np.array([[(int(m) >> s) & 1 for s in range(K)] for m in states])
    Dv = occ @ th
    assert Dv.min() >= tmin - 1e-12 and Dv.max() <= tmax + 1e-12
    Hg = H0 + gamma * np.eye(len(H0))
    ev = np.linalg.eigvalsh(Hg / np.sqrt(np.outer(Dv, Dv)))
    alpha0, c = P.alpha0_and_c(0.1, tmin, ev[0], ev[-1])
    prec = P.Preconditioner(th, tmin, tmax, 0.1, alpha0)
    Sd = prec.dense_diag(occ)
    ea = np.linalg.eigvalsh(Sd[:, None] * Hg * Sd[None, :])
    assert 1 - c - 1e-12 <= ea[0] and ea[-1] <= 1 + c + 1e-12


def test_block_scaling_matches_dense_preconditioner():
    # S_m x on the block-sparse MPS equals the diagonal matrix S_m on the dense vector
    K = 6
    species = F.site_species(K, 0)
    d = np.linspace(0.5, 3.0, K)
    prec = P.Preconditioner(d, 1.0, 10.0, 0.1, 0.7)
    dims = B.default_dims(species, (3, 0), 5)
    tmp = B.BSMPS(species, (3, 0), dims, [dict() for _ in range(K)])
    _, tot = tmp.layout()
    x = B.BSMPS.from_flat(species, (3, 0), dims, np.random.default_rng(1).standard_normal(tot))
    xd = B.to_dense(x)
    occ = np.array([[(i >> (K - 1 - s)) & 1 for s in range(K)] for i in range(1 << K)])
    acc = np.zeros_like(xd)
    for j in range(prec.n_terms):
        f0, f1 = prec.factors(j)
        acc += B.to_dense(B.scale_sites(x, f0, f1))
    assert np.abs(acc - prec.dense_diag(occ) * xd).max() < 1e-13


def test_energy_lower_bound_free_fermions_closed_form():
    # U = 0 open Hubbard chain: the bound is the exact ground energy
    # 2 sum_{j=1}^{L/2} -2 cos(pi j / (L + 1)) (closed form), and equals ED at L = 4
    from synth import hubbard_chain
    for L in (4, 32):
        wl = hubbard_chain(L=L, U=0.0)
        e = P.energy_lower_bound(wl.h, wl.eri, 1, L // 2, L // 2, cholesky=False)
        exact = 2.0 * sum(-2.0 * math.cos(math.pi * j / (L + 1)) for j in range(1, L // 2 + 1))
        assert abs(e - exact) <= 1e-12 * abs(exact)
    wl = hubbard_chain(L=4, U=0.0)
    H, _ = F.sector_hamiltonian(wl.h, wl.eri, 1, 2, 2)
    assert abs(np.linalg.eigvalsh(H)[0] - P.energy_lower_bound(wl.h, wl.eri, 1, 2, 2, False)) <= 1e-12


def test_energy_lower_bound_normal_ordering_term_is_tight():
    # one Cholesky vector L = diag(1, -1, 0, 0, 0) and h = diag(e): V = 1/2 (n_0 - n_1)^2
    # - 1/2 (n_0 + n_1); with two particles the ground state {0, 1} has energy
    # e_0 + e_1 - 1, which the bound reaches exactly (a wrong sign or factor of the
    # normal-ordering term misses it)
    e = np.array([0.0, 0.3, 2.0, 2.5, 3.0])
    lv = np.diag([1.0, -1.0, 0.0, 0.0, 0.0])
    eri = np.einsum("pq,rs->pqrs", lv, lv)
    H, _ = F.sector_hamiltonian(np.diag(e), eri, 0, 2, 0)
    e0 = np.linalg.eigvalsh(H)[0]
    assert abs(e0 - (e[0] + e[1] - 1.0)) <= 1e-13
    assert abs(P.energy_lower_bound(np.diag(e), eri, 0, 2, 0, cholesky=True) - e0) <= 1e-13


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_energy_lower_bound_below_exact_ground_energy(seed):
    # invariant: E_lb <= E_0 (ED) for Cholesky-built integrals and for U > 0 Hubbard
    from synth import hubbard_chain, molecule_like
    wl = spinless_random_chain(K=8, N=4, seed=seed)
    H, _ = F.sector_hamiltonian(wl.h, wl.eri, 0, 4, 0)
    assert P.energy_lower_bound(wl.h, wl.eri, 0, 4, 0, True) <= np.linalg.eigvalsh(H)[0] + 1e-12
    wl = molecule_like(L=4, n_up=2, n_dn=1, seed=seed)
    H, _ = F.sector_hamiltonian(wl.h, wl.eri, 1, 2, 1)
    assert P.energy_lower_bound(wl.h, wl.eri, 1, 2, 1, True) <= np.linalg.eigvalsh(H)[0] + 1e-12
    wl = hubbard_chain(L=4, U=2.0 + seed)
    H, _ = F.sector_hamiltonian(wl.h, wl.eri, 1, 2, 2)
    assert P.energy_lower_bound(wl.h, wl.eri, 1, 2, 2, False) <= np.linalg.eigvalsh(H)[0] + 1e-12
