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
    assert abs(0.5 * (1 - row["eps_iter"]) - row["eps_num"]) <= 0.005 + 1e-12


def test_printed_one_plus_minus_c():
    # lower/upper printed as 0.71/1.29 with c = eps_iter = 0.29 (appendix run exp14)
    assert abs((1 - 0.29) - 0.71) < 1e-12 and abs((1 + 0.29) - 1.29) < 1e-12


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
