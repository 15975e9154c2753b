"""Pins of the joint block MPS operations and of Alg. 4 (Sec. 6) in the oracle.

Every joint operation is checked against the dense 2^K x D matrix it
represents; the subspace iteration against exact diagonalisation, against the
Courant--Fischer bound (Ritz values of exactly computed Gram matrices lie above
the eigenvalues) and, for D = 1, against Alg. 2 (the paper states that the two
algorithms coincide there).
"""
import math

import numpy as np
import pytest

from oracle import bsmps as B
from oracle import fermion as OF
from oracle import joint as J
from oracle import pinvit as PI
from tests.test_oracle_pinvit import small_problem


def random_joint(species, target, r_max, D, seed):
    dims = B.default_dims(species, target, r_max, D)
    K = len(species)
    assert dims[K] == {tuple(target): D}
    tmp = B.BSMPS(species, target, dims, [dict() for _ in range(K)])
    _, tot = tmp.layout()
    return B.BSMPS.from_flat(species, target, dims, np.random.default_rng(seed).standard_normal(tot))


@pytest.fixture(scope="module")
def prob():
    return small_problem(K=6, N=3, r_max=6, dominant=True, lam1=0.5)


def test_joint_dense_matches_columns(prob):
    x = random_joint(prob["x0"].species, prob["x0"].target, 4, 3, 1)
    X = B.to_dense_cols(x)
    assert X.shape == (64, 3)
    assert np.allclose(X[~prob["in_sector"]], 0.0)
    # column i alone, as an MPS with one column, is x e_i
    for i in range(3):
        e = np.zeros((3, 1))
        e[i, 0] = 1.0
        assert np.allclose(B.to_dense(B.mix_columns(x, e)), X[:, i], atol=1e-14)


def test_gram_is_the_dense_matrix(prob):
    sp, tg = prob["x0"].species, prob["x0"].target
    a = random_joint(sp, tg, 4, 3, 2)
    b = random_joint(sp, tg, 5, 2, 3)
    Ad, Bd = B.to_dense_cols(a), B.to_dense_cols(b)
    G = B.gram(a, b, prob["mpo"])
    ref = Ad.T @ prob["Hf"] @ Bd
    assert G.shape == (3, 2)
    assert np.abs(G - ref).max() <= 1e-12 * np.abs(ref).max()
    assert np.abs(B.gram(a, b) - Ad.T @ Bd).max() <= 1e-13 * np.abs(Ad.T @ Bd).max()
    # a plain MPS: the 1 x 1 Gram matrix is the inner product
    x = prob["x0"]
    assert abs(B.gram(x, x, prob["mpo"])[0, 0] - B.dot(x, x, prob["mpo"])) < 1e-12 * abs(B.dot(x, x, prob["mpo"]))


def test_column_shift_apply(prob):
    x = random_joint(prob["x0"].species, prob["x0"].target, 4, 3, 4)
    cs = np.array([-0.7, 0.25, 1.5])
    y = B.apply_exact(prob["mpo"], x, 0.0, col_shift=cs)
    X = B.to_dense_cols(x)
    ref = prob["Hf"] @ X + X * cs[None, :]
    assert np.abs(B.to_dense_cols(y) - ref).max() <= 1e-12 * np.abs(ref).max()
    # the scalar shift and a constant column shift agree
    y2 = B.apply_exact(prob["mpo"], x, 0.3)
    y3 = B.apply_exact(prob["mpo"], x, 0.0, col_shift=np.full(3, 0.3))
    assert np.abs(B.to_dense_cols(y2) - B.to_dense_cols(y3)).max() <= 1e-12 * np.abs(ref).max()
    # no rank from the shift: the layout is the exact apply's
    assert y.bonds == B.apply_exact(prob["mpo"], x).bonds


def test_joint_add_mix_and_truncate(prob):
    sp, tg = prob["x0"].species, prob["x0"].target
    a = random_joint(sp, tg, 4, 3, 5)
    b = random_joint(sp, tg, 3, 2, 6)
    rng = np.random.default_rng(7)
    Wa, Wb = rng.standard_normal((3, 2)), rng.standard_normal((2, 2))
    s = B.add(B.mix_columns(a, Wa), B.mix_columns(b, Wb))
    ref = B.to_dense_cols(a) @ Wa + B.to_dense_cols(b) @ Wb
    S = B.to_dense_cols(s)
    assert np.abs(S - ref).max() <= 1e-13 * np.abs(ref).max()
    assert B.columns(s) == 2
    for eps_rel in (1e-1, 1e-3, 1e-8):
        eps = eps_rel * np.linalg.norm(S)
        y, dt, _ = B.truncate(s, eps)
        err = np.linalg.norm(B.to_dense_cols(y) - S)
        assert err <= eps * (1 + 1e-10)
        assert abs(err - dt) <= 1e-10 * max(eps, 1e-300) + 1e-13
        assert B.columns(y) == 2


def test_determinant_start(prob):
    sp, tg = prob["x0"].species, prob["x0"].target
    t_diag = [0.1, 0.4, 0.2, 0.9, 0.3, 0.5]
    occs = J.lowest_determinants(sp, tg, t_diag, 4)
    # brute force over all 3-of-6 occupations
    import itertools
    allc = sorted((sum(t_diag[i] for i in c), c) for c in itertools.combinations(range(6), 3))
    assert [tuple(i for i in range(6) if o[i]) for o in occs] == [c for _, c in allc[:4]]
    x = J.from_determinants(sp, tg, occs)
    X = B.to_dense_cols(x)
    for i, o in enumerate(occs):
        idx = int("".join(map(str, o)), 2)       # site 0 is the most significant bit
        e = np.zeros(64)
        e[idx] = 1.0
        assert np.array_equal(X[:, i], e)
    assert max(x.ranks()) <= 4
    # D = 1 with increasing t_ii gives e_1 of Sec. 7.1.4
    one = J.from_determinants(sp, tg, J.lowest_determinants(sp, tg, sorted(t_diag), 1))
    assert np.array_equal(B.to_dense_cols(one)[:, 0], B.to_dense(B.e1_mps(sp, tg)))


def test_d1_coincides_with_alg2(prob):
    params = PI.SolverParams(prob["c"], prob["delta"], r_max=6)
    x = prob["x0"]
    s2, s4 = PI.SolverState(), PI.SolverState()
    x2, x4 = x, x
    for _ in range(4):
        x2, i2 = PI.step(x2, prob["mpo"], prob["prec"], params, s2)
        x4, i4 = J.step(x4, prob["mpo"], prob["prec"], params, s4)
        assert abs(i4["lambda"][0] - i2["lambda"]) <= 1e-12 * i2["lambda"]
        assert abs(i4["rho"][0] - i2["rho"]) <= 1e-9 * i2["rho"]
        assert i4["eta_tries"] == i2["eta_tries"]
        if i2["converged"]:
            break
        assert abs(i4["lambda_star"][0] - i2["lambda_star"]) <= 1e-12 * i2["lambda_star"]
        assert i4["ranks"] == i2["ranks"]


@pytest.fixture(scope="module")
def joint_run(prob):
    sp, tg = prob["x0"].species, prob["x0"].target
    Hs = prob["Hf"][np.ix_(prob["in_sector"], prob["in_sector"])]
    lam_all = np.linalg.eigvalsh(Hs)
    D = 3
    params = PI.SolverParams(prob["c"], prob["delta"], tau=1e-8)
    x = random_joint(sp, tg, 6, D, 11)
    st = PI.SolverState()
    hist = []
    for _ in range(60):
        x, info = J.step(x, prob["mpo"], prob["prec"], params, st)
        hist.append(info)
        if info["converged"]:
            break
    return prob, lam_all, x, hist


def test_ritz_values_bound_the_eigenvalues(joint_run):
    _, lam_all, _, hist = joint_run
    for info in hist:
        assert np.all(info["lambda"] >= lam_all[:3] - 1e-12 * lam_all[:3])
        assert np.all(np.diff(info["lambda"]) >= 0.0)


def test_joint_iteration_reaches_the_lowest_eigenvalues(joint_run):
    prob, lam_all, x, hist = joint_run
    last = hist[-1]
    assert last["converged"]
    lam = last["lambda"]
    # column 1 is certified by the a-posteriori bound (Eq. (releigerr))
    assert (lam[0] - lam_all[0]) / lam_all[0] <= last["releig_bound"] * (1 + 1e-6) + 1e-13
    assert last["releig_bound"] < 1e-12
    # the other columns are not part of the termination test; they converge more
    # slowly (lambda_3 / lambda_4 = 0.94 here), from 3.1 and 4.7 at the start
    assert abs(lam[1] - lam_all[1]) <= 1e-5 * lam_all[1]
    assert abs(lam[2] - lam_all[2]) <= 1e-2 * lam_all[2]
    assert hist[0]["lambda"][2] - lam_all[2] > 100 * (lam[2] - lam_all[2])
    # the returned columns are A-orthonormal
    GA = J.gram_sums(x, x, prob["prec"], prob["mpo"])
    assert np.abs(GA - np.eye(3)).max() < 1e-10


def test_joint_iteration_spinful_hubbard():
    """Alg. 4 with two spin species (Hubbard L = 3, (n_up, n_dn) = (2, 1), D = 2)
    from the two lowest determinants: Ritz values above the exact eigenvalues at
    every step, and the first one certified by the bound at convergence."""
    from oracle import mpo as M
    from oracle import precond as P
    from synth import hubbard_chain
    wl = hubbard_chain(L=3, n_up=2, n_dn=1, U=2.0)
    H0, _ = OF.sector_hamiltonian(wl.h, wl.eri, 1, 2, 1)
    ev0 = np.linalg.eigvalsh(H0)
    gamma = 0.5 - ev0[0]
    lam = ev0 + gamma
    species = OF.site_species(3, 1)
    t_so, v_so = P.spin_orbital_accessors(wl.h, wl.eri, 1)
    th = P.theta_diag(t_so, v_so, 3, gamma, 6)
    tmin, tmax = P.spectrum_bounds(th, species, (2, 1))
    prec = P.Preconditioner(th, tmin, tmax, 0.1, 0.6)
    mpo = M.build_mpo(wl.h, wl.eri, 1, 3, gamma)
    delta = lam[1] / (lam[1] - lam[0])
    params = PI.SolverParams(0.6, delta, tau=1e-8)
    x = J.from_determinants(species, (2, 1), J.lowest_determinants(species, (2, 1), np.repeat(np.diag(wl.h), 2), 2))
    st = PI.SolverState()
    for _ in range(80):
        x, info = J.step(x, mpo, prec, params, st)
        assert np.all(info["lambda"] >= lam[:2] - 1e-12 * lam[:2])
        if info["converged"]:
            break
    assert info["converged"]
    assert (info["lambda"][0] - lam[0]) / lam[0] <= info["releig_bound"] * (1 + 1e-6) + 1e-13
    assert abs(info["lambda"][1] - lam[1]) <= 1e-4 * lam[1]
