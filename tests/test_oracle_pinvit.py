"""Pins of the oracle's Alg. 2 step against exact diagonalisation and the paper's bounds."""
import math

import numpy as np
import pytest

from oracle import bsmps as B
from oracle import fermion as F
from oracle import mpo as M
from oracle import pinvit as PI
from oracle import precond as P
from synth import spinless_random_chain


def small_problem(K=8, N=4, seed=3, r_max=8, dominant=False, lam1=1.0):
    wl = spinless_random_chain(K=K, N=N, seed=seed)
    if dominant:
        # diagonally dominant variant: D approximates H_gamma well, so c is small
        rng = np.random.default_rng(seed)
        g = 0.05 * rng.standard_normal((K, K))
        wl.h = np.diag(0.8 * np.arange(K)) + g + g.T
        wl.eri = 0.3 * wl.eri
    species = F.site_species(K, 0)
    H0, states = F.sector_hamiltonian(wl.h, wl.eri, 0, N, 0)
    gamma = lam1 - np.linalg.eigvalsh(H0)[0]
    Hf = F.full_hamiltonian(wl.h, wl.eri, 0, N, gamma)
    t_so, v_so = P.spin_orbital_accessors(wl.h, wl.eri, 0)
    th = P.theta_diag(t_so, v_so, N, gamma, K)
    tmin, tmax = P.spectrum_bounds(th, species, (N, 0))
    occ = np.array([[(i >> (K - 1 - s)) & 1 for s in range(K)] for i in range(1 << K)])
    in_sector = occ.sum(1) == N
    Dv = occ[in_sector] @ th
    Hs = Hf[np.ix_(in_sector, in_sector)]
    ev = np.linalg.eigvalsh(Hs / np.sqrt(np.outer(Dv, Dv)))
    alpha0, c = P.alpha0_and_c(0.1, tmin, ev[0], ev[-1])
    prec = P.Preconditioner(th, tmin, tmax, 0.1, alpha0)
    lam = np.linalg.eigvalsh(Hs)[:2]
    delta = lam[1] / (lam[1] - lam[0])
    mpo = M.build_mpo(wl.h, wl.eri, 0, N, gamma)
    dims = B.default_dims(species, (N, 0), r_max)
    tmp = B.BSMPS(species, (N, 0), dims, [dict() for _ in range(K)])
    _, tot = tmp.layout()
    x0 = B.BSMPS.from_flat(species, (N, 0), dims, np.random.default_rng(seed).standard_normal(tot))
    Sd = prec.dense_diag(occ)
    return dict(Hf=Hf, Sd=Sd, in_sector=in_sector, lam=lam, c=c, delta=delta,
                prec=prec, mpo=mpo, x0=x0)


@pytest.fixture(scope="module")
def prob():
    return small_problem()


def test_rayleigh_quotient_matches_dense(prob):
    x = prob["x0"]
    xd = B.to_dense(x)
    Sx = prob["Sd"] * xd
    lam, num, den = PI.rayleigh(x, prob["prec"], prob["mpo"])
    assert abs(num - Sx @ prob["Hf"] @ Sx) < 1e-10 * abs(num)
    assert abs(den - Sx @ Sx) < 1e-12 * abs(den)
    assert lam >= prob["lam"][0] - 1e-12


def test_residual_error_within_eta(prob):
    # Sec. 5.3.1: ||res_eta(x) - r(x)|| <= eta with r(x) = A x - lambda E x
    x = prob["x0"]
    lam, num, den = PI.rayleigh(x, prob["prec"], prob["mpo"])
    x = B.scale(x, 1 / math.sqrt(num))
    xd = B.to_dense(x)
    S, H = prob["Sd"], prob["Hf"]
    r_exact = S * (H @ (S * xd)) - lam * S * S * xd
    terms = PI.residual_terms(x, lam, prob["prec"], prob["mpo"])
    assert abs(sum(e[2] for e in terms) - sum(np.linalg.norm(B.to_dense(e[1])) for e in terms)) < 1e-10
    for eta in [1e-1, 1e-3, 1e-6]:
        r = PI.assemble_residual(terms, eta * np.linalg.norm(r_exact))
        assert np.linalg.norm(B.to_dense(r) - r_exact) <= eta * np.linalg.norm(r_exact) * (1 + 1e-9)


def test_two_by_two_rayleigh_ritz_is_minimal():
    rng = np.random.default_rng(0)
    for _ in range(20):
        X = rng.standard_normal((6, 2))
        Hm = rng.standard_normal((6, 6)); Hm = Hm @ Hm.T + np.eye(6)
        GH, GE = X.T @ Hm @ X, X.T @ X
        lam, v = PI.rr2(GH, GE)
        assert abs((v @ GH @ v) / (v @ GE @ v) - lam) < 1e-12
        assert abs(v @ GE @ v - 1) < 1e-12 and v[0] > 0
        for th in np.linspace(0, np.pi, 50):
            w = np.array([np.cos(th), np.sin(th)])
            assert (w @ GH @ w) / (w @ GE @ w) >= lam - 1e-12


def test_bounds_formulas():
    # Eq. (nicesin2bound) tends to its Taylor form rho^2 delta^2 from above
    # (for delta >= 2, where the second-order term is positive)
    for delta in (3.0, 10.9096):
        prev = math.inf
        for rho in (1e-2, 1e-3, 1e-4, 1e-5):
            b = PI.bdelta(rho, delta)
            s2 = delta * b * rho * rho
            ratio = s2 / (rho * delta) ** 2
            assert ratio >= 1.0 and ratio - 1.0 < prev
            prev = ratio - 1.0
        assert prev < 1e-6
    # b_delta is not real beyond rho^2 > 1/(4 delta (delta - 1))
    d = 3.0
    assert PI.bdelta(math.sqrt(1 / (4 * d * (d - 1))) * 1.01, d) is None
    assert PI.eigvec_bound(0.9, 3.0) == math.inf


@pytest.fixture(scope="module")
def prob_dominant():
    return small_problem(K=6, N=3, r_max=6, dominant=True, lam1=0.5)


def test_iteration_decrease_bounds_and_convergence(prob_dominant):
    prob = prob_dominant
    lam1 = prob["lam"][0]
    params = PI.SolverParams(prob["c"], prob["delta"], tau=1e-6)
    st = PI.SolverState()
    x = prob["x0"]
    infos = []
    for it in range(25):
        x, info = PI.step(x, prob["mpo"], prob["prec"], params, st)
        infos.append(info)
        assert info["lambda"] >= lam1 - 1e-10                # Rayleigh quotient above lambda_1
        # a-posteriori bounds are upper bounds of the true errors where Lemma lambdaqbound
        # applies: rho real-valued b_delta and lambda_1/lambda >= (2 delta - 2)/(2 delta - 1)
        d = prob["delta"]
        if math.isfinite(info["releig_bound"]) and lam1 / info["lambda"] >= (2 * d - 2) / (2 * d - 1):
            assert (info["lambda"] - lam1) / lam1 <= info["releig_bound"] * (1 + 1e-6) + 1e-13
        if info["converged"]:
            break
    for a, b in zip(infos[:-1], infos[1:]):
        if "lambda_star" in a:
            # Thm. conv (ii): lambda(x') <= lambda_* + t_eig (lambda(x) - lambda_*)
            assert b["lambda"] <= a["lambda_star"] + 0.5 * (a["lambda"] - a["lambda_star"]) + 1e-10
    assert infos[-1]["converged"]
    assert infos[-1]["lambda"] - lam1 < 1e-9


def _bisect_delta(rho, q):
    """Root of g(D) = sqrt(1 - D^2) - rho D - q on [0, 1] by bisection (g decreases)."""
    lo, hi = 0.0, 1.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if math.sqrt(1.0 - mid * mid) - rho * mid - q > 0.0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


@pytest.mark.parametrize("rho", [1e-8, 1e-3, 0.1, 0.5, 1.0, 3.0])
@pytest.mark.parametrize("q", [1e-3, 0.3, 0.7, 0.99, 1.0])
def test_delta_A_solves_its_defining_equation(rho, q):
    # Sec. 5.3.2: Delta_A is the solution in [0, 1] of sqrt(1 - Delta^2) - rho Delta = q
    # (checked in the squared form 1 - D^2 = (q + rho D)^2 with q + rho D >= 0, which
    # is well conditioned also where D is close to 1, plus an independent bisection)
    d = PI.delta_A(rho, q)
    assert 0.0 <= d <= 1.0
    assert q + rho * d >= 0.0
    assert abs((1.0 - d * d) - (q + rho * d) ** 2) <= 4e-16 * (1.0 + rho) ** 2
    assert abs(d - _bisect_delta(rho, q)) <= 1e-13


@pytest.mark.parametrize("rho", [1e-3, 0.5])
@pytest.mark.parametrize("q", [1.0 + 1e-12, 1.2])
def test_delta_A_clamped_when_q_exceeds_one(rho, q):
    # q > 1 (lambda_* above lambda^n at machine precision) has no root in [0, 1]:
    # the tolerance is clamped to 0
    assert PI.delta_A(rho, q) == 0.0


def test_compression_of_u_keeps_the_step(prob, monkeypatch):
    # reading of Sec. 5.3.1: u_k' compressed at U_REL ||u_k'|| = 1e-13 ||u_k'|| gives the
    # same iteration as the exactly applied terms (U_REL = 0) to 1e-12
    params = PI.SolverParams(prob["c"], prob["delta"], tau=1e-14, r_max=8)
    runs = []
    for u_rel in (0.0, 1e-13):
        monkeypatch.setattr(PI, "U_REL", u_rel)
        st = PI.SolverState()
        x = prob["x0"]
        infos = []
        for _ in range(3):
            x, info = PI.step(x, prob["mpo"], prob["prec"], params, st)
            infos.append(info)
        runs.append((infos, x))
    (ia, xa), (ib, xb) = runs
    for a, b in zip(ia, ib):
        assert abs(a["lambda"] - b["lambda"]) <= 1e-12 * abs(a["lambda"])
        assert abs(a["lambda_star"] - b["lambda_star"]) <= 1e-12 * abs(a["lambda_star"])
        assert a["eta_tries"] == b["eta_tries"] and a["ranks"] == b["ranks"]
    da, db = B.to_dense(xa), B.to_dense(xb)
    assert np.linalg.norm(da - db) <= 1e-12 * np.linalg.norm(da)
