"""Pins of the oracle's outer iteration (Alg. 3) against exact diagonalisation.

The problem is small enough for dense vectors: with H_gamma restricted to the
particle sector and S the preconditioner's diagonal, the pencil (S H S, S^2) has
the lower eigenvector u_1 = S^{-1} psi_1 (psi_1 the ground state of H_gamma),
and ||v||_A^2 = (S v)^T H (S v).
"""
import math

import numpy as np
import pytest

from oracle import bsmps as B
from oracle import pinvit as PI
from tests.test_oracle_pinvit import small_problem


@pytest.fixture(scope="module")
def run():
    prob = small_problem(K=6, N=3, r_max=6, dominant=True, lam1=0.5)
    params = PI.SolverParams(prob["c"], prob["delta"])
    y, recs, ok = PI.outer(prob["x0"], prob["mpo"], prob["prec"], params, tau=1e-9, alpha=1.0, keep=True)
    return prob, params, y, recs, ok


def a_norm_distance(prob, u1, v):
    S, H, sec = prob["Sd"], prob["Hf"], prob["in_sector"]
    vd = B.to_dense(v)
    assert np.allclose(vd[~sec], 0.0)
    # align the sign of u1 with v in the A inner product
    Su, Sv = S * u1, S * vd
    if Su @ H @ Sv < 0:
        u1 = -u1
        Su = -Su
    d = Su - Sv
    return math.sqrt(max(d @ H @ d, 0.0))


def ground_u1(prob):
    S, H, sec = prob["Sd"], prob["Hf"], prob["in_sector"]
    Hs = H[np.ix_(sec, sec)]
    w, V = np.linalg.eigh(Hs)
    psi = np.zeros(H.shape[0])
    psi[sec] = V[:, 0]
    u1 = np.zeros_like(psi)
    u1[sec] = psi[sec] / S[sec]
    Su = S * u1
    return u1 / math.sqrt(Su @ H @ Su), w[0]


def test_outer_converges_to_the_ground_energy(run):
    prob, params, y, recs, ok = run
    assert ok
    lam1 = prob["lam"][0]
    last = recs[-1]
    assert last["releig_bound"] < 1e-9
    # the reported bound is an upper bound of the true relative error (Eq. (releigerr))
    assert (last["lambda"] - lam1) / lam1 <= last["releig_bound"] * (1 + 1e-6) + 1e-13
    assert len(recs) >= 2   # the test exercises at least one outer truncation


def test_inner_result_within_tau_m(run):
    # Thm. aposterbound: after the inner iteration ||u_1 - y^+||_A <= tau_m
    prob, params, y, recs, ok = run
    u1, _ = ground_u1(prob)
    for r in recs:
        if r["inner_converged"]:
            assert a_norm_distance(prob, u1, r["y_plus"]) <= r["tau_m"] * (1 + 1e-6) + 1e-12


def test_outer_iterates_within_eta(run):
    # Thm. quasioptr: ||u_1 - y^{m+1}||_A <= eta_{m+1} = eta_m / 2
    prob, params, y, recs, ok = run
    u1, _ = ground_u1(prob)
    for r in recs:
        if "y_next" in r:
            assert a_norm_distance(prob, u1, r["y_next"]) <= 0.5 * r["eta_out"] * (1 + 1e-9)


def test_outer_truncation_never_raises_ranks(run):
    prob, params, y, recs, ok = run
    for r in recs:
        assert all(a <= b for a, b in zip(r["ranks_after"], r["ranks_before"]))
