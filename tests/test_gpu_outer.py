"""Outer iteration (Alg. 3) on the GPU vs the oracle, through the C ABI.

Same problems as the Alg. 2 step parity test; tolerances as there (lambda
1e-10 relative, ranks and step counts exact)."""
import numpy as np
import pytest

from oracle import pinvit as OPI
from synth import hubbard_chain, spinless_random_chain
from tests._common import oracle_mpo, oracle_random, precond_for
from tests.test_gpu_parity import _small_problem, gpu_random

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nat():
    from paper_2604_16118_gb300 import build, native
    build.build()
    return native


@pytest.fixture(scope="module")
def ctx(nat):
    return nat.Context(0)


@pytest.mark.parametrize("wl,r", [(spinless_random_chain(K=6, N=3, seed=4), 6),
                                  (hubbard_chain(L=3, n_up=2, n_dn=1, U=2.0), 6)])
def test_outer_iteration_matches_oracle(nat, ctx, wl, r):
    gamma, lam = _small_problem(wl)
    th, tmin, tmax, prec = precond_for(wl, gamma, alpha0=0.6)
    c, delta = 0.6, lam[1] / (lam[1] - lam[0])
    W = nat.mpo_from_integrals(ctx, wl.h, wl.eri, wl.spin, wl.n_particles, gamma)
    p = nat.make_precond(th, tmin, tmax, 0.1, 0.6)
    prm = nat.solver_params(c, delta)
    x, vals = gpu_random(nat, ctx, wl, r, 13)
    ox = oracle_random(wl, r, vals)
    tau = 1e-8
    y, recs, ok = nat.eigensolve_outer(ctx, W, p, prm, x, tau, alpha=1.0, max_outer=20, max_inner=60)
    oy, orecs, ook = OPI.outer(ox, oracle_mpo(wl, gamma), prec, OPI.SolverParams(c, delta), tau, alpha=1.0,
                               max_outer=20, max_inner=60)
    assert ok == ook and ok
    assert len(recs) == len(orecs) >= 2
    for g, o in zip(recs, orecs):
        assert g["inner_steps"] == o["inner_steps"]
        assert g["inner_converged"] == int(o["inner_converged"])
        assert abs(g["lambda"] - o["lambda"]) <= 1e-10 * abs(o["lambda"])
        assert abs(g["eta_out"] - o["eta_out"]) <= 1e-14 * o["eta_out"]
        assert g["max_rank_before"] == max(o["ranks_before"])
        assert g["max_rank_after"] == max(o["ranks_after"])
    assert y.bonds() == oy.bonds
    # the reported relative eigenvalue bound holds against exact diagonalisation
    last = recs[-1]
    assert last["releig_bound"] < tau
    assert (last["lambda"] - lam[0]) / lam[0] <= last["releig_bound"] * (1 + 1e-6) + 1e-12
