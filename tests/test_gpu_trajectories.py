"""Alg. 2 trajectories of the CUDA path against the oracle, step by step.

* The spinless random chain K = 12, N = 6 (sector dimension 924) from the
  random charge-conserving start of maximal rank 32 (seed 0), 20 steps with
  the rank cap 32 and the constants of exact diagonalisation: against the
  oracle's trajectory stored in tests/golden/oracle_config1_trajectory.json
  (written by tests/golden/make_config1_trajectory.py from the oracle alone;
  twenty oracle steps take about ten minutes on one core).  Per step: lambda
  to 1e-10 relative, the same eta_res passes, the same bonds (sector dims,
  bit-exact) of the next iterate; the final Rayleigh quotient against the
  exact lambda_1 of the sector.
* The open Hubbard chain L = 32 (64 spin-orbital sites, half filling, U = 4)
  from e_1 with the bench's constants: three steps against the oracle run in
  the test.
"""
import json
import os

import numpy as np
import pytest

from oracle import bsmps as OB
from oracle import fermion as OF
from oracle import mpo as OM
from oracle import pinvit as OPI
from oracle import precond as OP
from synth import hubbard_chain, random_block_values, spinless_random_chain

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden", "oracle_config1_trajectory.json")


@pytest.fixture(scope="module")
def nat():
    from paper_2604_16118_gb300 import build, native
    build.build()
    return native


@pytest.fixture(scope="module")
def ctx(nat):
    return nat.Context(0)


def bonds_of(rec_bonds):
    return [{tuple(q): d for q, d in b} for b in rec_bonds]


def test_config1_twenty_steps_match_oracle_trajectory(nat, ctx):
    g = json.load(open(GOLD))
    w, cst = g["workload"], g["constants"]
    wl = spinless_random_chain(K=w["K"], N=w["N"], r_max=w["r_max"], seed=w["seed"])
    vals = random_block_values(w["n_values"], w["seed"])
    x = nat.mps_create(ctx, wl.n_orb, 0, wl.n_up, 0, w["r_max"], vals)
    W = nat.mpo_from_integrals(ctx, wl.h, wl.eri, 0, wl.n_up, cst["gamma"])
    p = nat.make_precond(np.array(cst["theta"]), cst["t_min"], cst["t_max"], cst["c0"], cst["alpha0"])
    prm = nat.solver_params(cst["c"], cst["delta"], eps_num=cst["eps_num"], t_eig=cst["t_eig"], tau=1e-14,
                            r_max=w["r_max"])
    st = nat.solver_state()
    worst = 0.0
    for i, rec in enumerate(g["steps"]):
        x, info = nat.eigensolve_step(ctx, W, p, prm, st, x)
        rel = abs(info["lambda"] - rec["lambda"]) / abs(rec["lambda"])
        worst = max(worst, rel)
        assert rel <= 1e-10, (i, info["lambda"], rec["lambda"])
        assert info["eta_tries"] == rec["eta_tries"], i
        assert info["converged"] == int(rec["converged"]), i
        assert abs(info["rho"] - rec["rho"]) <= 1e-8 * rec["rho"], i
        assert x.bonds() == bonds_of(rec["bonds"]), i
    # the Rayleigh quotients stay above, and approach, the exact lambda_1 of the sector
    lam1 = cst["lambda1"]
    assert all(r["lambda"] >= lam1 - 1e-10 for r in g["steps"])
    assert info["lambda"] - lam1 <= 1e-3 * lam1
    print(f"config 1: 20 steps, worst relative lambda difference {worst:.2e}, "
          f"final lambda - lambda_1 = {info['lambda'] - lam1:.3e}")


def test_hubbard_L32_three_steps_match_oracle(nat, ctx):
    import bench
    S = bench.setup(ctx, nat, seed=None)
    prm = bench.load_params(32)
    L, n = 32, 16
    wl = hubbard_chain(L=L)
    gamma = 1.0 - OP.energy_lower_bound(wl.h, wl.eri, 1, n, n, cholesky=False)
    assert abs(gamma - S["gamma"]) <= 1e-12 * gamma
    oW = OM.build_mpo(wl.h, wl.eri, 1, 2 * n, gamma)
    t_so, v_so = OP.spin_orbital_accessors(wl.h, wl.eri, 1)
    species = OF.site_species(L, 1)
    th = OP.theta_diag(t_so, v_so, 2 * n, gamma, 2 * L)
    tmin, tmax = OP.spectrum_bounds(th, species, (n, n))
    prec = OP.Preconditioner(th, tmin, tmax, prm["c0"], prm["alpha0"])
    oprm = OPI.SolverParams(prm["c"], prm["delta"], eps_num=prm["eps_num"], t_eig=prm["t_eig"], tau=1e-8,
                            r_max=256)
    ost = OPI.SolverState()
    ox = OB.e1_mps(species, (n, n))
    st = nat.solver_state()
    x = S["x"]
    for i in range(3):
        x, info = nat.eigensolve_step(ctx, S["W"], S["p"], S["sp"], st, x)
        ox, oinfo = OPI.step(ox, oW, prec, oprm, ost)
        assert abs(info["lambda"] - oinfo["lambda"]) <= 1e-10 * abs(oinfo["lambda"]), i
        assert info["eta_tries"] == oinfo["eta_tries"], i
        assert abs(info["rho"] - oinfo["rho"]) <= 1e-8 * oinfo["rho"], i
        assert x.bonds() == ox.bonds, i
