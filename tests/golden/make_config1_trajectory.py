"""Write the oracle's Alg. 2 trajectory on the spinless random chain K = 12, N = 6
(oracle only; the GPU test compares the library with it step by step).

Workload: h_pq ~ N(0,1) exp(-|p-q|/3) + 0.5 p on the diagonal, (pq|rs) from
8 Cholesky vectors scaled by 0.1 (synth.spinless_random_chain, seed 0); the
random charge-conserving start of maximal rank 32 (block entries
synth.random_block_values, seed 0); 20 steps of Alg. 2 with the rank cap 32.

Constants, all by exact diagonalisation in the 924-dimensional sector:
gamma = 1 - E_0 (so lambda_1 = 1); C_lower / C_upper of D^{-1/2} H_gamma
D^{-1/2} (Eq. (lowerupper)) with theta of Sec. 7.1.1; alpha_0 and c by
Eq. (Sdef) and Eq. (precondcdef) with c_0 = 0.1 (Sec. 7.1.3);
delta = lambda_2 / (lambda_2 - lambda_1) (Alg. 2); eps_num = (1 - c)/2 and
t_eig = 1/2 (Sec. 7.1.3).

Run: python tests/golden/make_config1_trajectory.py   (about 10 minutes)
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import bsmps as B  # noqa: E402
from oracle import fermion as F  # noqa: E402
from oracle import mpo as M  # noqa: E402
from oracle import pinvit as PI  # noqa: E402
from oracle import precond as P  # noqa: E402
from synth import random_block_values, spinless_random_chain  # noqa: E402

K, N, R_MAX, SEED, STEPS, C0 = 12, 6, 32, 0, 20, 0.1


def constants(wl):
    H0, states = F.sector_hamiltonian(wl.h, wl.eri, 0, N, 0)
    ev = np.linalg.eigvalsh(H0)
    gamma = 1.0 - ev[0]
    t_so, v_so = P.spin_orbital_accessors(wl.h, wl.eri, 0)
    th = P.theta_diag(t_so, v_so, N, gamma, K)
    species = F.site_species(K, 0)
    tmin, tmax = P.spectrum_bounds(th, species, (N, 0))
    occ = np.array([[(int(m) >> s) & 1 for s in range(K)] for m in states])
    Dv = occ @ th
    Hg = H0 + gamma * np.eye(len(H0))
    mu = np.linalg.eigvalsh(Hg / np.sqrt(np.outer(Dv, Dv)))
    alpha0, c = P.alpha0_and_c(C0, tmin, float(mu[0]), float(mu[-1]))
    lam = ev[:2] + gamma
    return {"gamma": float(gamma), "theta": th.tolist(), "t_min": float(tmin), "t_max": float(tmax),
            "C_lower": float(mu[0]), "C_upper": float(mu[-1]), "c0": C0, "alpha0": float(alpha0),
            "c": float(c), "eps_num": 0.5 * (1.0 - c), "t_eig": 0.5,
            "lambda1": float(lam[0]), "lambda2": float(lam[1]),
            "delta": float(lam[1] / (lam[1] - lam[0]))}


def main():
    wl = spinless_random_chain(K=K, N=N, r_max=R_MAX, seed=SEED)
    cst = constants(wl)
    W = M.build_mpo(wl.h, wl.eri, 0, N, cst["gamma"])
    prec = P.Preconditioner(np.array(cst["theta"]), cst["t_min"], cst["t_max"], C0, cst["alpha0"])
    params = PI.SolverParams(cst["c"], cst["delta"], eps_num=cst["eps_num"], t_eig=cst["t_eig"], tau=1e-14,
                             r_max=R_MAX)
    species = F.site_species(K, 0)
    dims = B.default_dims(species, (N, 0), R_MAX)
    n = B.BSMPS(species, (N, 0), dims, [dict() for _ in range(K)]).layout()[1]
    x = B.BSMPS.from_flat(species, (N, 0), dims, random_block_values(n, SEED))
    st = PI.SolverState()
    steps = []
    for i in range(STEPS):
        t0 = time.time()
        x, info = PI.step(x, W, prec, params, st)
        rec = {k: info[k] for k in ("lambda", "rho", "eta_res", "res_norm", "eta_tries", "bound",
                                    "releig_bound", "converged")}
        for k in ("lambda_star", "eta_in", "delta_A", "cap_discarded"):
            if k in info:
                rec[k] = info[k]
        rec["bonds"] = [sorted([list(q), d] for q, d in b.items()) for b in x.bonds]
        steps.append(rec)
        print(i, round(time.time() - t0, 1), info["lambda"], info["eta_tries"], max(x.ranks()), flush=True)
        if info["converged"]:
            break
    out = {"citation": "Alg. 2 (inner PINVIT) with the residual of Sec. 5.3.1 and the constants of Sec. 7.1.3; "
                       "written by tests/golden/make_config1_trajectory.py from the oracle alone",
           "workload": {"K": K, "N": N, "r_max": R_MAX, "seed": SEED, "n_values": n},
           "constants": cst, "steps": steps}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_config1_trajectory.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path)


if __name__ == "__main__":
    main()
