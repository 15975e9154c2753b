"""Write the solver constants of the Alg. 4 bench workload (oracle only).

The paper's simultaneous-eigenvalue experiment (Sec. 7.2, D = 4): the
Coulomb-like model with K = 14 orbitals, N = 4, gamma = 4 (finite-difference
orbitals on 8192 grid points).  By exact diagonalisation of the N-particle
sector, as the paper does for K <= 14 (Sec. 7.1.3): C_lower / C_upper of
S H_gamma S with alpha_0 = 1 (Eq. (lowerupper)), alpha_0 = sqrt(2 / (C_l + C_u))
(centres the spectrum at 1), c = (C_u - C_l) / (C_u + C_l) (Eq. (precondcdef)),
the lowest six eigenvalues of H_gamma and delta = lambda_2 / (lambda_2 - lambda_1).
c_0 = 0.1; t_min / t_max by the reading of the oracle's spectrum_bounds.

Run: python tests/golden/make_joint_params.py
"""
import json
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import fermion as F  # noqa: E402
from oracle import precond as P  # noqa: E402
from synth import coulomb_1d  # noqa: E402

K, N, GAMMA, C0, N_GRID = 14, 4, 4.0, 0.1, 8192


def main():
    wl = coulomb_1d(K=K, N=N, n_grid=N_GRID)
    t_so, v_so = P.spin_orbital_accessors(wl.h, wl.eri, 0)
    th = P.theta_diag(t_so, v_so, N, GAMMA, K)
    tmin, tmax = P.spectrum_bounds(th, F.site_species(K, 0), (N, 0), t_diag=np.diag(wl.h))
    H, states = F.sector_hamiltonian(wl.h, wl.eri, 0, N, 0, gamma=GAMMA)
    prec = P.Preconditioner(th, tmin, tmax, C0, 1.0)
    occ = np.array([[(int(m) >> s) & 1 for s in range(K)] for m in states])
    S = prec.dense_diag(occ)
    mu = np.linalg.eigvalsh(S[:, None] * H * S[None, :])
    lam = np.linalg.eigvalsh(H)[:6]
    Cl, Cu = float(mu[0]), float(mu[-1])
    out = {
        "workload": f"coulomb_1d K={K} N={N} gamma={GAMMA} n_grid={N_GRID}",
        "c0": C0,
        "alpha0": math.sqrt(2.0 / (Cl + Cu)),
        "c": (Cu - Cl) / (Cu + Cl),
        "delta": float(lam[1] / (lam[1] - lam[0])),
        "t_eig": 0.5,
        "lambda_exact": [float(v) for v in lam],
        "C_lower": Cl,
        "C_upper": Cu,
    }
    out["eps_num"] = 0.5 * (1.0 - out["c"])
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "bench_params_coulomb14_D4.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
