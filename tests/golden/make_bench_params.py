"""Write the solver constants of the Hubbard L=32 bench workload (oracle only).

C_lower / C_upper of D^{-1/2} H_gamma D^{-1/2} (Eq. (lowerupper)) and delta are
computed by exact diagonalisation for the half-filled open Hubbard chains
L = 6 and L = 8 (t = 1, U = 4) and extrapolated to L = 32 with the rule of
Sec. 7.1.3: C_L = C_8^{1+k} C_6^{-k}, delta_L = max(delta_8, delta_8^{1+k}
delta_6^{-k}), k = (L - 8)/2 (the paper extrapolates from K = 12, 14 in
steps of two orbitals; here the step is two spatial sites).  alpha_0 and c
follow Eq. (Sdef) and Eq. (precondcdef) with c0 = 0.1.  The shift is
gamma = 1 - E_lb with E_lb the free-fermion energy (a lower bound for U >= 0).

Run: python tests/golden/make_bench_params.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import fermion as F  # noqa: E402
from oracle import precond as P  # noqa: E402
from synth import hubbard_chain  # noqa: E402


def constants(L, U=4.0):
    wl = hubbard_chain(L=L, U=U)
    n = L // 2
    ev = np.sort(np.linalg.eigvalsh(wl.h))
    gamma = 1.0 - 2.0 * ev[:n].sum()
    H, states = F.sector_hamiltonian(wl.h, wl.eri, 1, n, n, gamma=gamma)
    t_so, v_so = P.spin_orbital_accessors(wl.h, wl.eri, 1)
    th = P.theta_diag(t_so, v_so, L, gamma, 2 * L)
    occ = np.array([[(int(m) >> s) & 1 for s in range(2 * L)] for m in states])
    Dv = occ @ th
    mu = np.linalg.eigvalsh(H / np.sqrt(np.outer(Dv, Dv)))
    lam = np.linalg.eigvalsh(H)[:2]
    return {"L": L, "gamma": gamma, "C_lower": float(mu[0]), "C_upper": float(mu[-1]),
            "lambda1": float(lam[0]), "lambda2": float(lam[1]),
            "delta": float(lam[1] / (lam[1] - lam[0]))}


def main(L=32, U=4.0, c0=0.1):
    lo, hi = constants(6, U), constants(8, U)
    k = (L - 8) / 2.0
    cl = hi["C_lower"] ** (1 + k) * lo["C_lower"] ** (-k)
    cu = hi["C_upper"] ** (1 + k) * lo["C_upper"] ** (-k)
    delta = max(hi["delta"], hi["delta"] ** (1 + k) * lo["delta"] ** (-k))
    wl = hubbard_chain(L=L, U=U)
    n = L // 2
    ev = np.sort(np.linalg.eigvalsh(wl.h))
    gamma = 1.0 - 2.0 * ev[:n].sum()
    t_so, v_so = P.spin_orbital_accessors(wl.h, wl.eri, 1)
    th = P.theta_diag(t_so, v_so, L, gamma, 2 * L)
    tmin, tmax = P.spectrum_bounds(th, tuple(s % 2 for s in range(2 * L)), (n, n))
    alpha0, c = P.alpha0_and_c(c0, tmin, cl, cu)
    out = {"citation": "Sec. 7.1.3 (extrapolation of C_lower, C_upper, delta from two smaller sizes); "
                       "Eq. (Sdef), Eq. (precondcdef); written by tests/golden/make_bench_params.py",
           "workload": f"hubbard_chain L={L} t=1 U={U} n_up=n_dn={n}",
           "small_sizes": [lo, hi], "C_lower": cl, "C_upper": cu, "delta": delta,
           "gamma": gamma, "t_min": tmin, "t_max": tmax, "c0": c0, "alpha0": alpha0, "c": c,
           "eps_num": 0.5 * (1 - c), "t_eig": 0.5}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"bench_params_hubbard_L{L}.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path, json.dumps({k_: out[k_] for k_ in ("C_lower", "C_upper", "delta", "c", "alpha0", "gamma")}))


if __name__ == "__main__":
    main()
