"""Perturbed inverse subspace iteration on joint block MPS (Alg. 4, Sec. 6).

Test infrastructure only (see ``oracle/__init__.py``).

X = (x_1, ..., x_D) is one block-sparse MPS whose last bond (target sector)
has dimension D: the eigenvector-specific core of Sec. 6.2 sits after the last
site (position p = K + 1) and is absorbed into the last core.  Inner bonds
stack the vectors' bases block-diagonally, so their ranks are at most the sums
of the individual ranks.

Readings of the paper used here:
* Position of the joint core: after the last site (p = K + 1), one of the
  positions Sec. 6.2 allows.  Gram matrices <y_i, O z_j> are then the last
  left environment; column mixing X V multiplies the last core.
* Initial value: the D determinants with the smallest diagonal one-particle
  energy sum_{i occupied} t_ii (ties: occupation strings compared with site 0
  first, occupied before empty), so that the first is e_1 of Sec. 7.1.4.
* The Rayleigh--Ritz steps use the full Gram matrices of the represented
  columns (the paper substitutes the known Lambda^n block; both agree when the
  columns are A-orthonormal).  Generalised eigenvectors are normalised to
  V^T G_E V = I, then scaled by lambda^{-1/2} so the new columns are
  A-orthonormal; the largest-|.| entry of each column is made positive.
* Norms of joint terms (the sorted residual sum, eta_res) are Frobenius norms
  over all columns; the column norms ||r_i|| decide the eta_res loop and
  rho_i, as Alg. 4 prints.
* The termination test uses rho_1 (the lowest Ritz value), as in Alg. 4.
* Residual terms are formed as in Alg. 2 (reading in ``pinvit``):
  u_k' = H_gamma S_k' X - S_k' X Lambda applied exactly (the Lambda term enters
  on the identity rail of the MPO), compressed once at U_REL ||u_k'||, and
  s_{k,k'} = S_k u_k'.
"""

import itertools
import math

import numpy as np

from . import bsmps as B
from .pinvit import MAX_ETA_RETRIES, U_REL, delta_A, eigvec_bound, releig_bound


def lowest_determinants(species, target, t_diag, D):
    """Occupation strings of the D lowest diagonal energies in the sector
    (reading above).  Enumerates the sector: small K only."""
    K = len(species)
    sites = [[t for t in range(K) if species[t] == s] for s in (0, 1)]
    cand = []
    for occ0 in itertools.combinations(sites[0], target[0]):
        for occ1 in itertools.combinations(sites[1], target[1]):
            occ = [0] * K
            for t in occ0 + occ1:
                occ[t] = 1
            e = 0.0
            for t in range(K):
                if occ[t]:
                    e += t_diag[t]
            cand.append((e, tuple(-o for o in occ), tuple(occ)))
    cand.sort()
    assert len(cand) >= D, "sector smaller than D"
    return [c[2] for c in cand[:D]]


def from_determinants(species, target, occs):
    """Joint block MPS of the unit vectors e_i given by the occupation strings
    (Sec. 6.2): vector i owns one basis index per bond (block-diagonal stacking),
    the first core places the vectors side by side, the last core ends in
    column i."""
    K = len(species)
    D = len(occs)
    charges = []
    for occ in occs:
        q = (0, 0)
        path = [q]
        for t in range(K):
            q = B.add_charge(q, B.delta(species[t], occ[t]))
            path.append(q)
        assert q == tuple(target)
        charges.append(path)
    pos = [[0] * (K + 1) for _ in range(D)]
    bonds = []
    for b in range(K + 1):
        cnt = {}
        for i in range(D):
            q = charges[i][b]
            if b == 0:
                cnt[q] = 1
                pos[i][b] = 0
            elif b == K:
                cnt[q] = D
                pos[i][b] = i
            else:
                pos[i][b] = cnt.get(q, 0)
                cnt[q] = pos[i][b] + 1
        bonds.append(dict(sorted(cnt.items())))
    cores = [dict() for _ in range(K)]
    for t in range(K):
        for i in range(D):
            n, m = charges[i][t], charges[i][t + 1]
            key = (n, occs[i][t])
            if key not in cores[t]:
                cores[t][key] = np.zeros((bonds[t][n], bonds[t + 1][m]))
            cores[t][key][pos[i][t], pos[i][t + 1]] = 1.0
    # blocks of the layout that no vector touches are zero
    x = B.BSMPS(species, target, bonds, cores)
    for t in range(K):
        for (n, sg) in x.block_keys(t):
            m = B.add_charge(n, B.delta(species[t], sg))
            if (n, sg) not in x.cores[t]:
                x.cores[t][(n, sg)] = np.zeros((bonds[t][n], bonds[t + 1][m]))
    return x


def gram_sums(a, b, prec, mpo=None):
    """a^T A b = sum_{k,k'} (S_k a)^T H_gamma (S_k' b), or a^T E b with mpo=None
    (Sec. 6.1, summation formulas)."""
    G = np.zeros((B.columns(a), B.columns(b)))
    for k in range(prec.n_terms):
        fa0, fa1 = prec.factors(k)
        Sa = B.scale_sites(a, fa0, fa1)
        for kp in range(prec.n_terms):
            fb0, fb1 = prec.factors(kp)
            G += B.gram(Sa, B.scale_sites(b, fb0, fb1), mpo)
    return G


def frob(x):
    """Frobenius norm over all columns."""
    return float(math.sqrt(max(np.trace(B.gram(x, x)), 0.0)))


def column_norms(x):
    return np.sqrt(np.maximum(np.diag(B.gram(x, x)), 0.0))


def ritz(GA, GE, n):
    """Lowest n eigenpairs of the pencil (GA, GE) (library generalised eigh),
    columns normalised to V^T GE V = I, then scaled to V^T GA V = I; the
    largest-|.| entry of each column is positive."""
    import scipy.linalg
    w, V = scipy.linalg.eigh(GA, GE)
    w, V = w[:n], V[:, :n].copy()
    for i in range(n):
        V[:, i] /= math.sqrt(V[:, i] @ GE @ V[:, i])
        j = int(np.argmax(np.abs(V[:, i])))
        if V[j, i] < 0:
            V[:, i] = -V[:, i]
    return w, V / np.sqrt(w)[None, :]


def residual_terms(X, lams, prec, mpo):
    """s_{k,k'} = S_k (H_gamma S_k' X - S_k' X Lambda) and their norms (Eq. (respara))."""
    terms = []
    for kp in range(prec.n_terms):
        f0, f1 = prec.factors(kp)
        u = B.apply_exact(mpo, B.scale_sites(X, f0, f1), 0.0, col_shift=-np.asarray(lams))
        u, _, _ = B.truncate(u, U_REL * frob(u))
        for k in range(prec.n_terms):
            g0, g1 = prec.factors(k)
            s = B.scale_sites(u, g0, g1)
            terms.append(((k, kp), s, frob(s)))
    return terms


def assemble_residual(terms, eta):
    """res_eta(X): the sorted truncated sum of Sec. 5.3.1 on joint terms."""
    order = sorted(terms, key=lambda e: (e[2], e[0]))
    acc = 0.0
    j0 = 0
    while j0 < len(order) and acc + order[j0][2] <= eta / 3.0:
        acc += order[j0][2]
        j0 += 1
    rest = order[j0:]
    tail = sum(e[2] for e in rest)
    y = None
    for (_, s, ns) in rest:
        eps_j = eta * ns / (3.0 * tail) if tail > 0 else 0.0
        z = s if y is None else B.add(y, s)
        y, _, _ = B.truncate(z, eps_j)
    if y is None:
        return None
    y, _, _ = B.truncate(y, eta / 3.0)
    return y


def step(X, mpo, prec, params, state):
    """One pass of the loop body of Alg. 4.  Returns (X_next, info); when the
    termination test holds, X_next is the Ritz-rotated X^n."""
    D = B.columns(X)
    # Rayleigh--Ritz on span X^n: A-orthonormal columns, Lambda^n
    lams, V = ritz(gram_sums(X, X, prec, mpo), gram_sums(X, X, prec, None), D)
    X = B.mix_columns(X, V)
    zeta = params.zeta_res
    terms = residual_terms(X, lams, prec, mpo)
    eta = min(2.0 * state.eta_res, 0.8 * zeta * sum(e[2] for e in terms))
    tries = 0
    while True:
        R = assemble_residual(terms, eta)
        rn = np.zeros(D) if R is None else column_norms(R)
        if rn.min() >= (1.0 + 1.0 / zeta) * eta or tries >= MAX_ETA_RETRIES:
            break
        eta *= 0.8
        tries += 1
    state.eta_res = eta
    rho = (rn + eta) / math.sqrt(1.0 - params.c)       # ||x_i||_A = 1
    bound = eigvec_bound(rho[0], params.delta)
    info = {"n": state.n, "lambda": lams.copy(), "rho": rho.copy(), "eta_res": eta,
            "res_norms": rn.copy(), "eta_tries": tries, "bound": bound,
            "releig_bound": releig_bound(rho[0], params.delta), "converged": False}
    if bound <= params.tau or R is None:
        info["converged"] = True
        state.history.append(info)
        return X, info
    # Rayleigh--Ritz on span (X^n R^n) in the normalised basis (Sec. 6.1)
    GA = np.block([[gram_sums(X, X, prec, mpo), gram_sums(X, R, prec, mpo)],
                   [gram_sums(R, X, prec, mpo), gram_sums(R, R, prec, mpo)]])
    GE = np.block([[gram_sums(X, X, prec, None), gram_sums(X, R, prec, None)],
                   [gram_sums(R, X, prec, None), gram_sums(R, R, prec, None)]])
    xi = np.sqrt(np.diag(GE))
    Bm = GA / np.outer(xi, xi)
    Mm = GE / np.outer(xi, xi)
    Bm = 0.5 * (Bm + Bm.T)
    Mm = 0.5 * (Mm + Mm.T)
    lam_star, W = ritz(Bm, Mm, D)
    W1 = W[:D] / xi[:D, None]
    W2 = W[D:] / xi[D:, None]
    Xstar = B.add(B.mix_columns(X, W1), B.mix_columns(R, W2))
    dA = np.array([delta_A(rho[i], math.sqrt(lam_star[i] / (lam_star[i] + params.t_eig * (lams[i] - lam_star[i]))))
                   for i in range(D)])
    eta_in = dA.min() / math.sqrt(1.0 + params.c)       # ||X*_i||_A = 1
    Xn, _, cap = B.truncate(Xstar, eta_in, params.r_max)
    info.update({"lambda_star": lam_star.copy(), "eta_in": eta_in, "delta_A": dA,
                 "ranks": Xn.ranks(), "cap_discarded": cap})
    state.history.append(info)
    state.n += 1
    return Xn, info
