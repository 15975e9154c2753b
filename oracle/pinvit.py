"""One step of the perturbed preconditioned inverse iteration (Alg. 2).

Test infrastructure only (see ``oracle/__init__.py``).

Readings of the paper used here:
* Step size of Remark omegamin: with z_1 = Sx/||Sx||, z_2 = Sr/||Sr|| and the
  lower eigenvector v of the 2x2 pencil, the update of Alg. 2 is
  x* = (v_1/||Sx||) x + (v_2/||Sr||) r, i.e. omega = -(v_2 ||Sx||)/(v_1 ||Sr||);
  the printed ratio ||Sr||/||Sx|| is inverted relative to that derivation.
  v is scaled so that v^T G_E v = 1 (then ||x*||_A^2 = lambda_*) and v_1 > 0.
* Delta_A solves sqrt(1 - D^2) - rho D = q in closed form,
  D = (-q rho + sqrt(1 + rho^2 - q^2)) / (1 + rho^2).
* Residual terms s_{k,k'} = S_k (H_gamma - lambda) S_{k'} x are formed from
  u_{k'} = (H_gamma - lambda) S_{k'} x, applied exactly and then compressed
  once with trunc at U_REL ||u_{k'}|| (U_REL = 1e-13, far below any eta_res
  the iteration reaches, so the terms stay exact to working precision; U_REL = 0
  keeps the exactly applied terms); ties in the norm sort are broken by (k, k')
  ascending.
* The iterate truncation x^{n+1} = trunc_{eta_in}(x*) is capped at r_max ranks
  when r_max > 0 (the workload's maximal MPS rank); the cap's discarded norm
  is reported separately.
* The eta_res loop is capped at MAX_ETA_RETRIES passes.
* Delta_A is clamped at 0: at machine precision lambda_* can exceed lambda^n,
  q then exceeds 1 and the closed form turns (slightly) negative.
"""

import math

import numpy as np

from . import bsmps as B

MAX_ETA_RETRIES = 60
U_REL = 1e-13


class SolverParams:
    def __init__(self, c, delta, eps_num=None, t_eig=0.5, tau=1e-8, r_max=0):
        self.r_max = r_max              # rank cap of the iterate (0: none)
        self.c = c                      # spectral equivalence constant, Eq. (specequivA)
        self.delta = delta              # gap bound delta >= lambda_2/(lambda_2 - lambda_1)
        self.eps_num = 0.5 * (1.0 - c) if eps_num is None else eps_num   # Sec. 7.1.3
        self.t_eig = t_eig
        self.tau = tau

    @property
    def zeta_res(self):
        return self.eps_num / (1.0 + self.c)     # Lemma truncr


class SolverState:
    def __init__(self):
        self.eta_res = math.inf
        self.n = 0
        self.history = []


def pair_sums(a, b, prec, mpo=None):
    """sum_{k,k'} <O S_k a, S_k' b> with O = mpo (H_gamma) or the identity (Eq. (exactrq))."""
    tot = 0.0
    for k in range(prec.n_terms):
        fa0, fa1 = prec.factors(k)
        Sa = B.scale_sites(a, fa0, fa1)
        for kp in range(prec.n_terms):
            fb0, fb1 = prec.factors(kp)
            Sb = B.scale_sites(b, fb0, fb1)
            tot += B.dot(Sa, Sb, mpo)
    return tot


def rayleigh(x, prec, mpo):
    """lambda(x) and ||x||_A^2 (Eq. (exactrq), (rayleigh1))."""
    num = pair_sums(x, x, prec, mpo)
    den = pair_sums(x, x, prec, None)
    return num / den, num, den


def residual_terms(x, lam, prec, mpo):
    """s_{k,k'} = S_k (H_gamma - lambda) S_k' x and their norms (Sec. 5.3.1)."""
    terms = []
    for kp in range(prec.n_terms):
        f0, f1 = prec.factors(kp)
        u = B.apply_exact(mpo, B.scale_sites(x, f0, f1), shift=-lam)
        if U_REL > 0.0:
            u, _, _ = B.truncate(u, U_REL * B.norm(u))
        for k in range(prec.n_terms):
            g0, g1 = prec.factors(k)
            s = B.scale_sites(u, g0, g1)
            terms.append(((k, kp), s, B.norm(s)))
    return terms


def assemble_residual(terms, eta):
    """res_eta(x) (Sec. 5.3.1): sort by norm, drop the first J_0 terms whose norms
    sum to <= eta/3, add the rest with y_j = trunc_{eps_j}(y_{j-1} + s_j),
    eps_j = eta ||s_j|| / (3 sum_{i>J_0} ||s_i||), finish with trunc_{eta/3}."""
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


def bdelta(rho, delta):
    """b_delta(rho) of Eq. (bbetarho); None when the square root is not real."""
    disc = 1.0 - 4.0 * (delta - 1.0) * delta * rho * rho
    if disc < 0.0:
        return None
    return 2.0 * delta / (1.0 + 2.0 * delta * rho * rho + math.sqrt(disc))


def eigvec_bound(rho, delta):
    """2 sin(1/2 arcsin(sqrt(delta b_delta(rho)) rho)) (Thm. aposterbound); inf if invalid."""
    b = bdelta(rho, delta)
    if b is None:
        return math.inf
    arg = math.sqrt(delta * b) * rho
    if arg > 1.0:
        return math.inf
    return 2.0 * math.sin(0.5 * math.asin(arg))


def releig_bound(rho, delta):
    """Relative eigenvalue bound of Eq. (releigerr); inf if invalid."""
    b = bdelta(rho, delta)
    if b is None or b * rho * rho >= 1.0:
        return math.inf
    return b / (1.0 - b * rho * rho) * rho * rho


def rr2(GH, GE):
    """Lower eigenpair of the 2x2 pencil (GH, GE) (library generalized eigh)."""
    import scipy.linalg
    w, v = scipy.linalg.eigh(GH, GE)
    vec = v[:, 0]
    vec = vec / math.sqrt(vec @ GE @ vec)
    if vec[0] < 0:
        vec = -vec
    return float(w[0]), vec


def delta_A(rho, q):
    disc = max(1.0 + rho * rho - q * q, 0.0)
    return max((-q * rho + math.sqrt(disc)) / (1.0 + rho * rho), 0.0)


def step(x, mpo, prec, params, state):
    """One pass of the loop body of Alg. 2.  Returns (x_next, info).  When the
    termination test holds, x_next is the normalised x^n and info['converged']."""
    lam, num, den = rayleigh(x, prec, mpo)
    x = B.scale(x, 1.0 / math.sqrt(num))                 # x / ||x||_A
    zeta = params.zeta_res
    terms = residual_terms(x, lam, prec, mpo)
    sum_norms = sum(e[2] for e in terms)
    eta = min(2.0 * state.eta_res, 0.8 * zeta * sum_norms)
    tries = 0
    while True:
        r = assemble_residual(terms, eta)
        rnorm = 0.0 if r is None else B.norm(r)
        if rnorm >= (1.0 + 1.0 / zeta) * eta or tries >= MAX_ETA_RETRIES:
            break
        eta *= 0.8
        tries += 1
    state.eta_res = eta
    rho = (rnorm + eta) / math.sqrt(1.0 - params.c)     # ||x||_A = 1
    bound = eigvec_bound(rho, params.delta)
    info = {"n": state.n, "lambda": lam, "rho": rho, "eta_res": eta,
            "res_norm": rnorm, "eta_tries": tries, "bound": bound,
            "releig_bound": releig_bound(rho, params.delta), "converged": False}
    if bound <= params.tau or r is None:
        info["converged"] = True
        state.history.append(info)
        return x, info
    # 2x2 Rayleigh-Ritz on span{x, r} in the normalised basis (Remark omegamin)
    vecs = [x, r]
    GH = np.zeros((2, 2))
    GE = np.zeros((2, 2))
    for i in range(2):
        for j in range(2):
            GH[i, j] = pair_sums(vecs[i], vecs[j], prec, mpo)
            GE[i, j] = pair_sums(vecs[i], vecs[j], prec, None)
    nrm = np.sqrt(np.diag(GE))
    GHn = GH / np.outer(nrm, nrm)
    GEn = GE / np.outer(nrm, nrm)
    lam_star, v = rr2(GHn, GEn)
    c1, c2 = v[0] / nrm[0], v[1] / nrm[1]
    xstar = B.add(x, r, c1, c2)
    xstar_A = math.sqrt(max(lam_star, 0.0))
    q = math.sqrt(lam_star / (lam_star + params.t_eig * (lam - lam_star)))
    dA = delta_A(rho, q)
    eta_in = dA * xstar_A / math.sqrt(1.0 + params.c)
    xnext, _, cap = B.truncate(xstar, eta_in, params.r_max)
    info.update({"lambda_star": lam_star, "omega": -c2 / c1, "eta_in": eta_in,
                 "delta_A": dA, "ranks": xnext.ranks(), "cap_discarded": cap})
    state.history.append(info)
    state.n += 1
    return xnext, info


def outer_constants(c, K, alpha):
    """kappa of Eq. (kappadef) and theta of Thm. quasioptr."""
    kappa = math.sqrt((1.0 + c) / (1.0 - c)) * math.sqrt(K - 1)
    theta = (1.0 + alpha) * kappa / (2.0 * (1.0 + (1.0 + alpha) * kappa))
    return kappa, theta


def outer(y0, mpo, prec, params, tau, alpha=1.0, max_outer=20, max_inner=100, keep=False):
    """Outer perturbed inverse iteration (Alg. 3), D = 1.

    eta_0 = 1/(2 theta); in outer step m the inner iteration (Alg. 2, fresh
    state) runs from y^m until its eigenvector bound is at most
    tau_m = eta_m / (2 (1 + (1 + alpha) kappa)); the outer iteration stops when
    the relative eigenvalue bound of Eq. (releigerr) at the inner result is
    below tau, else y^{m+1} = trunc_{theta eta_m}(y^+) (Euclidean tolerance, as
    trunc is defined in Sec. 2.2) and eta_{m+1} = eta_m / 2.

    Readings: alpha is not fixed by the paper (alpha = 1 by default); the rank
    cap params.r_max applies inside the inner iteration only.
    Returns (y, records, converged); records[m] holds the inner step count,
    lambda, rho and bounds at y^+, eta_m, tau_m, and the ranks after the outer
    truncation (keep=True: also y^+ and y^{m+1})."""
    kappa, theta = outer_constants(params.c, y0.K, alpha)
    eta = 1.0 / (2.0 * theta)
    y = y0
    records = []
    for m in range(max_outer):
        tau_m = eta / (2.0 * (1.0 + (1.0 + alpha) * kappa))
        inner = SolverParams(params.c, params.delta, params.eps_num, params.t_eig, tau_m, params.r_max)
        st = SolverState()
        info = None
        n_inner = 0
        for _ in range(max_inner):
            y, info = step(y, mpo, prec, inner, st)
            n_inner += 1
            if info["converged"]:
                break
        rec = {"m": m, "inner_steps": n_inner, "inner_converged": bool(info["converged"]),
               "lambda": info["lambda"], "rho": info["rho"], "bound": info["bound"],
               "releig_bound": info["releig_bound"], "eta_out": eta, "tau_m": tau_m,
               "ranks_before": y.ranks()}
        if keep:
            rec["y_plus"] = y
        if info["releig_bound"] < tau:
            rec["ranks_after"] = y.ranks()
            records.append(rec)
            return y, records, True
        y, _, _ = B.truncate(y, theta * eta)
        rec["ranks_after"] = y.ranks()
        if keep:
            rec["y_next"] = y
        records.append(rec)
        eta *= 0.5
    return y, records, False
