"""Problem set-up for the solver: shift gamma, the diagonal D of the
preconditioner and the bounds of its spectrum (host-side scalars).

* gamma: H_gamma = H + gamma I must be positive definite (Sec. 3.1).  For
  two-electron integrals of the form (pq|rs) = sum_g L^g_pq L^g_rs (positive
  semidefinite) or an on-site U >= 0, H >= the one-body part minus the
  normal-ordering term, so E_0 >= E_lb with E_lb the sum of the lowest
  single-particle levels of h - 1/2 sum_g (L^g)^2 per species.  For the
  Hubbard model (U >= 0) the interaction is nonnegative and E_lb is the
  free-fermion ground energy.  gamma = margin - E_lb makes lambda_1 >= margin.
* d_i = theta_i = gamma/N + t_ii + sum_{j=k_i+1}^{k_i+N} (v_ijji - v_ijij),
  k_i = max(0, i-N) (1-based, Sec. 7.1.1), with v_ijkl = 1/2 (il|jk).
* t_min / t_max: sums of the N_s smallest / largest d_i of each species
  (the spectrum of D on the N-particle space).
"""

import itertools
import math

import numpy as np


def spin_orbital_pairs(n_orb, spin):
    if spin:
        return [(i // 2, i % 2) for i in range(2 * n_orb)]
    return [(i, 0) for i in range(n_orb)]


def free_fermion_bound(h, n_up, n_dn, spin):
    ev = np.sort(np.linalg.eigvalsh(h))
    if spin:
        return float(ev[:n_up].sum() + ev[:n_dn].sum())
    return float(ev[:n_up].sum())


def hubbard_shift(h, n_up, n_dn, margin=1.0):
    """gamma for U >= 0 on-site interactions."""
    return margin - free_fermion_bound(h, n_up, n_dn, 1)


def cholesky_shift(h, eri, n_up, n_dn, spin, margin=1.0):
    """gamma for PSD (pq|rs): H >= sum_pq (h_pq - 1/2 sum_r (pr|rq)) a_p^* a_q."""
    hk = h - 0.5 * np.einsum("prrq->pq", eri)
    return margin - free_fermion_bound(hk, n_up, n_dn, spin)


def theta_diagonal(h, eri, spin, n_particles, gamma):
    so = spin_orbital_pairs(h.shape[0], spin)
    K = len(so)
    N = n_particles

    def v(i, j, k, l):
        (pi, si), (pj, sj), (pk, sk), (pl, sl) = so[i], so[j], so[k], so[l]
        if si != sl or sj != sk:
            return 0.0
        return 0.5 * eri[pi, pl, pj, pk]

    th = np.zeros(K)
    for i1 in range(1, K + 1):
        i = i1 - 1
        pi, si = so[i]
        acc = gamma / N + h[pi, pi]
        ki = max(0, i1 - N)
        for j1 in range(ki + 1, ki + N + 1):
            j = j1 - 1
            acc += v(i, j, j, i) - v(i, j, i, j)
        th[i] = acc
    return th


def spectrum_bounds(theta, spin, n_up, n_dn, h=None):
    """t_min / t_max of the exponential-sum interval.  With the one-body matrix
    h given and its diagonal strictly increasing along a species' sites (the
    paper's orbital basis), the sums of theta over that species' first / last
    n sites (t_min = D at e_1, as the printed t_min, t_max and T of Sec. 7.2
    require); otherwise the sums of the n smallest / largest theta (the range
    of the spectrum of D)."""
    lo = hi = 0.0
    K = len(theta)
    diag = None
    if h is not None:
        d = np.diag(np.asarray(h, dtype=np.float64))
        diag = np.repeat(d, 2) if spin else d
    groups = [(np.arange(0, K, 2), n_up), (np.arange(1, K, 2), n_dn)] if spin else [(np.arange(K), n_up)]
    for idx, n in groups:
        if not n:
            continue
        vals = np.asarray(theta)[idx]
        if diag is None or not np.all(np.diff(diag[idx]) > 0):
            vals = np.sort(vals)
        lo += float(np.sum(vals[:n]))
        hi += float(np.sum(vals[-n:]))
    return lo, hi


def lowest_determinants(t_diag, spin, n_up, n_dn, D, max_configs=2_000_000):
    """Occupation strings (D x K, uint8) of the D determinants with the smallest
    diagonal one-particle energy sum_{i occupied} t_diag[i], the start of the
    subspace iteration (Sec. 7.1.4 uses e_1, ..., e_D).  Ties: occupation strings
    compared from site 0, occupied first (so the first string is e_1 when t_diag
    increases).  Energies are summed over the occupied sites in site order.
    The sector is enumerated: at most max_configs strings."""
    t_diag = [float(v) for v in t_diag]
    K = len(t_diag)
    species = [(i % 2) if spin else 0 for i in range(K)]
    want = [n_up, n_dn if spin else 0]
    pools = [[i for i in range(K) if species[i] == s] for s in (0, 1)]
    total = 1
    for s in (0, 1):
        total *= math.comb(len(pools[s]), want[s])
    if total > max_configs:
        raise ValueError(f"sector of {total} determinants is too large to enumerate")
    if total < D:
        raise ValueError("sector smaller than D")
    rows = []
    for a in itertools.combinations(pools[0], want[0]):
        for b in itertools.combinations(pools[1], want[1]):
            occ = bytearray(K)
            for i in a:
                occ[i] = 1
            for i in b:
                occ[i] = 1
            e = 0.0
            for i in range(K):
                if occ[i]:
                    e += t_diag[i]
            rows.append((e, bytes(1 - o for o in occ), bytes(occ)))
    rows.sort()
    return np.array([list(r[2]) for r in rows[:D]], dtype=np.uint8)
